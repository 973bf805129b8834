"""Mie series for spheres: perfectly conducting, homogeneous (possibly lossy) dielectric,
and a PEC core under a dielectric coat.  These are the reference solutions of Sec. III.A
(coated PEC sphere, RCS error of Eq. 5-25), for the lossy coating permittivity of Sec. III.D
(2.0 - 0.5j).

TEST INFRASTRUCTURE ONLY.

Bistatic scattering of a plane wave polarised along x and propagating along +z.  The series
is written in the exp(-i w t) convention of the classical treatment: psi_n(z) = z j_n(z),
zeta_n(z) = z y_n(z), xi_n(z) = z h_n^(1)(z), all of integer order from scipy.special
(library primitive).  A permittivity eps_r given in the exp(j w t) convention of the rest of
this project (loss: Im eps_r < 0) enters as its conjugate, relative index m = sqrt(conj eps_r)
with Re m > 0 (loss: Im m > 0).  |S1|, |S2| and so the RCS are the same in both conventions.

Coefficients from the boundary conditions of the Debye potentials u(rho), rho = m k r:
  TE (b_n): u and m u' continuous across an interface,  u = 0 on a PEC surface;
  TM (a_n): u and u' / m continuous,                     u' = 0 on a PEC surface.
Outside: u = psi_n(k r) - c xi_n(k r) with c = b_n (TE) or a_n (TM).  With the ratio
Q = u_in / (m u_in') (TE) or P = u_in' / (m u_in) (TM) of the inside solution at the outer
radius (x = k b):  b_n = (psi - Q psi') / (xi - Q xi'),  a_n = (psi' - P psi) / (xi' - P xi).
Amplitudes S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n), S2 = sum (2n+1)/(n(n+1))
(a_n tau_n + b_n pi_n), pi_n and tau_n from their three-term recurrences, and
sigma(t, phi) = (4 pi / k^2) (|S2|^2 cos^2 phi + |S1|^2 sin^2 phi), t from the forward direction.
"""
import numpy as np
from scipy import special


def _nmax(x):
    x = abs(x)
    return int(np.ceil(x + 4.05 * x ** (1 / 3) + 2)) + 10


def _riccati(n, z):
    """psi, psi', zeta, zeta' of (complex) argument z."""
    jn = special.spherical_jn(n, z)
    jnp = special.spherical_jn(n, z, derivative=True)
    yn = special.spherical_yn(n, z)
    ynp = special.spherical_yn(n, z, derivative=True)
    return z * jn, jn + z * jnp, z * yn, yn + z * ynp


def _outer(n, x, Q, P):
    """a_n, b_n from the inside ratios at the outer radius (see the module docstring)."""
    psi, dpsi, zeta, dzeta = _riccati(n, x)
    xi, dxi = psi + 1j * zeta, dpsi + 1j * dzeta
    b = (psi - Q * dpsi) / (xi - Q * dxi)
    a = (dpsi - P * psi) / (dxi - P * xi)
    return a, b


def index(eps_r):
    """Relative index of the classical convention for eps_r given with exp(j w t)."""
    m = np.sqrt(np.conj(complex(eps_r)))
    return m if m.real > 0 else -m


def coeffs_pec(x, nmax=None):
    """PEC sphere of size parameter x = k a: the inside ratios are those of u = 0 / u' = 0."""
    n = np.arange(1, (nmax or _nmax(x)) + 1)
    psi, dpsi, zeta, dzeta = _riccati(n, x)
    xi, dxi = psi + 1j * zeta, dpsi + 1j * dzeta
    return n, dpsi / dxi, psi / xi


def _log_derivative(z, nmax):
    """D_n(z) = psi_n'(z) / psi_n(z), n = 1..nmax, by the downward recurrence
    D_{n-1} = n/z - 1/(D_n + n/z), which follows from psi_n' = psi_{n-1} - (n/z) psi_n and
    psi_{n-1}' = (n/z) psi_{n-1} - psi_n.  Started far above nmax, it stays finite for any
    complex z (no growing Bessel functions of a lossy argument)."""
    start = int(max(nmax, abs(z))) + 30
    D = np.zeros(start + 1, complex)
    for n in range(start, 0, -1):
        D[n - 1] = n / z - 1.0 / (D[n] + n / z)
    return D[1:nmax + 1]


def coeffs_dielectric(x, eps_r, nmax=None):
    """Homogeneous sphere, x = k a, relative permittivity eps_r (exp(j w t)): the inside
    solution is psi_n(m k r), so Q = 1 / (m D_n(m x)) and P = D_n(m x) / m."""
    m = index(eps_r)
    n = np.arange(1, (nmax or _nmax(x)) + 1)
    D = _log_derivative(m * x, len(n))
    a, b = _outer(n, x, 1.0 / (m * D), D / m)
    return n, a, b


def coeffs_coated_pec(x_core, x_outer, eps_r, nmax=None):
    """PEC core of size parameter x_core = k a under a coat of permittivity eps_r out to
    x_outer = k b.  In the coat u = psi(rho) + beta zeta(rho), beta fixed at the core."""
    m = index(eps_r)
    n = np.arange(1, (nmax or _nmax(abs(m) * x_outer)) + 1)
    psi_a, dpsi_a, zeta_a, dzeta_a = _riccati(n, m * x_core)
    beta_te = -psi_a / zeta_a          # u(m k a) = 0
    beta_tm = -dpsi_a / dzeta_a        # u'(m k a) = 0
    psi_b, dpsi_b, zeta_b, dzeta_b = _riccati(n, m * x_outer)
    Q = (psi_b + beta_te * zeta_b) / (m * (dpsi_b + beta_te * dzeta_b))
    P = (dpsi_b + beta_tm * dzeta_b) / (m * (psi_b + beta_tm * zeta_b))
    a, b = _outer(n, x_outer, Q, P)
    return n, a, b


def _pitau(mu, nmax):
    pi = np.zeros((nmax + 1,) + np.shape(mu))
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) / (n - 1)) * mu * pi[n - 1] - (n / (n - 1)) * pi[n - 2]
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def _amplitudes(n, a, b, theta):
    mu = np.cos(np.asarray(theta, float))
    pi, tau = _pitau(mu, len(n))
    f = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(f * (a[:, None] * pi + b[:, None] * tau), 0)
    S2 = np.sum(f * (a[:, None] * tau + b[:, None] * pi), 0)
    return S1, S2


def _rcs(k, coeffs, theta, phi):
    S1, S2 = _amplitudes(*coeffs, theta)
    return (4 * np.pi / k ** 2) * (np.abs(S2) ** 2 * np.cos(phi) ** 2 + np.abs(S1) ** 2 * np.sin(phi) ** 2)


def amplitudes(ka, theta):
    """S1, S2 of a PEC sphere at scattering angles theta (radians from forward)."""
    return _amplitudes(*coeffs_pec(ka), theta)


def rcs_pec(k, radius, theta, phi=0.0):
    """Bistatic RCS (area units) of a PEC sphere, incidence along +z polarised along x."""
    return _rcs(k, coeffs_pec(k * radius), theta, phi)


def rcs_dielectric(k, radius, eps_r, theta, phi=0.0):
    """Bistatic RCS of a homogeneous sphere of permittivity eps_r (exp(j w t) convention)."""
    return _rcs(k, coeffs_dielectric(k * radius, eps_r), theta, phi)


def rcs_coated_pec(k, core_radius, outer_radius, eps_r, theta, phi=0.0):
    """Bistatic RCS of a PEC sphere of radius core_radius coated out to outer_radius."""
    return _rcs(k, coeffs_coated_pec(k * core_radius, k * outer_radius, eps_r), theta, phi)


def efficiencies_from(x, coeffs):
    """Extinction (forward amplitude, optical theorem), scattering and absorption
    efficiencies of a sphere of outer size parameter x."""
    n, a, b = coeffs
    qsca = (2 / x ** 2) * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    S1, _ = _amplitudes(n, a, b, np.array([0.0]))
    qext = (4 / x ** 2) * np.real(S1[0])
    return qext, qsca, qext - qsca


def efficiencies(ka):
    """Extinction and scattering efficiencies of a PEC sphere."""
    qe, qs, _ = efficiencies_from(ka, coeffs_pec(ka))
    return qe, qs
