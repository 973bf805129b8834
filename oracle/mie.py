"""Mie series for a perfectly conducting sphere (reference solution of Sec. III.A,
used with the RCS error of Eq. 5-25).

TEST INFRASTRUCTURE ONLY.

Bistatic scattering of a plane wave E = x exp(-jk z) (propagating along +z) by a PEC
sphere of radius a.  With Riccati-Bessel functions psi_n(x) = x j_n(x) and
xi_n(x) = x h_n(x) (the outgoing spherical Hankel function of the chosen time
convention; |coefficients| do not depend on it), the series coefficients are
    a_n = psi_n'(ka) / xi_n'(ka),     b_n = psi_n(ka) / xi_n(ka),
the amplitude functions
    S1(t) = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),
    S2(t) = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n),
with pi_n = P_n^1(cos t)/sin t and tau_n = d P_n^1(cos t)/dt from their three-term
recurrences, and the RCS
    sigma(t, phi) = (4 pi / k^2) (|S2|^2 cos^2 phi + |S1|^2 sin^2 phi),
t the angle from the forward (+z) direction.  Bessel functions of integer order come
from scipy.special (library primitive).
"""
import numpy as np
from scipy import special


def _coeffs(x, nmax):
    n = np.arange(1, nmax + 1)
    jn = special.spherical_jn(n, x)
    yn = special.spherical_yn(n, x)
    jnp = special.spherical_jn(n, x, derivative=True)
    ynp = special.spherical_yn(n, x, derivative=True)
    hn = jn - 1j * yn
    hnp = jnp - 1j * ynp
    psi = x * jn
    dpsi = jn + x * jnp
    xi = x * hn
    dxi = hn + x * hnp
    return n, dpsi / dxi, psi / xi


def _pitau(mu, nmax):
    pi = np.zeros((nmax + 1,) + np.shape(mu))
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) / (n - 1)) * mu * pi[n - 1] - (n / (n - 1)) * pi[n - 2]
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def amplitudes(ka, theta):
    """S1, S2 at scattering angles theta (radians from forward)."""
    nmax = int(np.ceil(ka + 4.05 * ka ** (1 / 3) + 2)) + 10
    n, a, b = _coeffs(ka, nmax)
    mu = np.cos(np.asarray(theta, float))
    pi, tau = _pitau(mu, nmax)
    f = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(f * (a[:, None] * pi + b[:, None] * tau), 0)
    S2 = np.sum(f * (a[:, None] * tau + b[:, None] * pi), 0)
    return S1, S2


def rcs_pec(k, radius, theta, phi=0.0):
    """Bistatic RCS (area units) of a PEC sphere, incidence along +z polarised along x."""
    S1, S2 = amplitudes(k * radius, theta)
    return (4 * np.pi / k ** 2) * (np.abs(S2) ** 2 * np.cos(phi) ** 2 + np.abs(S1) ** 2 * np.sin(phi) ** 2)


def efficiencies(ka):
    """Extinction (from the forward amplitude, optical theorem) and scattering efficiencies."""
    nmax = int(np.ceil(ka + 4.05 * ka ** (1 / 3) + 2)) + 10
    n, a, b = _coeffs(ka, nmax)
    qsca = (2 / ka ** 2) * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    S1, _ = amplitudes(ka, np.array([0.0]))
    qext = (4 / ka ** 2) * np.real(S1[0])
    return qext, qsca
