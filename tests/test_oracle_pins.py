"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, brute-force quadrature, operator invariants, the Mie series, the
structure of Eqs. 43-46 and the addition theorem behind the plane-wave expansion."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import mie
from paper_2210_04892_gb300.inputs import icosphere

K0 = 2 * np.pi
HERE = os.path.dirname(os.path.abspath(__file__))


def _sub(T, s):
    if s == 0:
        return [T]
    m01, m12, m20 = (T[0] + T[1]) / 2, (T[1] + T[2]) / 2, (T[2] + T[0]) / 2
    out = []
    for t in ([T[0], m01, m20], [m01, T[1], m12], [m20, m12, T[2]], [m01, m12, m20]):
        out += _sub(np.array(t), s - 1)
    return out


def _brute_rule(T, s=3, n=30):
    """Points and weights of a subdivided high-order rule over triangle T (numpy, independent)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = (x + 1) / 2
    w = w / 2
    U, V = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    b1 = U.ravel()
    b2 = ((1 - U) * V).ravel()
    ww = (WU * WV * (1 - U)).ravel() * 2
    pts, wts = [], []
    for t in _sub(np.asarray(T, float), s):
        a = np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0])) / 2
        pts.append(t[0] + b1[:, None] * (t[1] - t[0]) + b2[:, None] * (t[2] - t[0]))
        wts.append(ww * a)
    return np.concatenate(pts), np.concatenate(wts)


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("n", [3, 5, 8])
def test_conical_rule_exact(n):
    b, w = oracle.rule(0, n)
    assert abs(w.sum() - 1) < 1e-14
    deg = 2 * n - 2
    for a in range(deg + 1):
        for c in range(deg + 1 - a):
            exact = 2 * math.factorial(a) * math.factorial(c) / math.factorial(a + c + 2)
            assert abs(np.sum(w * b[:, 1] ** a * b[:, 2] ** c) - exact) < 1e-13


@pytest.mark.parametrize("kind", [1, 2])
def test_graded_rules_integrate_polynomials(kind):
    b, w = oracle.rule(kind, 14, 3)
    assert abs(w.sum() - 1) < 1e-12
    for a, c in ((1, 0), (0, 1), (2, 1), (1, 3)):
        exact = 2 * math.factorial(a) * math.factorial(c) / math.factorial(a + c + 2)
        assert abs(np.sum(w * b[:, 1] ** a * b[:, 2] ** c) - exact) < 1e-9


# ---------------------------------------------------- closed-form static parts
P_TRI = np.array([[0, 0, 0], [1, 0, 0], [0.2, 0.9, 0]], float)


@pytest.mark.parametrize("r", [[0.3, 0.3, 0.5], [0.3, 0.3, -0.2], [1.5, 0.4, 0.3], [-0.5, -0.5, 0.05],
                               [0.4, -0.3, 0.0], [0.3, 0.2, 0.1]])
def test_static_integrals_vs_brute_force(r):
    r = np.array(r, float)
    I1, Ir, Ig = oracle.static_tri(P_TRI, r)
    x, w = _brute_rule(P_TRI)
    d = x - r
    R = np.linalg.norm(d, axis=1)
    rho = r.copy()
    rho[2] = 0.0
    b1 = np.sum(w / R)
    br = np.sum(w[:, None] * (x - rho) / R[:, None], 0)
    bg = np.sum(w[:, None] * d / R[:, None] ** 3, 0)
    assert abs(I1 - b1) / b1 < 1e-9
    assert np.linalg.norm(Ir - br) / np.linalg.norm(br) < 1e-9
    assert np.linalg.norm(Ig - bg) / np.linalg.norm(bg) < 1e-8


def test_static_solid_angle_jump():
    """The normal part of int grad(1/R) is the solid angle: -2pi n just above an interior point."""
    r_up = np.array([0.3, 0.3, 1e-9])
    r_dn = np.array([0.3, 0.3, -1e-9])
    _, _, gu = oracle.static_tri(P_TRI, r_up)
    _, _, gd = oracle.static_tri(P_TRI, r_dn)
    assert abs(gu[2] + 2 * np.pi) < 1e-6 and abs(gd[2] - 2 * np.pi) < 1e-6


# -------------------------------------------------------------------- Gram
def _gram_closed(v, t, E):
    """Gram and twisted Gram from int lambda_a lambda_b = A (1 + delta_ab) / 12."""
    N = len(E["edges"])
    G = np.zeros((N, N))
    X = np.zeros((N, N))
    for tri in range(len(t)):
        p = v[t[tri]]
        nn = np.cross(p[1] - p[0], p[2] - p[0])
        A = np.linalg.norm(nn) / 2
        nn = nn / (2 * A)
        funcs = []
        for e in range(N):
            for side, tt, loc in ((1, E["tplus"][e], E["lplus"][e]), (-1, E["tminus"][e], E["lminus"][e])):
                if tt == tri:
                    l = np.linalg.norm(v[E["edges"][e][1]] - v[E["edges"][e][0]])
                    funcs.append((e, side * l / (2 * A), p[loc]))
        for (m, cm, a) in funcs:
            for (n, cn, b) in funcs:
                qa, qb = p - a, p - b
                g = (A / 12) * (np.sum(qa * qb) + np.dot(qa.sum(0), qb.sum(0)))
                qbx = np.cross(nn, qb)
                x = (A / 12) * (np.sum(qa * qbx) + np.dot(qa.sum(0), qbx.sum(0)))
                G[m, n] += cm * cn * g
                X[m, n] += cm * cn * x
    return G, X


def test_gram_closed_form_and_invariants():
    v, t = icosphere(1, 1.0)
    E = oracle.rwg(v, t)
    G, X = oracle.gram(v, t)
    Gc, Xc = _gram_closed(v, t, E)
    assert np.abs(G - Gc).max() < 1e-13
    assert np.abs(X - Xc).max() < 1e-13
    assert np.abs(G - G.T).max() < 1e-14
    assert np.abs(X + X.T).max() < 1e-14
    assert np.linalg.eigvalsh(G).min() > 0


def test_rwg_unit_right_triangle_hand_values():
    """int_T (r - a).(r - b) on the unit right triangle (0,0,0),(1,0,0),(0,1,0):
    int r.r = 1/6, int r = (1/6, 1/6, 0), area 1/2 (hand computation)."""
    p = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    a, b = p[1], p[2]
    hand = 1 / 6 - np.dot(a + b, [1 / 6, 1 / 6, 0]) + 0.5 * np.dot(a, b)
    qa, qb = p - a, p - b
    closed = (0.5 / 12) * (np.sum(qa * qb) + np.dot(qa.sum(0), qb.sum(0)))
    assert abs(hand - closed) < 1e-15


# ------------------------------------------------------------------ meshes
def test_rwg_rejects_bad_meshes():
    v, t = icosphere(1, 1.0)
    with pytest.raises(oracle.MeshError):
        oracle.rwg(v, t[:-1])                       # open surface
    t2 = t.copy()
    t2[0] = t2[0][[0, 2, 1]]
    with pytest.raises(oracle.MeshError):
        oracle.rwg(v, t2)                           # flipped triangle
    E = oracle.rwg(v, t)
    assert len(E["edges"]) == 30
    e = E["edges"]
    assert np.all(e[:, 0] < e[:, 1])
    assert np.all(np.diff(e[:, 0] * 1000 + e[:, 1]) > 0)


def test_table_mesh_size_convention():
    g = json.load(open(os.path.join(HERE, "golden", "table_t5_0.json")))
    for row in g["rows"]:
        # icosphere frequency giving this mean edge on radius 0.4
        def mean_edge(nu):
            v, t = icosphere(nu, g["radius_lambda"])
            p = v[t]
            return np.mean(np.linalg.norm(p - np.roll(p, 1, axis=1), axis=2))
        nu = min(range(2, 20), key=lambda n: abs(mean_edge(n) - row["edge_lambda"]))
        v, t = icosphere(nu, g["radius_lambda"])
        nbi = 2 * (3 * len(t) // 2)
        assert abs(nbi - row["N_BI"]) / row["N_BI"] < 0.25


# --------------------------------------------------------- operator invariants
@pytest.fixture(scope="module")
def ops_small():
    v, t = icosphere(4, 0.5)
    return v, t, oracle.operators(v, t, K0, 0)


def test_L_is_complex_symmetric(ops_small):
    _, _, (L, NL, K, NK) = ops_small
    assert np.linalg.norm(L - L.T) / np.linalg.norm(L) < 1e-7


def test_Kbar_is_symmetric(ops_small):
    """<f_m, Kbar f_n> = <f_n, Kbar f_m> (a.(b x c) and grad_r' G = -grad_r G)."""
    _, _, (L, NL, K, NK) = ops_small
    assert np.linalg.norm(K - K.T) / np.linalg.norm(K) < 1e-5


def test_static_limit_of_L():
    """k -> 0: the divergence part dominates, k^2 <f,Lf> -> j (1/4pi) int int div f div f / R."""
    v, t = icosphere(2, 0.5)
    kk = 1e-3
    L, _, _, _ = oracle.operators(v, t, kk, 0)
    L2, _, _, _ = oracle.operators(v, t, 2 * kk, 0)
    # j k <f, L f> tends to a k-independent real matrix times -1 (static charge term)
    A1, A2 = kk * L, 2 * kk * L2
    assert np.linalg.norm(A1 - A2) / np.linalg.norm(A1) < 1e-4
    assert np.linalg.norm(A1.real) / np.linalg.norm(A1.imag) < 1e-3


def _brute_blocks(Pm, Pn, k):
    """Raw blocks of one well-separated triangle pair by brute-force product quadrature
    of the surface forms (numpy; shares nothing with the C oracle)."""
    xm, wm = _brute_rule(Pm, s=2, n=12)
    xn, wn = _brute_rule(Pn, s=2, n=12)
    nm = np.cross(Pm[1] - Pm[0], Pm[2] - Pm[0])
    nm /= np.linalg.norm(nm)
    d = xn[None, :, :] - xm[:, None, :]          # r' - r
    R = np.linalg.norm(d, axis=2)
    G = np.exp(-1j * k * R) / (4 * np.pi * R)
    gt = (1 + 1j * k * R) * np.exp(-1j * k * R) / (4 * np.pi * R ** 3)
    gradG = d * gt[:, :, None]                    # grad_r G
    W = wm[:, None] * wn[None, :]
    out = np.zeros((4, 3, 3), complex)
    for i in range(3):
        gi = xm - Pm[i]
        ngi = np.cross(nm, gi)
        for j in range(3):
            gj = xn - Pn[j]
            gg = gi @ gj.T
            out[0, i, j] = -1j * k * np.sum(W * G * (gg - 4 / k ** 2))
            ngj = np.cross(nm[None, :], gj)
            t1 = gi @ ngj.T
            t2 = np.einsum("ad,abd->ab", ngi, gradG) * 2 * (1j / k)
            out[1, i, j] = np.sum(W * (-1j * k * G * t1 + t2))
            cr = np.cross(gradG, gj[None, :, :])
            out[2, i, j] = np.sum(W * np.einsum("ad,abd->ab", gi, cr))
            ncr = np.cross(nm[None, None, :], cr)
            out[3, i, j] = np.sum(W * np.einsum("ad,abd->ab", gi, ncr))
    return out


@pytest.mark.parametrize("offset", [[0.0, 0.05, 0.08], [0.2, -0.1, 0.15], [0.9, 0.3, -0.4]])
def test_pair_blocks_vs_brute_force(offset):
    """Separated pairs: the singularity-subtraction path (and for the closest pair the
    boundary form of the grad-Phi term) must agree with brute-force surface quadrature."""
    Pm = np.array([[0, 0, 0], [0.08, 0, 0], [0.02, 0.07, 0.01]], float)
    Pn = np.array([[0, 0, 0], [0.07, 0.01, 0.02], [0.01, 0.08, -0.01]], float) + np.array(offset)
    ours = oracle.pair_blocks(Pm, Pn, [0, 1, 2], [3, 4, 5], K0, 1)
    ref = _brute_blocks(Pm, Pn, K0)
    for q in range(4):
        err = np.abs(ours[q] - ref[q]).max() / np.abs(ref[q]).max()
        assert err < 2e-6, (q, err)


def test_same_triangle_kbar_vanishes():
    P = np.array([[0, 0, 0], [0.08, 0, 0], [0.02, 0.07, 0.0]], float)
    b = oracle.pair_blocks(P, P, [0, 1, 2], [0, 1, 2], K0, 0)
    assert np.abs(b[2]).max() == 0 and np.abs(b[3]).max() == 0


def test_quadrature_convergence_on_sphere_rows():
    v, t = icosphere(8, 0.5)
    rows = np.arange(0, 3840, 211).astype(np.int32)
    Z0 = oracle.rows(v, t, K0, 0, rows, 0)
    Z2 = oracle.rows(v, t, K0, 0, rows, 2)
    assert np.linalg.norm(Z0 - Z2) / np.linalg.norm(Z2) < 1e-6


# ------------------------------------------------- structure of Eqs. 43-46
def test_block_structure_of_C():
    """Z_JJ - Z_MM = G/2, Z_JM + Z_MJ = X/2, and the PEC matrix is Z_JJ - 3G/4."""
    v, t = icosphere(3, 0.5)
    Z0 = oracle.fill(v, t, K0, 0)
    Z1 = oracle.fill(v, t, K0, 1)
    G, X = oracle.gram(v, t)
    N = len(G)
    JJ, JM, MJ, MM = Z0[:N, :N], Z0[:N, N:], Z0[N:, :N], Z0[N:, N:]
    s = np.abs(Z0).max()
    assert np.abs(JJ - MM - G / 2).max() < 1e-12 * s
    assert np.abs(JM + MJ - X / 2).max() < 1e-12 * s
    assert np.abs(JJ - 0.75 * G - Z1).max() < 1e-12 * s


def test_rows_match_full_fill():
    v, t = icosphere(3, 0.5)
    Z0 = oracle.fill(v, t, K0, 0)
    rows = np.array([0, 5, 17, 90, 150, 179], np.int32)
    Zr = oracle.rows(v, t, K0, 0, rows)
    assert np.abs(Zr - Z0[rows]).max() < 1e-14 * np.abs(Z0).max()


# ----------------------------------------------------------------- Mie
def test_mie_rayleigh_limit_and_optical_theorem():
    ka = 0.05
    sb = mie.rcs_pec(ka, 1.0, np.array([np.pi]))[0] / np.pi
    assert abs(sb / (9 * ka ** 4) - 1) < 2e-3     # PEC sphere backscatter ~ 9 (ka)^4 pi a^2
    for ka in (0.5, 1.0, np.pi, 10.0):
        qe, qs = mie.efficiencies(ka)
        assert abs(qe - qs) < 1e-10                # lossless scatterer: extinction = scattering
    assert abs(mie.rcs_pec(60.0, 1.0, np.array([np.pi]))[0] / np.pi - 1) < 0.05   # optical limit


@pytest.mark.slow
def test_pec_sphere_rcs_vs_mie():
    """PEC combined-field solve on the 1280-triangle sphere of radius 0.5 lambda (ka = pi)
    reproduces the Mie RCS within 0.5 dB over the lit range (Sec. III.A error metric)."""
    v, t = icosphere(8, 0.5)
    Z = oracle.fill(v, t, K0, 1)
    b = oracle.rhs_planewave(v, t, K0, 1, [0, 0, 1.0], [1.0, 0, 0])[0]
    x = np.linalg.solve(Z, b)
    th = np.deg2rad(np.arange(0, 181))
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    s = oracle.rcs(v, t, K0, 1, x, dirs)
    sm = mie.rcs_pec(K0, 0.5, th)
    mask = 10 * np.log10(sm) >= 10 * np.log10(sm.max()) - 20
    assert np.abs(10 * np.log10(s / sm))[mask].max() < 0.5
    assert oracle.rcs_error(s, sm) < 0.05


# ---------------------------------------------------- addition theorem
def _hankel2(l, x):
    from scipy import special
    return special.spherical_jn(l, x) - 1j * special.spherical_yn(l, x)


def _expansion_error(digits, a=0.25, k=K0, sign=-1.0, seed=7):
    from scipy import special
    dmax = np.sqrt(3) * a
    kd = float(np.real(k)) * dmax                 # the rule takes Re k for a lossy medium
    L = int(math.ceil(kd + 1.8 * digits ** (2 / 3) * kd ** (1 / 3)))
    x, wx = np.polynomial.legendre.leggauss(L + 1)
    nphi = 2 * (L + 1)
    th = np.arccos(x)
    ph = 2 * np.pi * np.arange(nphi) / nphi
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    W = (wx[:, None] * np.ones(nphi)[None, :] * 2 * np.pi / nphi).ravel()
    KH = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    rng = np.random.default_rng(seed)
    worst = 0
    for X in ([2 * a, 0, 0], [2 * a, 2 * a, 0], [3 * a, -2 * a, 2 * a], [0, 0, -2 * a]):
        X = np.array(X, float)
        Xn = np.linalg.norm(X)
        cosang = KH @ (X / Xn)
        T = np.zeros(len(KH), complex)
        for l in range(L + 1):
            T += (-1j) ** l * (2 * l + 1) * _hankel2(l, k * Xn) * special.eval_legendre(l, cosang)
        for _ in range(20):
            r = (rng.random(3) - 0.5) * a         # receiver relative to its box center
            rp = (rng.random(3) - 0.5) * a        # source relative to its box center
            d = r - rp
            exact = np.exp(-1j * k * np.linalg.norm(X + d)) / (4 * np.pi * np.linalg.norm(X + d))
            approx = (-1j * k / (16 * np.pi ** 2)) * np.sum(W * np.exp(sign * 1j * k * (KH @ d)) * T)
            worst = max(worst, abs(approx - exact) / abs(exact))
    return worst


def test_addition_theorem_plane_wave_expansion():
    """exp(-jk|X+d|)/(4 pi |X+d|) = (-jk/16pi^2) sum_khat w exp(-jk khat.d) T_L(khat, X),
    T_L = sum_l (-j)^l (2l+1) h_l^(2)(k|X|) P_l(khat.Xhat), for boxes of size a one box apart,
    L from the excess-bandwidth rule.  The worst point-pair error tracks the digit count
    and the opposite phase sign fails: this fixes sign and normalisation."""
    e3 = _expansion_error(3)
    e5 = _expansion_error(5)
    assert e3 < 5e-3, e3
    assert e5 < 5e-4 and e5 < e3 / 5, e5
    assert _expansion_error(3, sign=+1.0) > 0.1


# ------------------------------------------- complex wavenumbers and two-region formulations
K_LOSSY = K0 * np.sqrt(2.0 - 0.5j)      # coating permittivity of Sec. III.D, exp(j w t): Im k < 0


def _pair_geometries():
    """Test triangle and source triangles sharing the triangle, an edge or a vertex with it,
    or lying close by (vertex ids decide the relation)."""
    Pm = np.array([[0, 0, 0], [0.08, 0, 0], [0.02, 0.07, 0.01]], float)
    out = {"same": (Pm, [0, 1, 2])}
    out["edge"] = (np.array([Pm[1], Pm[0], [0.05, -0.06, 0.03]]), [1, 0, 3])
    out["vertex"] = (np.array([Pm[2], [-0.03, 0.1, 0.0], [-0.06, 0.04, 0.04]]), [2, 4, 5])
    out["near"] = (np.array([[0, 0, 0], [0.07, 0.01, 0.02], [0.01, 0.08, -0.01]]) + [0.0, 0.05, 0.08], [6, 7, 8])
    return Pm, out


def test_pair_blocks_vs_brute_force_lossy():
    """The separated-pair check (singular subtraction and the boundary form of the grad-Phi
    term, as for a close pair) at the complex wavenumber of a lossy coating."""
    Pm = np.array([[0, 0, 0], [0.08, 0, 0], [0.02, 0.07, 0.01]], float)
    Pn = np.array([[0, 0, 0], [0.07, 0.01, 0.02], [0.01, 0.08, -0.01]], float) + np.array([0.0, 0.05, 0.08])
    ours = oracle.pair_blocks(Pm, Pn, [0, 1, 2], [3, 4, 5], K_LOSSY, 1)
    ref = _brute_blocks(Pm, Pn, K_LOSSY)
    for q in range(4):
        err = np.abs(ours[q] - ref[q]).max() / np.abs(ref[q]).max()
        assert err < 2e-6, (q, err)


@pytest.mark.parametrize("rel", ["same", "edge", "vertex", "near"])
def test_pair_blocks_are_analytic_in_k(rel):
    """Every entry is an analytic function of k (the kernels contain k only through exp(-jkR),
    powers of k and their series), so the Cauchy-Riemann relation d/d(Im k) = j d/d(Re k)
    holds on the singular paths too.  A stray modulus, conjugate or real part of k anywhere
    in the singular subtraction or the boundary term breaks it."""
    Pm, geo = _pair_geometries()
    Pn, idn = geo[rel]
    h = 1e-4 * abs(K_LOSSY)

    def f(k):
        return oracle.pair_blocks(Pm, Pn, [0, 1, 2], idn, k, 0)

    d_re = (f(K_LOSSY + h) - f(K_LOSSY - h)) / (2 * h)
    d_im = (f(K_LOSSY + 1j * h) - f(K_LOSSY - 1j * h)) / (2 * h)
    for q in range(4):
        scale = np.abs(d_re[q]).max()
        if scale == 0:
            assert np.abs(d_im[q]).max() == 0
            continue
        assert np.abs(d_im[q] - 1j * d_re[q]).max() / scale < 1e-6, (rel, q)


def test_operators_symmetric_at_complex_k():
    v, t = icosphere(3, 0.4)
    L, _, K, _ = oracle.operators(v, t, K_LOSSY, 0)
    assert np.linalg.norm(L - L.T) / np.linalg.norm(L) < 1e-7
    assert np.linalg.norm(K - K.T) / np.linalg.norm(K) < 1e-5


def test_mie_dielectric_and_coated_limits():
    """The dielectric and coated series reduce to the PEC series and to each other where
    they must, follow the Rayleigh law, conserve energy without loss and absorb with it."""
    th = np.deg2rad(np.arange(0, 181))
    pec = mie.rcs_pec(K0, 0.3, th)
    assert mie.rcs_dielectric(K0, 0.4, 1.0, th).max() < 1e-25 * pec.max()          # no contrast
    assert np.abs(mie.rcs_coated_pec(K0, 0.3, 0.4, 1.0, th) / pec - 1).max() < 1e-12  # air coat
    assert np.abs(mie.rcs_coated_pec(K0, 0.4, 0.4, 4.0, th) / mie.rcs_pec(K0, 0.4, th) - 1).max() < 1e-12
    hom = mie.rcs_dielectric(K0, 0.4, 2 - 0.5j, th)
    assert np.abs(mie.rcs_coated_pec(K0, 1e-4, 0.4, 2 - 0.5j, th) / hom - 1).max() < 1e-6  # vanishing core
    # a good conductor tends to PEC as 1/|m| (surface impedance)
    e1 = np.abs(mie.rcs_dielectric(K0, 0.4, 1e5 * (1 - 1j), th) / mie.rcs_pec(K0, 0.4, th) - 1).max()
    e2 = np.abs(mie.rcs_dielectric(K0, 0.4, 1e7 * (1 - 1j), th) / mie.rcs_pec(K0, 0.4, th) - 1).max()
    assert e2 < 0.02 and 7 < e1 / e2 < 13
    # Rayleigh: sigma_back = 4 pi k^4 a^6 |(eps - 1)/(eps + 2)|^2
    a, eps = 0.01, 4 - 1j
    sb = mie.rcs_dielectric(1.0, a, eps, np.array([np.pi]))[0]
    assert abs(sb / (4 * np.pi * a ** 6 * abs((eps - 1) / (eps + 2)) ** 2) - 1) < 1e-4
    # energy: no absorption without loss, absorption with Im eps < 0 (exp(j w t))
    for x, e in ((2.5, 4.0), (10.0, 2.25)):
        qe, qs, qa = mie.efficiencies_from(x, mie.coeffs_dielectric(x, e))
        assert abs(qa) < 1e-10 * qe
    qe, qs, qa = mie.efficiencies_from(K0 * 0.4, mie.coeffs_coated_pec(K0 * 0.3, K0 * 0.4, 8.0))
    assert abs(qa) < 1e-10 * qe
    for coeffs in (mie.coeffs_dielectric(K0 * 0.4, 2 - 0.5j), mie.coeffs_coated_pec(K0 * 0.3, K0 * 0.4, 2 - 0.5j)):
        qe, qs, qa = mie.efficiencies_from(K0 * 0.4, coeffs)
        assert qa > 0.1 * qe


def _sphere_rcs_check(s, sm):
    mask = 10 * np.log10(sm) >= 10 * np.log10(sm.max()) - 20
    return np.abs(10 * np.log10(s / sm))[mask].max(), oracle.rcs_error(s, sm)


def test_two_region_invisible_sphere():
    """With eps_r = 1 the body is free space: the PMCHWT solution radiates nothing."""
    v, t = icosphere(4, 0.4)
    Z = oracle.two_region(v, t, K0, 1.0)
    b = oracle.two_region_rhs(v, t, K0, [0, 0, 1.0], [1.0, 0, 0])[0]
    x = np.linalg.solve(Z, b)
    th = np.deg2rad(np.arange(0, 181, 5))
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    s = oracle.rcs(v, t, K0, 0, x, dirs)
    assert s.max() < 1e-4 * mie.rcs_pec(K0, 0.4, th).max()


@pytest.mark.slow
def test_two_region_dielectric_sphere_rcs_vs_mie():
    """PMCHWT with the interior operators at k1 = k0 sqrt(eps_r): homogeneous spheres of radius
    0.4 lambda, lossy (2 - 0.5j) and lossless (4), against the Mie series; the error of
    Eq. 5-25 falls with the mesh size."""
    th = np.deg2rad(np.arange(0, 181))
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    errs = {}
    for nu, eps in ((5, 2 - 0.5j), (7, 2 - 0.5j), (6, 4.0)):
        v, t = icosphere(nu, 0.4)
        x = np.linalg.solve(oracle.two_region(v, t, K0, eps),
                            oracle.two_region_rhs(v, t, K0, [0, 0, 1.0], [1.0, 0, 0])[0])
        db, err = _sphere_rcs_check(oracle.rcs(v, t, K0, 0, x, dirs), mie.rcs_dielectric(K0, 0.4, eps, th))
        assert db < 0.5 and err < 0.05, (nu, eps, db, err)
        errs[(nu, eps)] = err
    assert errs[(7, 2 - 0.5j)] < 0.8 * errs[(5, 2 - 0.5j)]


@pytest.mark.slow
def test_coated_pec_sphere_rcs_vs_mie():
    """The object of Sec. III.A: PEC sphere of radius 0.3 lambda under a 0.1 lambda coat, in a
    surface-only form (PMCHWT on the coat's outer surface, zero tangential E on the core),
    against the coated-sphere Mie series; lossy coat (2 - 0.5j) at two mesh sizes and the
    paper's eps_r = 8."""
    th = np.deg2rad(np.arange(0, 181))
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    errs = {}
    for (nu1, nu2), eps in (((6, 5), 2 - 0.5j), ((7, 6), 2 - 0.5j), ((7, 6), 8.0)):
        v1, t1 = icosphere(nu1, 0.4)
        v2, t2 = icosphere(nu2, 0.3)
        Z, rhs, n1, n2 = oracle.coated_pec(v1, t1, v2, t2, K0, eps)
        x = np.linalg.solve(Z, rhs([0, 0, 1.0], [1.0, 0, 0])[0])
        s = oracle.rcs(v1, t1, K0, 0, x[:2 * n1], dirs)
        db, err = _sphere_rcs_check(s, mie.rcs_coated_pec(K0, 0.3, 0.4, eps, th))
        assert db < 0.5 and err < 0.05, (nu1, eps, db, err)
        errs[(nu1, eps)] = err
    assert errs[(7, 2 - 0.5j)] < 0.85 * errs[(6, 2 - 0.5j)]


def test_addition_theorem_at_lossy_wavenumber():
    """The plane-wave expansion behind the translations, at the coating's complex wavenumber
    k1 = k0 sqrt(2 - 0.5j): the same formulas ((-j)^l h_l^(2), exp(-jk khat.d)) continue
    analytically, and the excess-bandwidth rule with Re k keeps the 3-digit worst-pair error of
    0.25-wavelength boxes (free-space wavelengths) at the level of the real-k case (measured
    1.8e-3 against 3.1e-3).  The wrong phase sign fails, as at real k."""
    e3 = _expansion_error(3, k=K_LOSSY)
    assert e3 < 5e-3, e3
    assert _expansion_error(3, k=K_LOSSY, sign=+1.0) > 0.1
    # the coat's own wavelength is shorter: boxes of a quarter of it behave like free-space ones
    a1 = 0.25 * K0 / abs(K_LOSSY)
    assert _expansion_error(4, a=a1, k=K_LOSSY) < 2e-3


def _rwg_patterns(v, t, k, khat, center, sign):
    """Per RWG n of mesh (v, t): int f_n exp(sign j k khat.(r - center)) dS and the same for
    n x f_n, on every direction (numpy, subdivided Gauss rule per triangle; independent of
    the C oracle except for the RWG numbering)."""
    r = oracle.rwg(v, t)
    e, tp, tm, lp, lm = r["edges"], r["tplus"], r["tminus"], r["lplus"], r["lminus"]
    N = len(e)
    P = np.zeros((N, len(khat), 3), complex)
    PX = np.zeros_like(P)
    for n in range(N):
        length = np.linalg.norm(v[e[n, 1]] - v[e[n, 0]])
        for tri, loc, s in ((tp[n], lp[n], 1.0), (tm[n], lm[n], -1.0)):
            T = v[t[tri]]
            area = np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0])) / 2
            nrm = np.cross(T[1] - T[0], T[2] - T[0]) / (2 * area)
            x, w = _brute_rule(T, s=1, n=6)
            f = s * (length / (2 * area)) * (x - T[loc])            # RWG on this triangle
            ph = np.exp(sign * 1j * k * ((x - center) @ khat.T))    # [q, dir]
            P[n] += np.einsum("q,qd,qc->dc", w, ph, f)
            PX[n] += np.einsum("q,qd,qc->dc", w, ph, np.cross(nrm, f))
    return P, PX


@pytest.mark.parametrize("k", [K0, K_LOSSY], ids=["real_k", "lossy_k"])
def test_far_field_factorisation_of_the_four_operators(k):
    """The far-field forms on which the multilevel product rests, checked on two small spheres
    three box sizes apart against the oracle's dense cross blocks:
        <L>   = -jk c R.F_t,     <n x L>    =  jk c RX.F_t,
        <Kbar> = -jk c R.(khat x F),  <n x Kbar> = jk c RX.(khat x F),
    with c = (-jk/16 pi^2) sum_khat w T_L, F = int f exp(+jk khat.(r' - c_s)),
    R = int f exp(-jk khat.(r - c_b)), RX the same for n x f.  At a complex k, R is not
    conj(F) and must be integrated as such."""
    from scipy import special
    a = 0.2
    cb, cs = np.array([0.0, 0.0, 0.0]), np.array([3 * a, 0.0, 0.0])
    vb, tb = icosphere(2, 0.04, center=cb)
    vs, ts = icosphere(2, 0.04, center=cs)
    v = np.concatenate([vb, vs])
    t = np.concatenate([tb, ts + len(vb)])
    L, NL, K, NK = oracle.operators(v, t, k, 1)
    nb = len(oracle.rwg(vb, tb)["edges"])
    blocks = [A[:nb, nb:] for A in (L, NL, K, NK)]
    # directions and the translation operator for the box offset X = c_b - c_s
    kr = float(np.real(k)) * np.sqrt(3) * a
    Lmax = int(math.ceil(kr + 1.8 * 6 ** (2 / 3) * kr ** (1 / 3)))
    x, wx = np.polynomial.legendre.leggauss(Lmax + 1)
    nphi = 2 * (Lmax + 1)
    TH, PH = np.meshgrid(np.arccos(x), 2 * np.pi * np.arange(nphi) / nphi, indexing="ij")
    W = (wx[:, None] * np.ones(nphi)[None, :] * 2 * np.pi / nphi).ravel()
    kh = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    X = cb - cs
    Xn = np.linalg.norm(X)
    cosg = kh @ (X / Xn)
    T = sum((-1j) ** l * (2 * l + 1) * (special.spherical_jn(l, k * Xn) - 1j * special.spherical_yn(l, k * Xn))
            * special.eval_legendre(l, cosg) for l in range(Lmax + 1))
    c = (-1j * k / (16 * np.pi ** 2)) * W * T                        # per direction
    R, RX = _rwg_patterns(vb, tb, k, kh, cb, -1.0)
    F, _ = _rwg_patterns(vs, ts, k, kh, cs, +1.0)
    Ft = F - kh[None] * np.einsum("ndc,dc->nd", F, kh)[..., None]
    kxF = np.cross(kh[None], F)
    far = [-1j * k * np.einsum("d,mdc,ndc->mn", c, R, Ft),
           1j * k * np.einsum("d,mdc,ndc->mn", c, RX, Ft),
           -1j * k * np.einsum("d,mdc,ndc->mn", c, R, kxF),
           1j * k * np.einsum("d,mdc,ndc->mn", c, RX, kxF)]
    for q, (dense, ff) in enumerate(zip(blocks, far)):
        err = np.abs(dense - ff).max() / np.abs(dense).max()
        assert err < 1e-6, (q, err)
    # R = conj(F) (and so the antipodal packing of the stored patterns) holds at real k only
    Fb, _ = _rwg_patterns(vb, tb, k, kh, cb, +1.0)
    via_conj = -1j * k * np.einsum("d,mdc,ndc->mn", c, np.conj(Fb), Ft)
    err_conj = np.abs(blocks[0] - via_conj).max() / np.abs(blocks[0]).max()
    if np.imag(k) == 0:
        assert err_conj < 1e-6
    else:
        assert err_conj > 1e-2


# ------------------------------------------------- plane-wave right-hand sides (Eqs. 49-50)
def _rwg_independent(v, t):
    """RWG functions built here from the mesh alone: edges sorted by (min, max) vertex; T+ is
    the triangle that runs along the edge from its smaller to its larger vertex (as listed)."""
    owners = {}
    for ti, tri in enumerate(t):
        for i in range(3):
            a, b = int(tri[i]), int(tri[(i + 1) % 3])
            owners.setdefault((min(a, b), max(a, b)), []).append((ti, a < b, int(tri[(i + 2) % 3])))
    out = []
    for e in sorted(owners):
        (t0, fwd0, p0), (t1, fwd1, p1) = owners[e]
        plus, minus = ((t0, p0), (t1, p1)) if fwd0 else ((t1, p1), (t0, p0))
        out.append((e, plus, minus))
    return out


def _rhs_by_quadrature(v, t, k, khat, phat, rule):
    """b^J = <f, E/2 + n x H/2>, b^M = <f, H/2 - n x E/2> (Eqs. 49-50) for E = p exp(-jk khat.r),
    H = (khat x p) exp(-jk khat.r), integrated with rule(triangle vertices) -> (points, weights)."""
    khat, phat = np.asarray(khat, float), np.asarray(phat, float)
    hp = np.cross(khat, phat)
    funcs = _rwg_independent(v, t)
    N = len(funcs)
    b = np.zeros(2 * N, complex)
    for m, (e, plus, minus) in enumerate(funcs):
        l = np.linalg.norm(v[e[1]] - v[e[0]])
        for sgn, (ti, pv) in ((1.0, plus), (-1.0, minus)):
            P = v[t[ti]]
            nn = np.cross(P[1] - P[0], P[2] - P[0])
            A = np.linalg.norm(nn) / 2
            nn /= 2 * A
            x, w = rule(P)
            f = sgn * (l / (2 * A)) * (x - v[pv])
            ph = np.exp(-1j * k * (x @ khat))
            tj = phat + np.cross(nn, hp)          # E + n x H (both times the phase)
            tm = hp - np.cross(nn, phat)          # H - n x E
            b[m] += 0.5 * np.sum(w * ph * (f @ tj))
            b[N + m] += 0.5 * np.sum(w * ph * (f @ tm))
    return b


def _centroid_rule(P):
    """At k = 0 the integrand is linear in r: the centroid rule is exact."""
    A = np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0])) / 2
    return P.mean(0)[None, :], np.array([A])


KH_RHS = np.array([0.36, -0.48, 0.8])
PH_RHS = np.cross(KH_RHS, [0.0, 0.0, 1.0]) / np.linalg.norm(np.cross(KH_RHS, [0.0, 0.0, 1.0]))


def test_rwg_numbering_of_the_pins_matches_the_oracle():
    v, t = icosphere(1, 0.3)
    E = oracle.rwg(v, t)
    mine = _rwg_independent(v, t)
    assert [tuple(e) for e in E["edges"]] == [f[0] for f in mine]
    assert list(E["tplus"]) == [f[1][0] for f in mine]
    assert list(E["tminus"]) == [f[2][0] for f in mine]


def test_planewave_rhs_closed_form_at_zero_frequency():
    """At k = 0, int_T f = +-(l/2)(centroid - p): b^J and b^M of Eqs. 49-50 are sums of dot
    products with the constant fields.  A flipped n x E (or n x H) term fails by O(1)."""
    v, t = icosphere(1, 0.3)
    b = oracle.rhs_planewave(v, t, 0.0, 0, KH_RHS, PH_RHS)[0]
    ref = _rhs_by_quadrature(v, t, 0.0, KH_RHS, PH_RHS, _centroid_rule)
    N = len(ref) // 2
    assert np.abs(b - ref).max() < 1e-14 * np.abs(ref).max()
    # the pin separates the signs of Eq. 50: H/2 + n x E/2 is far from the oracle's row
    hp = np.cross(KH_RHS, PH_RHS)
    funcs = _rwg_independent(v, t)
    flip = np.zeros(N, complex)
    for m, (e, plus, minus) in enumerate(funcs):
        l = np.linalg.norm(v[e[1]] - v[e[0]])
        for sgn, (ti, pv) in ((1.0, plus), (-1.0, minus)):
            P = v[t[ti]]
            nn = np.cross(P[1] - P[0], P[2] - P[0])
            nn /= np.linalg.norm(nn)
            flip[m] += 0.5 * sgn * (l / 2) * np.dot(P.mean(0) - v[pv], hp + np.cross(nn, PH_RHS))
    assert np.linalg.norm(flip - b[N:]) > 0.3 * np.linalg.norm(b[N:])


@pytest.mark.parametrize("mode", [0, 1])
def test_planewave_rhs_vs_brute_force(mode):
    """At k = 2 pi on a 0.3-wavelength sphere, against a subdivided Gauss product rule.  Mode 1
    (the PEC combined-field row) is the J half of mode 0."""
    v, t = icosphere(2, 0.3)
    b = oracle.rhs_planewave(v, t, K0, mode, KH_RHS, PH_RHS)[0]
    ref = _rhs_by_quadrature(v, t, K0, KH_RHS, PH_RHS, lambda P: _brute_rule(P, s=1, n=8))
    N = len(ref) // 2
    if mode == 1:
        ref = ref[:N]
    assert np.linalg.norm(b - ref) / np.linalg.norm(ref) < 1e-6
