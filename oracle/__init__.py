"""CPU FP64 oracle for the boundary-integral operator of Eqs. 42-46.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg, never by the product package.  It shares no code
with the CUDA path; both consume only the seeded inputs of
paper_2210_04892_gb300.inputs.

Functions (each cites the passage it follows):
  rwg(verts, tris)            RWG functions on triangle pairs (Sec. II.C, Eq. exp4-5)
  fill(verts, tris, k, mode)  dense matrix, mode 0 = C block (Eqs. 43-46), mode 1 = PEC
                              combined field G/4 - P (Eqs. 24a/24b, alpha = 1/2)
  rows(..., rows)             selected rows of the same matrix
  operators(...)              <f,Lf>, <f,n x Lf>, <f,Kbar f>, <f,n x Kbar f>
  gram(...)                   <f_m,f_n>, <f_m, n x f_n>
  rhs_planewave(...)          Eqs. 49-50 with the plane wave of Sec. III (mode 2: <f,E>, <f,H>)
  farfield(...)               far field of J, M (Eq. 22a), RCS sigma = 4 pi |F|^2
  rcs_error(...)              Eq. 5-25
  two_region(...)             surface-only formulation of a homogeneous (lossy) body: exterior
                              operators at k0, interior at k1 = k0 sqrt(eps_r mu_r)
  coated_pec(...)             the same for a PEC core under a coat (the object of Sec. III.A)
Mie series for PEC, dielectric and coated PEC spheres: oracle.mie.
Coupling blocks D^{X Lambda}, D^{Lambda X} of the hybrid system (Eqs. 40a/b, 47, 48):
oracle.coupling.

Complex wavenumbers (lossy media, Im k < 0 with exp(j w t)) are accepted by fill, rows,
operators and pair_blocks.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.POINTER(ctypes.c_int)
        _lib.or_rwg.argtypes = [ctypes.c_int, d, ctypes.c_int, i, i, i, i, i, i]
        _lib.or_fill_rows.argtypes = [ctypes.c_int, d, ctypes.c_int, i, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, i, d]
        _lib.or_operators.argtypes = [ctypes.c_int, d, ctypes.c_int, i, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, d, d, d, d]
        _lib.or_gram.argtypes = [ctypes.c_int, d, ctypes.c_int, i, d, d]
        _lib.or_rhs_planewave.argtypes = [ctypes.c_int, d, ctypes.c_int, i, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, d, d, d]
        _lib.or_farfield.argtypes = [ctypes.c_int, d, ctypes.c_int, i, ctypes.c_double, ctypes.c_int, d,
                                     ctypes.c_int, d, d]
        _lib.or_static_tri.argtypes = [d, d, d, d, d]
        _lib.or_pair_blocks.argtypes = [d, d, i, i, ctypes.c_double, ctypes.c_double, ctypes.c_int, d]
        _lib.or_rule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, d, d]
        _lib.or_num_threads.restype = ctypes.c_int
    return _lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _mesh(verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    return v, t


class MeshError(ValueError):
    pass


def rwg(verts, tris):
    """Returns dict(edges[N,2], tplus, tminus, lplus, lminus)."""
    v, t = _mesh(verts, tris)
    nt = len(t)
    cap = 3 * nt // 2 + 1
    e = np.zeros((cap, 2), np.int32)
    tp, tm, lp, lm = (np.zeros(cap, np.int32) for _ in range(4))
    n = lib().or_rwg(len(v), _p(v), nt, _p(t, ctypes.c_int), _p(e, ctypes.c_int), _p(tp, ctypes.c_int),
                     _p(tm, ctypes.c_int), _p(lp, ctypes.c_int), _p(lm, ctypes.c_int))
    if n < 0:
        raise MeshError({-1: "open or non-manifold edge", -2: "inconsistent orientation",
                         -3: "degenerate triangle"}[n])
    return dict(edges=e[:n], tplus=tp[:n], tminus=tm[:n], lplus=lp[:n], lminus=lm[:n])


def num_unknowns(verts, tris, mode):
    n = len(rwg(verts, tris)["edges"])
    return 2 * n if mode == 0 else n


def rows(verts, tris, k, mode, rows_idx, level=0):
    v, t = _mesh(verts, tris)
    nun = num_unknowns(v, t, mode)
    r = np.ascontiguousarray(rows_idx, dtype=np.int32)
    Z = np.zeros((len(r), nun), np.complex128)
    kc = complex(k)
    rc = lib().or_fill_rows(len(v), _p(v), len(t), _p(t, ctypes.c_int), kc.real, kc.imag, int(mode), int(level),
                            len(r), _p(r, ctypes.c_int), _p(Z.view(np.float64)))
    if rc:
        raise MeshError(rc)
    return Z


def fill(verts, tris, k, mode, level=0):
    v, t = _mesh(verts, tris)
    nun = num_unknowns(v, t, mode)
    Z = np.zeros((nun, nun), np.complex128)
    kc = complex(k)
    rc = lib().or_fill_rows(len(v), _p(v), len(t), _p(t, ctypes.c_int), kc.real, kc.imag, int(mode), int(level),
                            0, None, _p(Z.view(np.float64)))
    if rc:
        raise MeshError(rc)
    return Z


def operators(verts, tris, k, level=0):
    v, t = _mesh(verts, tris)
    n = num_unknowns(v, t, 1)
    out = [np.zeros((n, n), np.complex128) for _ in range(4)]
    kc = complex(k)
    rc = lib().or_operators(len(v), _p(v), len(t), _p(t, ctypes.c_int), kc.real, kc.imag, int(level),
                            *[_p(o.view(np.float64)) for o in out])
    if rc:
        raise MeshError(rc)
    return out


def gram(verts, tris):
    v, t = _mesh(verts, tris)
    n = num_unknowns(v, t, 1)
    G = np.zeros((n, n))
    X = np.zeros((n, n))
    lib().or_gram(len(v), _p(v), len(t), _p(t, ctypes.c_int), _p(G), _p(X))
    return G, X


def rhs_planewave(verts, tris, k, mode, khat, phat):
    v, t = _mesh(verts, tris)
    kh = np.ascontiguousarray(np.atleast_2d(khat), np.float64)
    ph = np.ascontiguousarray(np.atleast_2d(phat), np.float64)
    nun = num_unknowns(v, t, 1) * (1 if mode == 1 else 2)
    b = np.zeros((len(kh), nun), np.complex128)
    lib().or_rhs_planewave(len(v), _p(v), len(t), _p(t, ctypes.c_int), float(k), int(mode), len(kh),
                           _p(kh), _p(ph), _p(b.view(np.float64)))
    return b


def farfield(verts, tris, k, mode, x, dirs):
    v, t = _mesh(verts, tris)
    xx = np.ascontiguousarray(x, np.complex128)
    dd = np.ascontiguousarray(np.atleast_2d(dirs), np.float64)
    F = np.zeros((len(dd), 3), np.complex128)
    lib().or_farfield(len(v), _p(v), len(t), _p(t, ctypes.c_int), float(k), int(mode), _p(xx.view(np.float64)),
                      len(dd), _p(dd), _p(F.view(np.float64)))
    return F


def rcs(verts, tris, k, mode, x, dirs):
    F = farfield(verts, tris, k, mode, x, dirs)
    return 4 * np.pi * np.sum(np.abs(F) ** 2, axis=1)


def rcs_error(sigma, sigma_ref):
    """Eq. 5-25: L2 norm of the relative RCS error over the sampled angles."""
    sigma = np.asarray(sigma)
    sigma_ref = np.asarray(sigma_ref)
    return float(np.sqrt(np.sum(np.abs(sigma - sigma_ref) ** 2) / np.sum(np.abs(sigma_ref) ** 2)))


def static_tri(P, r):
    P = np.ascontiguousarray(P, np.float64).reshape(9)
    r = np.ascontiguousarray(r, np.float64)
    I1 = np.zeros(1)
    Ir = np.zeros(3)
    Ig = np.zeros(3)
    lib().or_static_tri(_p(P), _p(r), _p(I1), _p(Ir), _p(Ig))
    return I1[0], Ir, Ig


def pair_blocks(Pm, Pn, idm, idn, k, level=0):
    Pm = np.ascontiguousarray(Pm, np.float64).reshape(9)
    Pn = np.ascontiguousarray(Pn, np.float64).reshape(9)
    a = np.ascontiguousarray(idm, np.int32)
    b = np.ascontiguousarray(idn, np.int32)
    out = np.zeros((4, 3, 3), np.complex128)
    kc = complex(k)
    lib().or_pair_blocks(_p(Pm), _p(Pn), _p(a, ctypes.c_int), _p(b, ctypes.c_int), kc.real, kc.imag, int(level),
                         _p(out.view(np.float64)))
    return out


def rule(kind, n, q=3):
    b = np.zeros((4096, 3))
    w = np.zeros(4096)
    m = lib().or_rule(kind, n, q, _p(b), _p(w))
    return b[:m], w[:m]


def threads():
    return lib().or_num_threads()


# ------------------------------------------------------------ two-region surface formulations
#
# Fields of surface currents (J, M) radiating in a medium of wavenumber k_i and relative wave
# impedance eta_i (normalised fields: E scaled by sqrt(eps0/mu0), so eta_0 = 1; M = E x n as in
# Sec. II.C):
#     E = eta_i L_i J - K_i M,      H = K_i J + L_i M / eta_i,
# with L and K the operators of Sec. II.C at k_i.  A region's field is radiated by the currents
# n x H, E x n of its boundary with n pointing into it (equivalence principle); the outside
# currents of a surface therefore appear with a minus sign in the region it encloses.  Matching
# the tangential E and H on the interface (the traces tested with f_m) and letting the
# principal-value jumps of the two sides cancel gives the PMCHWT system
#     [ L0 + eta L1     -(K0 + K1)       ] [J]   [ -<f, E_inc> ]
#     [ K0 + K1          L0 + L1 / eta   ] [M] = [ -<f, H_inc> ]
# (Poggio-Miller-Chang-Harrington-Wu-Tsai).  The interior of the paper's method is its HDG
# volume discretisation coupled through Eq. 52; this surface-only form stands in for it on
# homogeneous and layered spheres, where the Mie series gives the answer.

def _k_eta(k0, eps_r, mu_r):
    k1 = complex(k0) * np.sqrt(complex(eps_r) * complex(mu_r))
    if k1.real < 0:
        k1 = -k1
    eta = np.sqrt(complex(mu_r) / complex(eps_r))
    if eta.real < 0:
        eta = -eta
    return k1, eta


def two_region(verts, tris, k0, eps_r, mu_r=1.0, level=0):
    """PMCHWT matrix (2N x 2N, unknowns J then M) of a homogeneous body of relative
    permittivity eps_r (exp(j w t): loss is Im eps_r < 0) in free space."""
    k1, eta = _k_eta(k0, eps_r, mu_r)
    L0, _, K0_, _ = operators(verts, tris, k0, level)
    L1, _, K1_, _ = operators(verts, tris, k1, level)
    K = K0_ + K1_
    return np.block([[L0 + eta * L1, -K], [K, L0 + L1 / eta]])


def two_region_rhs(verts, tris, k0, khat, phat):
    """Right-hand side [-<f, E_inc>; -<f, H_inc>] of two_region for plane waves."""
    return -rhs_planewave(verts, tris, k0, 2, khat, phat)


def _union(v1, t1, v2, t2):
    v1 = np.asarray(v1, float)
    v = np.concatenate([v1, np.asarray(v2, float)])
    t = np.concatenate([np.asarray(t1, np.int32), np.asarray(t2, np.int32) + len(v1)])
    return v, t


def coated_pec(v_out, t_out, v_core, t_core, k0, eps_r, mu_r=1.0, level=0):
    """System of a PEC core (surface S2) under a coat of relative permittivity eps_r whose
    outer surface S1 faces free space.  Unknowns [J1, M1, J2] (J1, M1 on S1, J2 = n2 x H on
    the core, n2 pointing into the coat).  The coat's field is radiated by (-J1, -M1) on S1
    and J2 on S2 in the coat medium:
        E1 = -eta L1 J1 + K1 M1 + eta L1 J2,   H1 = -K1 J1 - L1 M1 / eta + K1 J2.
    Rows: tangential E and H matched on S1 (as in two_region, plus the core's coupling),
    tangential E1 = 0 on S2.  Returns (Z, rhs, N1, N2): rhs(khat, phat) builds the right-hand
    sides, and the RWG functions of S1 come first (J1 and M1 are the first 2 N1 unknowns)."""
    k1, eta = _k_eta(k0, eps_r, mu_r)
    v, t = _union(v_out, t_out, v_core, t_core)
    e = rwg(v, t)["edges"]
    on1 = e[:, 0] < len(v_out)
    n1 = int(on1.sum())
    if not np.all(on1[:n1]) or np.any(on1[n1:]):
        raise MeshError("RWG functions of the outer surface must come first")
    n2 = len(e) - n1
    L0, _, K0_, _ = operators(v_out, t_out, k0, level)
    L1, _, K1_, _ = operators(v, t, k1, level)
    a, b = slice(0, n1), slice(n1, n1 + n2)
    K = K0_ + K1_[a, a]
    Z = np.block([
        [L0 + eta * L1[a, a], -K, -eta * L1[a, b]],
        [K, L0 + L1[a, a] / eta, -K1_[a, b]],
        [-eta * L1[b, a], K1_[b, a], eta * L1[b, b]],
    ])

    def rhs(khat, phat):
        eh = two_region_rhs(v_out, t_out, k0, khat, phat)
        return np.concatenate([eh, np.zeros((eh.shape[0], n2), complex)], axis=1)

    return Z, rhs, n1, n2
