"""Pins of the coupling-block oracle (Eqs. 40a/b, 47, 48) against facts that do not come
from it: the defining properties of the RWG and edge functions, the Gram matrices of the
C oracle (pinned on their own in test_oracle_pins), closed-form integrals of constant fields
and the antisymmetry of the rotation n x."""
import numpy as np
import pytest

import oracle
from oracle import coupling
from paper_2210_04892_gb300.inputs import ellipsoid, icosphere


def _random_triangle(rng):
    P = rng.standard_normal((3, 3))
    if np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0])) < 0.3:
        P[2] += 1.0
    return P


def _tetrahedron():
    v = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.2, 0.9, 0], [0.3, 0.25, 0.8]])
    t = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]], np.int32)
    return v, t


@pytest.mark.parametrize("seed", range(4))
def test_edge_function_tangential_moments(seed):
    """eta_k has tangential component 1 along its own edge (from the smaller to the larger
    global vertex number) and 0 along the other two edges, at every point of the edges."""
    rng = np.random.default_rng(seed)
    P = _random_triangle(rng)
    gid = rng.permutation(10)[:3]
    s = np.linspace(0, 1, 7)
    for k in range(3):
        for j in range(3):
            a, b = (j + 1) % 3, (j + 2) % 3
            if gid[a] > gid[b]:
                a, b = b, a
            lam = np.zeros((len(s), 3))
            lam[:, a], lam[:, b] = 1 - s, s
            tang = (P[b] - P[a]) / np.linalg.norm(P[b] - P[a])
            val = coupling.whitney(P, gid, k, lam) @ tang
            np.testing.assert_allclose(val, 1.0 if j == k else 0.0, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_edge_functions_reproduce_constant_tangential_fields(seed):
    """Any constant field c tangential to the triangle equals sum_k (c . t_k) eta_k."""
    rng = np.random.default_rng(10 + seed)
    P = _random_triangle(rng)
    gid = rng.permutation(10)[:3]
    _, n, _ = coupling.face_frame(P)
    c = rng.standard_normal(3)
    c -= (c @ n) * n
    lam = rng.dirichlet(np.ones(3), size=5)
    acc = np.zeros((5, 3))
    for k in range(3):
        a, b = (k + 1) % 3, (k + 2) % 3
        if gid[a] > gid[b]:
            a, b = b, a
        tang = (P[b] - P[a]) / np.linalg.norm(P[b] - P[a])
        acc += (c @ tang) * coupling.whitney(P, gid, k, lam)
    np.testing.assert_allclose(acc, np.repeat(c[None], 5, 0), atol=1e-12)


def test_rwg_normal_flux_and_tangency():
    """The RWG function's normal component across its own edge is 1 and it is tangent to
    the two edges that meet at its free vertex."""
    rng = np.random.default_rng(3)
    P = _random_triangle(rng)
    _, n, _ = coupling.face_frame(P)
    s = np.linspace(0, 1, 5)
    for free in range(3):
        a, b = (free + 1) % 3, (free + 2) % 3
        lam = np.zeros((len(s), 3))
        lam[:, a], lam[:, b] = 1 - s, s
        edge = P[b] - P[a]
        out = np.cross(edge, n)
        out /= np.linalg.norm(out)
        if out @ (P[a] - P[free]) < 0:
            out = -out
        f = coupling.rwg_on_face(P, free, np.linalg.norm(edge), 1.0, lam)
        np.testing.assert_allclose(f @ out, 1.0, atol=1e-12)
        for o in (a, b):
            lam2 = np.zeros((len(s), 3))
            lam2[:, free], lam2[:, o] = 1 - s, s
            f2 = coupling.rwg_on_face(P, free, np.linalg.norm(edge), 1.0, lam2)
            e2 = (P[o] - P[free]) / np.linalg.norm(P[o] - P[free])
            np.testing.assert_allclose(np.linalg.norm(np.cross(f2, e2), axis=1), 0.0, atol=1e-12)


@pytest.mark.parametrize("mesh", ["tetra", "sphere", "ellipsoid"])
def test_conforming_blocks_equal_the_gram_matrices(mesh):
    """On flat triangles n x f_e is the conforming edge function of edge e (both have unit
    tangential moment on e and none on the other edges), so with the conforming layout
    D^{J Lambda} = G / 2, D^{M Lambda} = X / 2, D^{Lambda J} = -G, D^{Lambda M} = -X^T, with
    G = <f_m, f_n> and X = <f_m, n x f_n> from the C oracle."""
    v, t = {"tetra": _tetrahedron, "sphere": lambda: icosphere(3, 0.5),
            "ellipsoid": lambda: ellipsoid(3, (1.0, 0.7, 0.4))}[mesh]()
    G, X = oracle.gram(v, t)
    DJL, DML, DLJ, DLM = coupling.coupling_blocks(v, t, conforming=True)
    sc = np.abs(G).max()
    np.testing.assert_allclose(DJL, 0.5 * G, atol=1e-12 * sc)
    np.testing.assert_allclose(DML, 0.5 * X, atol=1e-12 * sc)
    np.testing.assert_allclose(DLJ, -G, atol=1e-12 * sc)
    np.testing.assert_allclose(DLM, -X.T, atol=1e-12 * sc)


def test_face_blocks_against_constant_field_integrals():
    """Per face: sum_k (c . t_k) <f_m, eta_k>_T = <f_m, c>_T = sign (l/2) (centroid - p) . c for
    constant tangential c, and <f_m, eta_k>_T = 0 for the edge k of f_m itself (there
    eta_k = n x f_m is perpendicular to f_m)."""
    v, t = icosphere(2, 0.5)
    R = oracle.rwg(v, t)
    _, DML, _, _ = coupling.coupling_blocks(v, t, conforming=False)
    rng = np.random.default_rng(5)
    for m in range(len(R["edges"])):
        a, b = R["edges"][m]
        ln = np.linalg.norm(v[b] - v[a])
        for f, free, sign in ((R["tplus"][m], R["lplus"][m], 1.0), (R["tminus"][m], R["lminus"][m], -1.0)):
            P = v[t[f]]
            _, n, _ = coupling.face_frame(P)
            c = rng.standard_normal(3)
            c -= (c @ n) * n
            acc = 0.0
            for k in range(3):
                ia, ib = sorted((t[f][(k + 1) % 3], t[f][(k + 2) % 3]))
                tang = (v[ib] - v[ia]) / np.linalg.norm(v[ib] - v[ia])
                acc += (c @ tang) * 2 * DML[m, 3 * f + k]
            exact = sign * 0.5 * ln * (P.mean(0) - P[free]) @ c
            assert abs(acc - exact) < 1e-12 * ln
            assert abs(DML[m, 3 * f + free]) < 1e-14


def test_transpose_relations_and_face_sums():
    """a . (n x b) = -b . (n x a) gives D^{Lambda J} = -2 (D^{J Lambda})^T and
    D^{Lambda M} = -2 (D^{M Lambda})^T; summing the two face columns of each edge turns the
    face layout into the conforming one."""
    v, t = ellipsoid(2, (1.0, 0.8, 0.6))
    F = coupling.coupling_blocks(v, t, conforming=False)
    C = coupling.coupling_blocks(v, t, conforming=True)
    for DJL, DML, DLJ, DLM in (F, C):
        np.testing.assert_allclose(DLJ, -2 * DJL.T, atol=1e-14)
        np.testing.assert_allclose(DLM, -2 * DML.T, atol=1e-14)
    R = oracle.rwg(v, t)
    S = np.zeros((3 * len(t), len(R["edges"])))
    ids = {(int(a), int(b)): n for n, (a, b) in enumerate(R["edges"])}
    for f in range(len(t)):
        for k in range(3):
            S[3 * f + k, ids[tuple(sorted((int(t[f][(k + 1) % 3]), int(t[f][(k + 2) % 3]))))]] = 1.0
    np.testing.assert_allclose(F[0] @ S, C[0], atol=1e-14)
    np.testing.assert_allclose(F[1] @ S, C[1], atol=1e-14)
    np.testing.assert_allclose(S.T @ F[2], C[2], atol=1e-14)
