"""Seeded synthetic workloads: closed triangle meshes and complex test vectors.

This module only builds inputs.  It contains none of the method's arithmetic
(no basis functions, no Green's function, no quadrature), so both the CUDA
path and the CPU oracle may consume what it produces.

Meshes follow the conventions of the boundary-integral formulation (Sec. II.B):
vertices ``verts[nv][3]`` (float64, lengths in wavelengths), triangles
``tris[nt][3]`` (int32), counter-clockwise when seen from outside, so the
right-hand normal points out of the enclosed volume.  A mesh may hold several
disjoint closed components (Sec. II.F, comment 2).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20221011

_PHI = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_V = np.array(
    [[-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
     [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
     [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1]], dtype=np.float64)
_ICO_F = np.array(
    [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
     [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
     [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
     [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)


def _orient_outward(verts: np.ndarray, tris: np.ndarray, center=None) -> np.ndarray:
    """Flip triangles whose right-hand normal points toward ``center``
    (valid for star-shaped components about that center)."""
    c = verts.mean(axis=0) if center is None else np.asarray(center, dtype=np.float64)
    p0, p1, p2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    cen = (p0 + p1 + p2) / 3.0
    flip = np.einsum("ij,ij->i", nrm, cen - c) < 0
    out = tris.copy()
    out[flip] = out[flip][:, [0, 2, 1]]
    return out


def icosphere(nu: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere of frequency ``nu``: 20*nu^2 triangles, 30*nu^2 edges,
    10*nu^2+2 vertices, every vertex projected onto the sphere."""
    if nu < 1:
        raise ValueError("nu must be >= 1")
    M = 12 * (nu + 1) + 1
    keys_all, pts_all, tri_keys = [], [], []
    ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nu + 1), indexing="ij")
    sel = ii + jj <= nu
    ii, jj = ii[sel], jj[sel]
    kk = nu - ii - jj
    # local index of grid point (i, j) inside one face
    lid = -np.ones((nu + 1, nu + 1), dtype=np.int64)
    lid[ii, jj] = np.arange(ii.size)
    # the two triangle families of the subdivided face, counter-clockwise like (A, B, C)
    ci, cj = np.meshgrid(np.arange(nu), np.arange(nu), indexing="ij")
    up = ci + cj <= nu - 1
    t_up = np.stack([lid[ci[up], cj[up]], lid[ci[up] + 1, cj[up]], lid[ci[up], cj[up] + 1]], 1)
    dn = ci + cj <= nu - 2
    t_dn = np.stack([lid[ci[dn] + 1, cj[dn]], lid[ci[dn] + 1, cj[dn] + 1], lid[ci[dn], cj[dn] + 1]], 1)
    local_tris = np.concatenate([t_up, t_dn], 0)
    for f, (a, b, c) in enumerate(_ICO_F):
        # weights of vertices a, b, c (sum nu); exact integer key, independent of the face
        w = np.stack([kk, ii, jj], 1)
        vid = np.array([a, b, c], dtype=np.int64)
        order = np.argsort(vid)
        vs, ws = vid[order], w[:, order]
        code = np.where(ws > 0, vs[None, :] * (nu + 1) + ws, 0)
        # push zero slots to the end so the key does not depend on which face built the point
        code = -np.sort(-code, axis=1)
        key = (code[:, 0] * M + code[:, 1]) * M + code[:, 2]
        pts = (kk[:, None] * _ICO_V[a] + ii[:, None] * _ICO_V[b] + jj[:, None] * _ICO_V[c]) / nu
        keys_all.append(key)
        pts_all.append(pts)
        tri_keys.append(key[local_tris])
    keys = np.concatenate(keys_all)
    pts = np.concatenate(pts_all)
    uk, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    verts = pts[first]
    verts = verts / np.linalg.norm(verts, axis=1, keepdims=True) * radius + np.asarray(center)
    tk = np.concatenate(tri_keys)
    tris = np.searchsorted(uk, tk).astype(np.int32)
    return verts.astype(np.float64), tris.astype(np.int32)


def _box_surface(lo, hi, spacing_fn):
    """Closed surface of an axis-aligned box, triangulated on graded tensor grids.
    ``spacing_fn(length)`` returns the node coordinates in [0, length]."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    axes = [lo[d] + spacing_fn(hi[d] - lo[d]) for d in range(3)]
    verts = {}
    vlist = []

    def vid(p):
        key = tuple(np.round(p, 10))
        if key not in verts:
            verts[key] = len(vlist)
            vlist.append(p)
        return verts[key]

    tris = []
    for d in range(3):
        u, v = [(d + 1) % 3, (d + 2) % 3]
        for side, coord in ((0, lo[d]), (1, hi[d])):
            gu, gv = axes[u], axes[v]
            for a in range(len(gu) - 1):
                for b in range(len(gv) - 1):
                    q = []
                    for (x, y) in ((a, b), (a + 1, b), (a + 1, b + 1), (a, b + 1)):
                        p = np.zeros(3)
                        p[d], p[u], p[v] = coord, gu[x], gv[y]
                        q.append(vid(p))
                    tris.append([q[0], q[1], q[2]])
                    tris.append([q[0], q[2], q[3]])
    V = np.array(vlist)
    T = np.array(tris, dtype=np.int64)
    return V, _orient_outward(V, T, center=(lo + hi) / 2)


def _zip_rings(outer, inner, phi_o, phi_i, tris):
    """Triangulate the band between two closed rings (vertex ids with their angles), both
    counter-clockwise in angle, by advancing along whichever ring has the smaller next angle."""
    no, ni = len(outer), len(inner)
    i = j = 0
    while i < no or j < ni:
        ao = phi_o[i] + (2 * np.pi if i >= no else 0) if i < no else np.inf
        ai = phi_i[j] if j < ni else np.inf
        next_o = phi_o[(i + 1) % no] + (2 * np.pi if i + 1 >= no else 0)
        next_i = phi_i[(j + 1) % ni] + (2 * np.pi if j + 1 >= ni else 0)
        if (i < no) and (j >= ni or next_o <= next_i):
            tris.append([outer[i % no], outer[(i + 1) % no], inner[j % ni]])
            i += 1
        else:
            tris.append([outer[i % no], inner[(j + 1) % ni], inner[j % ni]])
            j += 1


def _cylinder_surface(center, radius, height, h):
    """Closed cylinder (axis z) with flat caps, triangle size about ``h``: a structured side
    and caps made of concentric rings whose point counts follow their circumference."""
    center = np.asarray(center, float)
    nphi = max(8, int(np.ceil(2 * np.pi * radius / h)))
    nz = max(2, int(np.ceil(height / h)))
    nr = max(1, int(round(radius / h)))
    vlist, tris = [], []

    def add(p):
        vlist.append(np.asarray(p, float))
        return len(vlist) - 1

    phis = 2 * np.pi * np.arange(nphi) / nphi
    ring = [[add(center + np.array([radius * np.cos(p), radius * np.sin(p), -height / 2 + height * k / nz]))
             for p in phis] for k in range(nz + 1)]
    for k in range(nz):
        for a in range(nphi):
            b = (a + 1) % nphi
            tris.append([ring[k][a], ring[k][b], ring[k + 1][b]])
            tris.append([ring[k][a], ring[k + 1][b], ring[k + 1][a]])
    for zk in (0, nz):
        zc = center[2] - height / 2 + height * zk / nz
        outer, phi_o = ring[zk], phis
        for r in range(nr - 1, 0, -1):
            rr = radius * r / nr
            m = max(6, int(round(2 * np.pi * rr / h)))
            off = np.pi / m * (r % 2)
            phi_i = off + 2 * np.pi * np.arange(m) / m
            inner = [add([center[0] + rr * np.cos(p), center[1] + rr * np.sin(p), zc]) for p in phi_i]
            _zip_rings(outer, inner, phi_o, phi_i, tris)
            outer, phi_o = inner, phi_i
        ctr = add([center[0], center[1], zc])
        for a in range(len(outer)):
            tris.append([outer[a], outer[(a + 1) % len(outer)], ctr])
    V = np.array(vlist)
    T = np.array(tris, dtype=np.int64)
    return V, _orient_outward(V, T, center=center)


def cube_with_cylinder(size=5.0, h_face=1 / 10.7, h_edge=1 / 16, cyl_radius=1.0, cyl_height=3.0, h_cyl=1 / 16):
    """Two disjoint closed components: a cube of side ``size`` on tensor grids graded
    smoothly from ``h_face`` (face centres) to ``h_edge`` (cube edges), and a closed coaxial
    cylinder strictly inside it (the shape of a layered cube with an embedded body, Sec. III.E).
    The defaults give about 100k RWG functions."""

    def graded(length):
        # x(s) = L (s - a sin(2 pi s) / (2 pi)): spacing (1 - a) h0 at the ends, (1 + a) h0 mid-face
        a = (h_face - h_edge) / (h_face + h_edge)
        n = max(2, int(round(length * (1 - a) / h_edge)))
        sgrid = np.arange(n + 1) / n
        return length * (sgrid - a * np.sin(2 * np.pi * sgrid) / (2 * np.pi))

    half = size / 2
    Vc, Tc = _box_surface((-half, -half, -half), (half, half, half), graded)
    Vy, Ty = _cylinder_surface((0.0, 0.0, 0.0), cyl_radius, cyl_height, h_cyl)
    V = np.concatenate([Vc, Vy], 0)
    T = np.concatenate([Tc, Ty + len(Vc)], 0)
    return V.astype(np.float64), T.astype(np.int32)


def ellipsoid(nu: int, axes=(1.0, 0.75, 0.5)):
    v, t = icosphere(nu, 1.0)
    return (v * np.asarray(axes)[None, :]).astype(np.float64), t


def cube(n_per_side: int, size: float = 1.0):
    """Closed cube surface of side ``size`` on a uniform n x n grid per face."""
    half = size / 2
    V, T = _box_surface((-half, -half, -half), (half, half, half), lambda L: np.linspace(0.0, L, n_per_side + 1))
    return V.astype(np.float64), T.astype(np.int32)


def serving_requests(count: int, min_unknowns: int, max_unknowns: int, max_rhs: int, seed: int = SEED_BASE + 3):
    """Requests of a serving stream: shape uniform over {sphere, ellipsoid 1:0.75:0.5, cube},
    unknowns log-uniform in [min, max], mode PEC (N unknowns) or C block (2N unknowns) with
    probability 1/2, nrhs uniform in 1..max_rhs, plane waves with random directions and
    polarisations, k0 chosen so that the mean edge is lambda/10.  Returns dicts with
    verts, tris, k0, op_mode, khat, phat."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        shape = ["sphere", "ellipsoid", "cube"][rng.integers(3)]
        op_mode = int(rng.integers(2))
        unknowns = float(np.exp(rng.uniform(np.log(min_unknowns), np.log(max_unknowns))))
        n_rwg = unknowns / (2 if op_mode == 0 else 1)
        if shape == "cube":
            n = max(2, int(round(np.sqrt(n_rwg / 18.0))))     # 6 faces x 2 n^2 triangles, 1.5 edges per triangle
            v, t = cube(n, 1.0)
        else:
            nu = max(2, int(round(np.sqrt(n_rwg / 30.0))))    # 30 nu^2 edges
            v, t = icosphere(nu, 1.0) if shape == "sphere" else ellipsoid(nu, (1.0, 0.75, 0.5))
        p = v[t]
        mean_edge = float(np.mean(np.linalg.norm(p - np.roll(p, 1, axis=1), axis=2)))
        k0 = 2 * np.pi / (10.0 * mean_edge)
        nrhs = int(rng.integers(1, max_rhs + 1))
        kh = rng.standard_normal((nrhs, 3))
        kh /= np.linalg.norm(kh, axis=1, keepdims=True)
        ph = rng.standard_normal((nrhs, 3))
        ph -= np.sum(ph * kh, axis=1, keepdims=True) * kh
        ph /= np.linalg.norm(ph, axis=1, keepdims=True)
        out.append(dict(shape=shape, verts=v, tris=t, k0=k0, op_mode=op_mode, khat=kh, phat=ph))
    return out


def complex_gaussian(n: int, nrhs: int = 1, seed: int = SEED_BASE):
    """x = (N(0,1) + j N(0,1)) / sqrt(2), column-major [nrhs][n], complex128."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((nrhs, n))
    im = rng.standard_normal((nrhs, n))
    return ((re + 1j * im) / np.sqrt(2.0)).astype(np.complex128)


def sample_rows(n_total: int, count: int, seed: int):
    rng = np.random.default_rng(seed)
    count = min(count, n_total)
    return np.sort(rng.choice(n_total, size=count, replace=False)).astype(np.int32)


# Named workloads (sizes in wavelengths; k0 = 2*pi).
def workload(name: str):
    """Return (verts, tris, meta) for a named synthetic surface."""
    if name == "sphere_r0.5_nu8":          # PEC sphere radius 0.5 lambda, 1280 triangles
        v, t = icosphere(8, 0.5)
        return v, t, dict(radius=0.5, levels=3, leaf=0.25, seed=SEED_BASE + 0)
    if name == "sphere_r0.5_nu8_leaf0.125":
        v, t = icosphere(8, 0.5)
        return v, t, dict(radius=0.5, levels=4, leaf=0.125, seed=SEED_BASE + 0)
    if name == "sphere_r2_nu32":           # coated-sphere outer surface, radius 2 lambda, 20480 triangles
        v, t = icosphere(32, 2.0)
        return v, t, dict(radius=2.0, levels=5, leaf=0.25, seed=SEED_BASE + 1)
    if name == "cube5_cyl":                # cube 5 lambda with embedded cylinder
        v, t = cube_with_cylinder()
        return v, t, dict(levels=6, leaf=0.25, seed=SEED_BASE + 2)
    if name == "sphere_r20_nu241":         # large sphere radius 20 lambda, 1161620 triangles
        v, t = icosphere(241, 20.0)
        return v, t, dict(radius=20.0, levels=9, leaf=0.25, seed=SEED_BASE + 4)
    raise KeyError(name)
