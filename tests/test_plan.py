"""Host-only checks of the set-up of the multilevel product (bi_plan_*): RWG numbering, octree,
near and interaction lists of the MLFMA (Sec. II.D), parent-centred translation lists, angular
sampling, Lagrange interpolation between levels and the translation Hankel table.  The plan
runs the same host code as bi_setup without a device, so these run on any machine.  Every
expected value below follows from geometry, from the mathematics of the quadrature, the
interpolation and the special functions, from radiation patterns integrated directly (the
aggregation step), or from the oracle's dense operator (the whole multilevel chain, run in
numpy on the plan's tables); none comes from the library."""
import numpy as np
import pytest

from paper_2210_04892_gb300 import inputs

K0 = 2 * np.pi          # wavelength 1
NONE = 0xFFFF


@pytest.fixture(scope="module")
def bi():
    from paper_2210_04892_gb300 import bi as mod
    try:
        mod.load()
    except (ImportError, OSError) as e:  # pragma: no cover - library not built here
        pytest.skip(f"library not loadable: {e}")
    return mod


@pytest.fixture(scope="module")
def sphere():
    # sphere of radius 2 wavelengths: 5 levels with 0.25-wavelength leaves (far field on 2..4)
    v, t = inputs.icosphere(20, radius=2.0)
    return v, t


@pytest.fixture(scope="module")
def plan(bi, sphere):
    v, t = sphere
    p = bi.Plan(v, t, K0, digits=3)
    yield p
    p.close()


GEOMETRIES = {
    # 5 levels, one closed component
    "sphere_r2": lambda: inputs.icosphere(20, radius=2.0),
    # two disjoint closed components (cube with a cylinder inside), flat faces, ragged octree
    "cube_cylinder": lambda: inputs.cube_with_cylinder(size=2.0, h_face=1 / 6, h_edge=1 / 8, cyl_radius=0.4,
                                                       cyl_height=1.2, h_cyl=1 / 8),
    # elongated: many partly filled parents
    "ellipsoid": lambda: tuple(a * 3.0 if i == 0 else a for i, a in enumerate(inputs.ellipsoid(12))),
    # smaller than two leaf boxes: no far field, everything is near
    "tiny_sphere": lambda: inputs.icosphere(3, radius=0.1),
}


@pytest.fixture(scope="module", params=sorted(GEOMETRIES))
def geo_plan(bi, request):
    v, t = GEOMETRIES[request.param]()
    p = bi.Plan(v, t, K0, digits=3)
    yield request.param, v, t, p
    p.close()


def ancestors(plan, info):
    """anc[l][leaf box] = its ancestor at level l."""
    lf = info["leaf_level"]
    anc = {lf: np.arange(info["boxes"][lf])}
    for l in range(lf, 0, -1):
        anc[l - 1] = plan.get(4, l)[anc[l]]
    return anc


def test_rwg_numbering_is_the_interior_edges(plan, sphere):
    v, t = sphere
    info = plan.info()
    edges = plan.get(13).reshape(-1, 2)
    tp, tm = plan.get(14), plan.get(15)
    assert info["n_rwg"] == len(edges) == 3 * len(t) // 2     # closed surface: every edge shared
    assert info["n_unknowns"] == 2 * info["n_rwg"]             # J and M per RWG (Eq. 42)
    # each RWG's edge belongs to both of its triangles, traversed a -> b in T+ and b -> a in T-
    for n in range(0, len(edges), 97):
        a, b = edges[n]
        for tri, fwd in ((t[tp[n]], True), (t[tm[n]], False)):
            cyc = list(tri) + [tri[0]]
            pairs = {(cyc[k], cyc[k + 1]) for k in range(3)}
            assert ((a, b) in pairs) == fwd and ((b, a) in pairs) == (not fwd)
    assert len({(int(a), int(b)) for a, b in edges}) == len(edges)


def test_sphere_level_count(plan):
    info = plan.info()
    assert info["levels"] == 5 and info["leaf_level"] == 4


def test_octree_boxes_hold_their_rwgs(geo_plan):
    _, v, _, plan = geo_plan
    info = plan.info()
    lf = info["leaf_level"]
    perm = plan.get(12)
    assert np.array_equal(np.sort(perm), np.arange(info["n_rwg"]))
    start = plan.get(0)
    assert start[0] == 0 and start[-1] == info["n_rwg"] and np.all(np.diff(start) > 0)
    coords = plan.get(3, lf).reshape(-1, 3)
    edges = plan.get(13).reshape(-1, 2)
    mid = 0.5 * (v[edges[:, 0]] + v[edges[:, 1]])
    a = info["root_size"] / 2**lf
    assert a == pytest.approx(0.25)
    lo = 0.5 * (mid.min(0) + mid.max(0)) - 0.5 * info["root_size"]
    for b in range(len(coords)):
        m = mid[perm[start[b]:start[b + 1]]]
        cell = np.clip(np.floor((m - lo) / a).astype(int), 0, 2**lf - 1)
        assert np.all(cell == coords[b])
    # parents hold their children contiguously, each child's cell inside its parent's
    for l in range(1, lf + 1):
        par = plan.get(4, l)
        cp = plan.get(5, l - 1)
        assert np.all(np.diff(par) >= 0)
        assert np.array_equal(np.repeat(np.arange(len(cp) - 1), np.diff(cp)), par)
        assert np.all(np.diff(cp) <= 8) and np.all(np.diff(cp) >= 1)
        c = plan.get(3, l).reshape(-1, 3)
        pc = plan.get(3, l - 1).reshape(-1, 3)
        assert np.array_equal(c >> 1, pc[par])


def test_near_and_interactions_cover_every_pair_once(geo_plan):
    """Sec. II.D: a pair of leaf boxes is handled exactly once, either by the near-field blocks
    (touching boxes) or by one translation between ancestors that are not neighbours but whose
    parents are."""
    name, _, _, plan = geo_plan
    info = plan.info()
    lf = info["leaf_level"]
    nb = info["boxes"][lf]
    anc = ancestors(plan, info)
    cover = np.zeros((nb, nb), np.int32)
    nptr, nsrc = plan.get(1), plan.get(2)
    for b in range(nb):
        cover[b, nsrc[nptr[b]:nptr[b + 1]]] += 1
    coords_lf = plan.get(3, lf).reshape(-1, 3)
    for b in range(nb):
        s = nsrc[nptr[b]:nptr[b + 1]]
        assert np.all(np.abs(coords_lf[s] - coords_lf[b]).max(1) <= 1)
    total = 0
    for l in range(2, lf + 1):
        ptr, src = plan.get(6, l), plan.get(7, l)
        total += len(src)
        assert info["interactions"][l] == len(src)
        members = [np.flatnonzero(anc[l] == c) for c in range(info["boxes"][l])]
        for c in range(info["boxes"][l]):
            rows = members[c]
            for s in src[ptr[c]:ptr[c + 1]]:
                cover[np.ix_(rows, members[s])] += 1
    assert (total > 0) == (lf >= 2), (name, lf)
    assert np.all(cover == 1), np.unique(cover, return_counts=True)


def _neighbour_pairs(coords):
    """(box, other) index pairs of the boxes of one level at Chebyshev distance <= 1 (the box
    itself included), from their integer cell coordinates."""
    key = (coords[:, 0].astype(np.int64) << 40) | (coords[:, 1].astype(np.int64) << 20) | coords[:, 2]
    order = np.argsort(key)
    skey = key[order]
    a_all, b_all = [], []
    for d in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")).reshape(3, -1).T:
        c = coords + d
        ok = np.all(c >= 0, axis=1)
        k = (c[:, 0].astype(np.int64) << 40) | (c[:, 1].astype(np.int64) << 20) | c[:, 2]
        i = np.minimum(np.searchsorted(skey, k), len(skey) - 1)
        hit = ok & (skey[i] == k)
        a_all.append(np.flatnonzero(hit))
        b_all.append(order[i[hit]])
    return np.concatenate(a_all), np.concatenate(b_all)


@pytest.mark.slow
def test_headline_tree_lists_at_full_size(bi):
    """The set-up lists of the large scatterer itself (sphere of radius 20 wavelengths,
    1,742,430 RWG, 9 levels, 110,456 leaf boxes), checked exhaustively rather than by sampled
    rows, from the boxes' cell coordinates alone:
    - every RWG sits in the leaf box of its midpoint's cell, and every child in its parent;
    - the near list of each leaf box is exactly its existing neighbours (Chebyshev distance
      <= 1, itself included);
    - on every level l >= 2, the children of the neighbours of a box's parent split exactly
      into the box's own neighbours and its interaction list (Sec. II.D), with no entry twice;
    - the offset codes are the coordinate differences, and the parent-centred lists hold the
      same (box, source, code) triples as the per-box lists.
    With level 1 (whose boxes all touch) as the start, the split on every level covers each
    pair of leaf boxes exactly once: by a near block if the two touch, else by the one
    translation between their ancestors on the finest level where those do not touch."""
    v, t, meta = inputs.workload("sphere_r20_nu241")
    p = bi.Plan(v, t, K0, digits=3)
    info = p.info()
    lf = info["leaf_level"]
    assert info["levels"] == 9 and info["n_rwg"] == 1742430 and info["boxes"][lf] == 110456
    # octree membership, vectorised over the RWGs
    perm, start = p.get(12), p.get(0)
    edges = p.get(13).reshape(-1, 2)
    mid = 0.5 * (v[edges[:, 0]] + v[edges[:, 1]])
    lo = 0.5 * (mid.min(0) + mid.max(0)) - 0.5 * info["root_size"]
    a = info["root_size"] / 2 ** lf
    cell = np.clip(np.floor((mid - lo) / a).astype(np.int64), 0, 2 ** lf - 1)
    box_of_tree_pos = np.repeat(np.arange(len(start) - 1), np.diff(start))
    coords = {l: p.get(3, l).reshape(-1, 3).astype(np.int64) for l in range(lf + 1)}
    assert np.array_equal(cell[perm], coords[lf][box_of_tree_pos])
    for l in range(1, lf + 1):
        assert np.array_equal(coords[l] >> 1, coords[l - 1][p.get(4, l)])
    # near lists at the leaf level = existing neighbours
    nb = info["boxes"][lf]
    na, nn = _neighbour_pairs(coords[lf])
    nptr, nsrc = p.get(1), p.get(2)
    near = np.repeat(np.arange(nb), np.diff(nptr)).astype(np.int64) * nb + nsrc
    assert len(np.unique(near)) == len(near)
    assert np.array_equal(np.sort(near), np.sort(na.astype(np.int64) * nb + nn))
    for l in range(2, lf + 1):
        n_l = info["boxes"][l]
        cp = p.get(5, l - 1)                      # children of each box of level l - 1
        # children of the parent's neighbours, for every box of level l
        qa, qb = _neighbour_pairs(coords[l - 1])
        nq, nr = np.diff(cp)[qa], np.diff(cp)[qb]
        cnt = nq * nr
        grp = np.repeat(np.arange(len(qa)), cnt)
        k = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        c = cp[qa][grp] + k // nr[grp]
        s = cp[qb][grp] + k % nr[grp]
        cand = np.sort(c.astype(np.int64) * n_l + s)
        assert len(np.unique(cand)) == len(cand)
        la, lb = _neighbour_pairs(coords[l])
        nbr = la.astype(np.int64) * n_l + lb
        ptr, src, off = p.get(6, l), p.get(7, l), p.get(8, l)
        recv = np.repeat(np.arange(n_l), np.diff(ptr)).astype(np.int64)
        il = recv * n_l + src
        assert info["interactions"][l] == len(il) and len(np.unique(il)) == len(il), l
        assert np.array_equal(np.sort(np.concatenate([nbr, il])), cand), l
        o = coords[l][recv] - coords[l][src]
        assert np.array_equal(off, (o[:, 0] + 3) * 49 + (o[:, 1] + 3) * 7 + (o[:, 2] + 3)), l
        # parent-centred lists: the same (box, source, code) triples
        tptr, tsrc = p.get(9, l), p.get(10, l)
        tcode = p.get(11, l).reshape(-1, 8).astype(np.int64)
        par_of_row = np.repeat(np.arange(len(tptr) - 1), np.diff(tptr))
        slot_box = cp[par_of_row][:, None] + np.arange(8)[None, :]
        live = tcode != NONE
        assert np.all(slot_box[live] < cp[par_of_row + 1][np.nonzero(live)[0]]), l
        pc_keys = (slot_box[live].astype(np.int64) * n_l + np.repeat(tsrc, 8).reshape(-1, 8)[live]) * 344 + tcode[live]
        pl_keys = il * 344 + off
        assert np.array_equal(np.sort(pc_keys), np.sort(pl_keys)), l
    p.close()


def test_interaction_offsets_match_box_coordinates(geo_plan):
    plan = geo_plan[3]
    info = plan.info()
    for l in range(2, info["leaf_level"] + 1):
        c = plan.get(3, l).reshape(-1, 3)
        par = plan.get(4, l)
        pc = plan.get(3, l - 1).reshape(-1, 3)
        ptr, src, off = plan.get(6, l), plan.get(7, l), plan.get(8, l)
        recv = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
        o = c[recv] - c[src]
        assert np.array_equal(off, (o[:, 0] + 3) * 49 + (o[:, 1] + 3) * 7 + (o[:, 2] + 3))
        cheb = np.abs(o).max(1)
        assert np.all(cheb >= 2) and np.all(cheb <= 3)
        assert np.all(np.abs(pc[par[recv]] - pc[par[src]]).max(1) <= 1)


def test_parent_centred_lists_equal_the_interaction_lists(geo_plan):
    plan = geo_plan[3]
    info = plan.info()
    for l in range(2, info["leaf_level"] + 1):
        cp = plan.get(5, l - 1)
        ptr, src, off = plan.get(6, l), plan.get(7, l), plan.get(8, l)
        tptr, tsrc = plan.get(9, l), plan.get(10, l)
        tcode = plan.get(11, l).reshape(-1, 8)
        assert len(tptr) == len(cp) and len(tsrc) == len(tcode)
        n_live = 0
        for p in range(len(cp) - 1):
            for j in range(8):
                if cp[p] + j >= cp[p + 1]:
                    assert np.all(tcode[tptr[p]:tptr[p + 1], j] == NONE)
                    continue
                b = cp[p] + j
                got = {(int(s), int(k)) for s, k in zip(tsrc[tptr[p]:tptr[p + 1]], tcode[tptr[p]:tptr[p + 1], j])
                       if k != NONE}
                want = {(int(s), int(k)) for s, k in zip(src[ptr[b]:ptr[b + 1]], off[ptr[b]:ptr[b + 1]])}
                assert got == want, (l, p, j)
                n_live += len(got)
        assert n_live == len(src)
        # no source entry without a live slot, and no source twice for one parent
        assert np.all((tcode != NONE).any(1))
        for p in range(len(cp) - 1):
            s = tsrc[tptr[p]:tptr[p + 1]]
            assert len(np.unique(s)) == len(s)


def test_theta_sampling_is_gauss_legendre(plan):
    info = plan.info()
    for l in range(2, info["leaf_level"] + 1):
        th, w = plan.get(20, l), plan.get(21, l)
        L = info["L"][l]
        assert len(th) == L + 1 and info["K"][l] == (L + 1) * 2 * (L + 1)
        assert np.all(np.diff(th) > 0) and th[0] > 0 and th[-1] < np.pi
        x = np.cos(th)
        assert np.allclose(x, -x[::-1], atol=1e-14) and np.allclose(w, w[::-1], rtol=1e-12)
        # exact for polynomials of degree 2n - 1 in cos(theta)
        for k in range(2 * len(x)):
            exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
            assert abs(np.dot(w, x**k) - exact) < 1e-12, (l, k)
        # the bandwidth covers at least the box diagonal k*sqrt(3)*a (excess-bandwidth rule)
        a = info["root_size"] / 2**l
        assert L >= K0 * np.sqrt(3) * a
    Ls = [info["L"][l] for l in range(2, info["leaf_level"] + 1)]
    assert all(p > c for p, c in zip(Ls, Ls[1:]))


def interp_matrices(plan, l, nth_c, nph_c, nth_p, nph_p):
    """Dense theta and phi interpolation of the transverse components from level l + 1 to l,
    as the tap lists define them (a theta tap with the flip bit reads the column half a turn
    away and negates both components)."""
    src, flip, w = plan.get(22, l), plan.get(23, l), plan.get(24, l)
    p_th = len(src) // nth_p
    Kc = nth_c * nph_c
    A = np.zeros((nth_p * nph_c, Kc))
    for ip in range(nth_p):
        for t in range(p_th):
            e = ip * p_th + t
            for jc in range(nph_c):
                jj = (jc + nph_c // 2) % nph_c if flip[e] else jc
                A[ip * nph_c + jc, src[e] * nph_c + jj] += -w[e] if flip[e] else w[e]
    ps, pw = plan.get(25, l), plan.get(26, l)
    p_ph = len(ps) // nph_p
    B = np.zeros((nph_p, nph_c))
    for jp in range(nph_p):
        for q in range(p_ph):
            B[jp, ps[jp * p_ph + q]] += pw[jp * p_ph + q]
    return A, B, p_th, p_ph


def transverse_field(theta, phi, k0, sources):
    """Theta and phi components of sum_i (I - k k) p_i exp(j k0 k . r_i) on a (theta, phi) grid:
    the radiation pattern of a few point dipoles, a smooth transverse field on the sphere."""
    T, P = np.meshgrid(theta, phi, indexing="ij")
    kh = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    th = np.stack([np.cos(T) * np.cos(P), np.cos(T) * np.sin(P), -np.sin(T)], -1)
    ph = np.stack([-np.sin(P), np.cos(P), np.zeros_like(P)], -1)
    F = np.zeros(T.shape + (3,), complex)
    for r, pvec in sources:
        F += np.exp(1j * k0 * kh @ r)[..., None] * pvec
    return np.sum(F * th, -1), np.sum(F * ph, -1)


def test_interpolation_weights_and_transposes(plan):
    info = plan.info()
    for l in range(2, info["leaf_level"]):
        nth_c, nph_c = info["L"][l + 1] + 1, 2 * (info["L"][l + 1] + 1)
        nth_p, nph_p = info["L"][l] + 1, 2 * (info["L"][l] + 1)
        src, flip, w = plan.get(22, l), plan.get(23, l), plan.get(24, l)
        ps, pw = plan.get(25, l), plan.get(26, l)
        p_th, p_ph = len(src) // nth_p, len(ps) // nph_p
        assert p_th == min(10, nth_c) and p_ph == min(10, nph_c)
        # Lagrange weights reproduce constants
        assert np.allclose(w.reshape(nth_p, p_th).sum(1), 1.0, atol=1e-12)
        assert np.allclose(pw.reshape(nph_p, p_ph).sum(1), 1.0, atol=1e-12)
        assert np.all((src >= 0) & (src < nth_c)) and np.all((ps >= 0) & (ps < nph_c))
        # the transposed lists are exactly the transposes of the forward lists
        fwd = {}
        for ip in range(nth_p):
            for t in range(p_th):
                e = ip * p_th + t
                key = (int(src[e]), ip, int(flip[e]))
                fwd[key] = fwd.get(key, 0.0) + w[e]
        tptr, tdst, tflip, tw = plan.get(27, l), plan.get(28, l), plan.get(29, l), plan.get(30, l)
        assert len(tptr) == nth_c + 1 and tptr[-1] == len(src)
        back = {}
        for ic in range(nth_c):
            for q in range(tptr[ic], tptr[ic + 1]):
                key = (ic, int(tdst[q]), int(tflip[q]))
                back[key] = back.get(key, 0.0) + tw[q]
        assert fwd.keys() == back.keys()
        assert all(abs(fwd[k] - back[k]) < 1e-15 for k in fwd)
        fph, bph = np.zeros((nph_p, nph_c)), np.zeros((nph_p, nph_c))
        for jp in range(nph_p):
            for q in range(p_ph):
                fph[jp, ps[jp * p_ph + q]] += pw[jp * p_ph + q]
        pptr, pdst, pwt = plan.get(31, l), plan.get(32, l), plan.get(33, l)
        assert len(pptr) == nph_c + 1
        for jc in range(nph_c):
            for q in range(pptr[jc], pptr[jc + 1]):
                bph[pdst[q], jc] += pwt[q]
        assert np.allclose(fph, bph, rtol=0, atol=1e-15)


def interp_error(plan, info, l, sources, drop_reflection_sign=False):
    """Largest error, relative to the field's peak, of interpolating the dipole pattern from
    the level-(l + 1) grid to the level-l grid through the plan's tap lists."""
    Lc, Lp = info["L"][l + 1], info["L"][l]
    nth_c, nph_c, nth_p, nph_p = Lc + 1, 2 * (Lc + 1), Lp + 1, 2 * (Lp + 1)
    th_c, th_p = plan.get(20, l + 1), plan.get(20, l)
    ph_c = 2 * np.pi * np.arange(nph_c) / nph_c
    ph_p = 2 * np.pi * np.arange(nph_p) / nph_p
    A, B, _, _ = interp_matrices(plan, l, nth_c, nph_c, nth_p, nph_p)
    if drop_reflection_sign:
        A = np.abs(A)
    ref = transverse_field(th_p, ph_p, K0, sources)
    scale = max(np.abs(r).max() for r in ref)
    err = 0.0
    for comp, r in zip(transverse_field(th_c, ph_c, K0, sources), ref):
        out = (A @ comp.reshape(-1)).reshape(nth_p, nph_c) @ B.T
        err = max(err, np.abs(out - r).max() / scale)
    return err


def dipoles_in_box(rng, a, count=6):
    out = []
    for _ in range(count):
        d = rng.normal(size=3)
        out.append((0.5 * a * rng.uniform(-1, 1, 3), d / np.linalg.norm(d)))
    return out


def test_interpolation_of_a_transverse_field_across_the_poles(plan):
    """Interpolating the pattern of dipoles inside a child box to the parent's denser grid
    (theta pass with pole reflection, then phi) reproduces the field sampled directly.  The
    reflection sign matters: dropping it leaves O(1) errors near the poles."""
    info = plan.info()
    rng = np.random.default_rng(inputs.SEED_BASE + 77)
    for l in range(2, info["leaf_level"]):
        src = dipoles_in_box(rng, info["root_size"] / 2 ** (l + 1))
        # order-10 local Lagrange on the excess-bandwidth grids: a few 1e-6 measured
        assert interp_error(plan, info, l, src) < 5e-5, l
        assert interp_error(plan, info, l, src, drop_reflection_sign=True) > 1e-2, l


def test_interpolation_error_falls_with_the_order(bi, sphere):
    v, t = sphere
    rng = np.random.default_rng(inputs.SEED_BASE + 78)
    errs = []
    for order in (4, 6, 10):
        p = bi.Plan(v, t, K0, digits=3, interp_order=order)
        info = p.info()
        src = dipoles_in_box(np.random.default_rng(inputs.SEED_BASE + 78), info["root_size"] / 2**3)
        errs.append(interp_error(p, info, 2, src))
        p.close()
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[0] / errs[2] > 30, errs


def test_plan_rejects_open_and_bad_meshes(bi):
    v, t = inputs.icosphere(4)
    with pytest.raises(bi.BIError):
        bi.Plan(v, t[:-1], K0)                    # one triangle removed: open surface
    bad = t.copy()
    bad[0] = bad[0][::-1]
    with pytest.raises(bi.BIError):
        bi.Plan(v, bad, K0)                       # inconsistent orientation
    with pytest.raises(bi.BIError):
        bi.Plan(v, t, -1.0)
    for bad in (dict(digits=0), dict(digits=-2), dict(leaf_box=0.0), dict(leaf_box=float("nan")),
                dict(interp_order=1), dict(levels=22), dict(op_mode=2)):
        with pytest.raises(bi.BIError):
            bi.Plan(v, t, K0, **bad)              # the parameter ranges of bi_setup
    p = bi.Plan(v, t, K0)
    with pytest.raises(bi.BIError):
        p.get(99)
    with pytest.raises(bi.BIError):
        p.get(6, 1)                               # no interaction list above level 2
    p.close()


def test_plan_rejects_degenerate_inputs_and_accepts_the_smallest_surface(bi):
    """The error contract of the set-up on degenerate input (the same checks run in bi_setup
    before any device work): an empty mesh, vertex indices outside the vertex array, non-finite
    coordinates, a triangle with a repeated or collinear vertex (zero area), and edges shared
    by more than two triangles are refused with BI_ERR_ARG or BI_ERR_MESH; the smallest closed
    surface, a tetrahedron, is accepted with its 6 RWG functions."""
    v, t = inputs.icosphere(4)
    cases = {"empty mesh": (v, np.zeros((0, 3), np.int32))}
    t2 = t.copy()
    t2[0, 1] = len(v) + 5
    cases["index past the vertices"] = (v, t2)
    t2 = t.copy()
    t2[0, 1] = -1
    cases["negative index"] = (v, t2)
    for bad in (np.nan, np.inf):
        v2 = v.copy()
        v2[3] = bad
        cases["vertex %r" % bad] = (v2, t)
    t2 = t.copy()
    t2[0, 1] = t2[0, 0]
    cases["repeated vertex"] = (v, t2)
    v2 = v.copy()
    a, b, c = t[0]
    v2[c] = 0.5 * (v2[a] + v2[b])
    cases["collinear triangle"] = (v2, t)
    cases["duplicated triangle"] = (v, np.concatenate([t, t[:1]]))
    tv = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]) * 0.1
    tt = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    # a second tetrahedron on the edge (0, 1): four triangles on one edge
    V = np.concatenate([tv, [[0, -0.1, 0], [0, 0, -0.1]]])
    T = np.concatenate([tt, np.array([[0, 4, 1], [0, 1, 5], [0, 5, 4], [1, 4, 5]], np.int32)])
    cases["non-manifold edge"] = (V, T)
    for name, (vv, ttt) in cases.items():
        with pytest.raises(bi.BIError) as e:
            bi.Plan(vv, ttt, K0)
        assert e.value.code in (bi.BI_ERR_ARG, bi.BI_ERR_MESH), name
    with pytest.raises(bi.BIError):
        bi.Plan(v, t, float("nan"))
    p = bi.Plan(tv, tt, K0)
    info = p.info()
    assert info["n_rwg"] == 6 and info["levels"] == 1
    p.close()


@pytest.mark.parametrize("digits,leaf_box", [(3, 0.25), (6, 0.125)])
def test_translation_hankel_table(bi, sphere, digits, leaf_box):
    """Spherical Hankel functions h_n^(2)(k|X|) = j_n - i y_n behind the translation operators
    of every level, for every far offset, against scipy.  j_n comes from Miller's downward
    recurrence, so beyond the turning point (n > x) it must keep its relative accuracy too;
    near its zeros only the absolute error is meaningful."""
    special = pytest.importorskip("scipy.special")
    v, t = sphere
    p = bi.Plan(v, t, K0, digits=digits, leaf_box=leaf_box)
    info = p.info()
    for l in range(2, info["leaf_level"] + 1):
        L = info["L"][l]
        di = p.get(40, l)
        hk = p.get(41, l).reshape(-1, L + 1, 2)
        a = info["root_size"] / 2**l
        sq = set()
        for o in range(343):
            off = np.array([o // 49 - 3, (o // 7) % 7 - 3, o % 7 - 3])
            if np.abs(off).max() <= 1:
                assert di[o] == -1
                continue
            sq.add(int(off @ off))
            x = K0 * a * np.linalg.norm(off)
            n = np.arange(L + 1)
            j, y = special.spherical_jn(n, x), special.spherical_yn(n, x)
            g = hk[di[o]]
            assert np.abs(g[:, 0] - j).max() < 1e-13, (l, o)
            h = j - 1j * y
            assert np.all(np.abs(g[:, 0] + 1j * g[:, 1] - h) <= 1e-13 * np.abs(h)), (l, o)
            deep = n > x + 2
            if deep.any():
                assert np.all(np.abs(g[deep, 0] - j[deep]) <= 1e-12 * np.abs(j[deep])), (l, o)
        assert di.max() + 1 == len(sq) == 15      # distinct |X|^2 among the 316 far offsets
    p.close()


def test_translation_hankel_table_at_complex_k(bi, sphere):
    """The same table for a lossy medium (the coating's k1 = k0 sqrt(2 - 0.5j)): h_n^(2) of the
    complex argument k1 |X| on every level against scipy.  Here y_n runs upward and j_n
    downward, normalised with the closed form of the larger of j_0, j_1 (neither vanishes off
    the real axis).  At low orders and large |Im z| (8 on the coarsest level) h_n is the small
    difference of j_n and j y_n, each about e^|Im z| / |z|: the error is bounded against
    |j_n| + |y_n|, and relative to h_n wherever no such cancellation occurs."""
    special = pytest.importorskip("scipy.special")
    v, t = sphere
    k1 = K0 * np.sqrt(2.0 - 0.5j)
    p = bi.Plan(v, t, k1, digits=3)
    info = p.info()
    assert info["levels"] >= 5
    for l in range(2, info["leaf_level"] + 1):
        L = info["L"][l]
        di = p.get(40, l)
        hk = p.get(41, l).reshape(-1, L + 1, 2)
        a = info["root_size"] / 2**l
        for o in range(343):
            off = np.array([o // 49 - 3, (o // 7) % 7 - 3, o % 7 - 3])
            if np.abs(off).max() <= 1:
                continue
            z = k1 * a * np.linalg.norm(off)
            n = np.arange(L + 1)
            j, y = special.spherical_jn(n, z), special.spherical_yn(n, z)
            h = j - 1j * y
            g = hk[di[o]]
            err = np.abs(g[:, 0] + 1j * g[:, 1] - h)
            assert np.all(err <= 1e-12 * (np.abs(j) + np.abs(y))), (l, o)
            if abs(z.imag) < 2:
                assert np.all(err <= 1e-11 * np.abs(h)), (l, o)
    p.close()


def _rwg_pattern_subset(v, t, rwg, idx, k, khat, center, twisted=False):
    """int f_n exp(+jk khat.(r - center)) dS for the RWG indices idx (numpy: a 6 x 6 conical
    Gauss rule on each of the four midpoint sub-triangles of every triangle); with `twisted`,
    n x f_n in place of f_n (n the triangle's outward normal)."""
    e, tp, tm, lp, lm = rwg["edges"], rwg["tplus"], rwg["tminus"], rwg["lplus"], rwg["lminus"]
    g, gw = np.polynomial.legendre.leggauss(6)
    g, gw = (g + 1) / 2, gw / 2
    U, V = np.meshgrid(g, g, indexing="ij")
    b1, b2 = U.ravel(), ((1 - U) * V).ravel()
    ww = (np.outer(gw, gw) * (1 - U)).ravel() * 2
    P = np.zeros((len(idx), len(khat), 3), complex)
    for j, n in enumerate(idx):
        length = np.linalg.norm(v[e[n, 1]] - v[e[n, 0]])
        for tri, loc, s in ((tp[n], lp[n], 1.0), (tm[n], lm[n], -1.0)):
            T = v[t[tri]]
            nrm = np.cross(T[1] - T[0], T[2] - T[0])
            area = np.linalg.norm(nrm) / 2
            m01, m12, m20 = (T[0] + T[1]) / 2, (T[1] + T[2]) / 2, (T[2] + T[0]) / 2
            for S in ((T[0], m01, m20), (m01, T[1], m12), (m20, m12, T[2]), (m01, m12, m20)):
                x = S[0] + b1[:, None] * (S[1] - S[0]) + b2[:, None] * (S[2] - S[0])
                f = s * (length / (2 * area)) * (x - T[loc])
                if twisted:
                    f = np.cross(nrm / (2 * area), f)
                ph = np.exp(1j * k * ((x - center) @ khat.T))
                P[j] += np.einsum("q,qd,qc->dc", ww * area / 4, ph, f)
    return P


def _directions(theta, nph):
    TH, PH = np.meshgrid(theta, 2 * np.pi * np.arange(nph) / nph, indexing="ij")
    kh = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    th = np.stack([np.cos(TH) * np.cos(PH), np.cos(TH) * np.sin(PH), -np.sin(TH)], -1).reshape(-1, 3)
    ph = np.stack([-np.sin(PH), np.cos(PH), 0 * PH], -1).reshape(-1, 3)
    return kh, th, ph


@pytest.mark.parametrize("k", [K0, K0 * np.sqrt(2.0 - 0.5j)], ids=["real_k", "lossy_k"])
def test_aggregation_step_reproduces_the_parent_pattern(bi, k):
    """One upward step of the multilevel product, with the plan's tables: each child box's
    outgoing pattern (RWG radiation patterns about the child centre, random coefficients) is
    interpolated to the parent grid and multiplied by exp(+jk khat.(c_child - c_parent)); the
    sum over the children equals the pattern computed directly about the parent centre, in
    both transverse components.  The opposite shift sign fails.  At the coating's complex k
    the sampling comes from Re k."""
    import oracle
    v, t = inputs.icosphere(16, 1.0)
    p = bi.Plan(v, t, float(np.real(k)), digits=3)
    info = p.info()
    lf = info["leaf_level"]
    l = lf - 1
    a = info["root_size"] / 2 ** l
    edges, perm, start = p.get(13).reshape(-1, 2), p.get(12), p.get(0)
    mid = 0.5 * (v[edges[:, 0]] + v[edges[:, 1]])
    lo = 0.5 * (mid.min(0) + mid.max(0)) - 0.5 * info["root_size"]
    cp, cc, pc = p.get(5, l), p.get(3, lf).reshape(-1, 3), p.get(3, l).reshape(-1, 3)
    q = int(np.argmax(np.diff(cp)))                     # the parent with the most children
    c_par = lo + (pc[q] + 0.5) * a
    nth_c, nph_c = info["L"][lf] + 1, 2 * (info["L"][lf] + 1)
    nth_p, nph_p = info["L"][l] + 1, 2 * (info["L"][l] + 1)
    khc, thc, phc = _directions(p.get(20, lf), nph_c)
    khp, thp, php = _directions(p.get(20, l), nph_p)
    A, B, _, _ = interp_matrices(p, l, nth_c, nph_c, nth_p, nph_p)
    rwg = oracle.rwg(v, t)
    rng = np.random.default_rng(inputs.SEED_BASE + 79)
    direct = np.zeros((len(khp), 3), complex)
    up = {+1: [0, 0], -1: [0, 0]}
    for b in range(cp[q], cp[q + 1]):
        c_ch = lo + (cc[b] + 0.5) * (a / 2)
        rows = perm[start[b]:start[b + 1]]
        x = rng.normal(size=len(rows)) + 1j * rng.normal(size=len(rows))
        Fc = np.einsum("n,ndc->dc", x, _rwg_pattern_subset(v, t, rwg, rows, k, khc, c_ch))
        direct += np.einsum("n,ndc->dc", x, _rwg_pattern_subset(v, t, rwg, rows, k, khp, c_par))
        for sgn in (+1, -1):
            sh = np.exp(sgn * 1j * k * (khp @ (c_ch - c_par)))
            for i, comp in enumerate((thc, phc)):
                g = (A @ np.einsum("dc,dc->d", Fc, comp)).reshape(nth_p, nph_c) @ B.T
                up[sgn][i] = up[sgn][i] + g.reshape(-1) * sh
    ref = [np.einsum("dc,dc->d", direct, thp), np.einsum("dc,dc->d", direct, php)]
    scale = max(np.abs(r).max() for r in ref)
    err = {s: max(np.abs(up[s][i] - ref[i]).max() for i in range(2)) / scale for s in (+1, -1)}
    assert err[+1] < 1e-4, err
    assert err[-1] > 0.1, err


class _MultilevelModel:
    """The multilevel product in numpy, built only from the plan's tables (sampling from
    Re k, interpolation taps, interaction lists, box tree) for one wavenumber k:
    - leaf patterns F and R (integrated separately: at complex k, R is not conj F);
    - upward interpolation and shift;
    - diagonal translations T_L, with weights and -jk/16 pi^2 folded in;
    - downward shift and exact-transpose anterpolation.
    `propagate` maps the outgoing theta/phi fields of the leaf boxes to their incoming ones;
    the operator-specific outgoing fields and receive sums are left to the caller."""

    def __init__(self, bi, v, t, k, leaf, digits):
        import oracle
        self.k = k
        self.p = p = bi.Plan(v, t, float(np.real(k)), digits=digits, leaf_box=leaf)
        self.info = info = p.info()
        self.lf = lf = info["leaf_level"]
        self.rwg = rwg = oracle.rwg(v, t)
        edges, self.perm, self.start = p.get(13).reshape(-1, 2), p.get(12), p.get(0)
        mid = 0.5 * (v[edges[:, 0]] + v[edges[:, 1]])
        lo = 0.5 * (mid.min(0) + mid.max(0)) - 0.5 * info["root_size"]
        self.size = {l: info["root_size"] / 2 ** l for l in range(lf + 1)}
        self.cen = {l: lo + (p.get(3, l).reshape(-1, 3) + 0.5) * self.size[l] for l in range(2, lf + 1)}
        self.grids = {}
        for l in range(2, lf + 1):
            nth, nph = info["L"][l] + 1, 2 * (info["L"][l] + 1)
            self.grids[l] = (nth, nph) + _directions(p.get(20, l), nph) + (p.get(21, l),)
        nth, nph, kh, th, ph, _ = self.grids[lf]
        self.N = N = len(rwg["edges"])
        self.nb = nb = info["boxes"][lf]
        self.F = np.zeros((2, N, nth * nph), complex)       # theta, phi components
        self.R = np.zeros_like(self.F)
        for b in range(nb):
            rows = self.rows(b)
            Fp = _rwg_pattern_subset(v, t, rwg, rows, k, kh, self.cen[lf][b])
            Rp = _rwg_pattern_subset(v, t, rwg, rows, -k, kh, self.cen[lf][b])   # exp(-jk khat.(r - c))
            for i, comp in enumerate((th, ph)):
                self.F[i, rows] = np.einsum("ndc,dc->nd", Fp, comp)
                self.R[i, rows] = np.einsum("ndc,dc->nd", Rp, comp)
        self.interp = {}
        for l in range(lf - 1, 1, -1):
            nthc, nphc = self.grids[l + 1][:2]
            nthp, nphp = self.grids[l][:2]
            A, B, _, _ = interp_matrices(p, l, nthc, nphc, nthp, nphp)
            self.interp[l] = (A, B)
        self.T = {l: {} for l in range(2, lf + 1)}

    def rows(self, b):
        return self.perm[self.start[b]:self.start[b + 1]]

    def outgoing(self, xa, xb):
        """Leaf outgoing fields of sum_n (xa_n F_n + xb_n khat x F_n), theta/phi components
        ((khat x F)_theta = -F_phi, (khat x F)_phi = F_theta)."""
        U = np.zeros((self.nb, 2, self.F.shape[2]), complex)
        for b in range(self.nb):
            r = self.rows(b)
            U[b, 0] = xa[r] @ self.F[0, r] - xb[r] @ self.F[1, r]
            U[b, 1] = xa[r] @ self.F[1, r] + xb[r] @ self.F[0, r]
        return U

    def _translation(self, l, o):
        from scipy import special
        if o not in self.T[l]:
            k = self.k
            nthl, nphl, khl, _, _, wl = self.grids[l]
            W = (wl[:, None] * np.ones(nphl)[None, :] * 2 * np.pi / nphl).ravel()
            X = np.array([o // 49 - 3, (o // 7) % 7 - 3, o % 7 - 3]) * self.size[l]
            Xn = np.linalg.norm(X)
            cg = khl @ (X / Xn)
            Lt = self.info["L"][l]
            h2 = [special.spherical_jn(n, k * Xn) - 1j * special.spherical_yn(n, k * Xn) for n in range(Lt + 1)]
            T = sum((-1j) ** n * (2 * n + 1) * h2[n] * special.eval_legendre(n, cg) for n in range(Lt + 1))
            self.T[l][o] = (-1j * k / (16 * np.pi ** 2)) * W * T
        return self.T[l][o]

    def propagate(self, U_leaf):
        p, info, lf, k, cen, grids = self.p, self.info, self.lf, self.k, self.cen, self.grids
        U = {lf: U_leaf}
        for l in range(lf - 1, 1, -1):
            A, B = self.interp[l]
            nphc = grids[l + 1][1]
            nthp, nphp, khp = grids[l][:3]
            cp = p.get(5, l)
            U[l] = np.zeros((info["boxes"][l], 2, nthp * nphp), complex)
            for q in range(info["boxes"][l]):
                for c in range(cp[q], cp[q + 1]):
                    sh = np.exp(1j * k * (khp @ (cen[l + 1][c] - cen[l][q])))
                    for i in range(2):
                        U[l][q, i] += ((A @ U[l + 1][c, i]).reshape(nthp, nphc) @ B.T).reshape(-1) * sh
        V = {l: np.zeros_like(U[l]) for l in U}
        for l in range(2, lf + 1):
            ptr, src, off = p.get(6, l), p.get(7, l), p.get(8, l)
            for b in range(info["boxes"][l]):
                for e in range(ptr[b], ptr[b + 1]):
                    V[l][b] += self._translation(l, int(off[e]))[None] * U[l][src[e]]
        for l in range(2, lf):
            A, B = self.interp[l]
            nthp, nphp, khp = grids[l][:3]
            cp = p.get(5, l)
            for q in range(info["boxes"][l]):
                for c in range(cp[q], cp[q + 1]):
                    sh = np.exp(-1j * k * (khp @ (cen[l + 1][c] - cen[l][q])))
                    for i in range(2):
                        V[l + 1][c, i] += A.T @ ((V[l][q, i] * sh).reshape(nthp, nphp) @ B).reshape(-1)
        return V[lf]

    def receive(self, V, twisted=False):
        """-jk sum_khat R_m . V (twisted: R_m . (khat x V)) for every RWG m."""
        y = np.zeros(self.N, complex)
        for b in range(self.nb):
            r = self.rows(b)
            if twisted:
                y[r] = -1j * self.k * (-self.R[0, r] @ V[b, 1] + self.R[1, r] @ V[b, 0])
            else:
                y[r] = -1j * self.k * (self.R[0, r] @ V[b, 0] + self.R[1, r] @ V[b, 1])
        return y

    def near(self, Z, x):
        """Near-pair part of the dense N x N block Z times x (pairs of this plan's near lists)."""
        nptr, nsrc = self.p.get(1), self.p.get(2)
        y = np.zeros(self.N, complex)
        for b in range(self.nb):
            rb = self.rows(b)
            cols = np.concatenate([self.rows(s) for s in nsrc[nptr[b]:nptr[b + 1]]])
            y[rb] += Z[np.ix_(rb, cols)] @ x[cols]
        return y


def _multilevel_L_product(bi, k, nu, radius, leaf, digits):
    """<f, L f> x by the multilevel model (far pairs) plus the oracle's dense near pairs.
    Returns (levels, relative error of the whole product, relative error of its far part)
    against the oracle's dense product."""
    import oracle
    v, t = inputs.icosphere(nu, radius)
    m = _MultilevelModel(bi, v, t, k, leaf, digits)
    rng = np.random.default_rng(inputs.SEED_BASE + 80)
    x = rng.normal(size=m.N) + 1j * rng.normal(size=m.N)
    yfar = m.receive(m.propagate(m.outgoing(x, np.zeros(m.N))))
    Ld, _, _, _ = oracle.operators(v, t, k, 0)
    ynear = m.near(Ld, x)
    ref = Ld @ x
    err_all = np.linalg.norm(ynear + yfar - ref) / np.linalg.norm(ref)
    err_far = np.linalg.norm(yfar - (ref - ynear)) / np.linalg.norm(ref - ynear)
    return m.info["levels"], err_all, err_far


@pytest.mark.slow
@pytest.mark.parametrize("k", [K0, K0 * np.sqrt(2.0 - 0.5j)], ids=["real_k", "lossy_k"])
def test_multilevel_product_model_matches_the_dense_operator(bi, k):
    """The whole multilevel chain on the 1280-triangle sphere of radius 0.5 lambda, with leaf
    boxes of a quarter wavelength (of Re k) and 3 digits, reproduces the dense <f, L f> x of
    the oracle within the 1e-3 bar, at real k (measured 1.2e-4; the GPU product gives 1.3e-4
    on this mesh) and at the coating's complex k (1.5e-4)."""
    levels, e_all, e_far = _multilevel_L_product(bi, k, 8, 0.5, 0.25, 3)
    assert levels >= 3
    assert e_all < 5e-4, (e_all, e_far)


@pytest.mark.slow
def test_two_region_product_model_matches_the_dense_pmchwt(bi):
    """The far-field form planned for a two-region (PMCHWT) product, checked against the
    oracle's dense two_region matrix on a lossy sphere (eps_r = 2 - 0.5j, radius 0.5 lambda).
    Each medium has its own plan, with sampling from its Re k. Per box and medium there are
    two transverse fields:
    - U_E = eta x_J F - x_M khat x F, received as -jk R.V_E by the E-tested rows;
    - U_H = x_J F - x_M khat x F / eta, received as -jk R.(khat x V_H) by the H-tested rows.
    Near pairs come from each medium's dense L and Kbar. Measured 2.8e-4. With eta in place
    of 1/eta in U_H the error is 1.7e-2; with an untwisted H receive it is 5.7e-2."""
    import oracle
    eps = 2.0 - 0.5j
    v, t = inputs.icosphere(6, 0.5)
    k1 = K0 * np.sqrt(eps)
    k1 = k1 if k1.real > 0 else -k1
    eta1 = np.sqrt(1.0 / eps)
    eta1 = eta1 if eta1.real > 0 else -eta1
    rng = np.random.default_rng(inputs.SEED_BASE + 81)
    N = len(oracle.rwg(v, t)["edges"])
    xJ = rng.normal(size=N) + 1j * rng.normal(size=N)
    xM = rng.normal(size=N) + 1j * rng.normal(size=N)
    yE = np.zeros(N, complex)
    yH = np.zeros(N, complex)
    for k, eta in ((K0, 1.0), (k1, eta1)):
        m = _MultilevelModel(bi, v, t, k, 0.25, 3)
        L, _, K, _ = oracle.operators(v, t, k, 0)
        yE += m.receive(m.propagate(m.outgoing(eta * xJ, -xM)))
        yE += m.near(eta * L, xJ) - m.near(K, xM)
        yH += m.receive(m.propagate(m.outgoing(xJ, -xM / eta)), twisted=True)
        yH += m.near(K, xJ) + m.near(L / eta, xM)
    ref = oracle.two_region(v, t, K0, eps) @ np.concatenate([xJ, xM])
    err = np.linalg.norm(np.concatenate([yE, yH]) - ref) / np.linalg.norm(ref)
    assert err < 1e-3, err


@pytest.mark.slow
def test_c_block_far_field_model_between_two_bodies(bi):
    """The far field of the C block (Eqs. 43-46) through the whole multilevel chain, between
    two spheres of radius 0.25 lambda 2 lambda apart: 5 levels, one child per parent, and every
    coupling between the bodies carried by translations on the two coarsest levels.  The numpy
    model runs on the plan's tables with the four Galerkin operators factorised as
      <f, L f>      -> R  . F          <f, Kbar f>      -> R  . (khat x F)
      <f, n x L f>  -> -RX . F         <f, n x Kbar f>  -> -RX . (khat x F)
    (one receive constant, RX the receive pattern of n x f), then
      y_J = -P x_J - Q x_M,  y_M = Q x_J - P x_M,  P = (L + n x Kbar)/2,  Q = (n x L - Kbar)/2.
    Against the oracle's dense cross block (currents on the second body, rows of the first)
    the error is the 3-digit truncation of the closest far interactions: measured 1.08e-3,
    3.9e-4 and 2.3e-4 on three seeded columns (the GPU product gives the same 1.08e-3 on the
    first).  With the sign of the n x terms flipped the error is O(1)."""
    import oracle
    v1, t1 = inputs.icosphere(4, 0.25, center=(-1.0, 0.0, 0.0))
    v2, t2 = inputs.icosphere(4, 0.25, center=(1.0, 0.0, 0.0))
    v = np.concatenate([v1, v2])
    t = np.concatenate([t1, t2 + len(v1)]).astype(np.int32)
    m = _MultilevelModel(bi, v, t, K0, 0.25, 3)
    assert m.info["levels"] == 5 and m.info["interactions"][m.lf] == 0
    nth, nph, kh, th, ph, _ = m.grids[m.lf]
    RX = np.zeros_like(m.R)
    for b in range(m.nb):
        rows = m.rows(b)
        P = _rwg_pattern_subset(v, t, m.rwg, rows, -K0, kh, m.cen[m.lf][b], twisted=True)
        for i, comp in enumerate((th, ph)):
            RX[i, rows] = np.einsum("ndc,dc->nd", P, comp)

    def recv(Rm, V):
        y = np.zeros(m.N, complex)
        for b in range(m.nb):
            r = m.rows(b)
            y[r] = -1j * m.k * (Rm[0, r] @ V[b, 0] + Rm[1, r] @ V[b, 1])
        return y

    N = m.N
    zero = np.zeros(N)
    second = np.nonzero(m.rwg["edges"][:, 0] >= len(v1))[0]
    cols = np.concatenate([second, second + N])
    rows_first = np.setdiff1d(np.arange(2 * N), cols)
    Z = oracle.fill(v, t, K0, 0)
    x = inputs.complex_gaussian(2 * N, 3, seed=inputs.SEED_BASE + 71)
    errs = {+1: [], -1: []}
    for r in range(3):
        xs = np.zeros(2 * N, complex)
        xs[cols] = x[r, cols]
        ref = (Z @ xs)[rows_first]
        xJ, xM = xs[:N], xs[N:]
        VJ, VJk = m.propagate(m.outgoing(xJ, zero)), m.propagate(m.outgoing(zero, xJ))
        VM, VMk = m.propagate(m.outgoing(xM, zero)), m.propagate(m.outgoing(zero, xM))
        for sgn in (+1, -1):
            # L, Kbar, n x L, n x Kbar applied to x_J and to x_M
            L_J, K_J, nL_J, nK_J = recv(m.R, VJ), recv(m.R, VJk), -sgn * recv(RX, VJ), -sgn * recv(RX, VJk)
            L_M, K_M, nL_M, nK_M = recv(m.R, VM), recv(m.R, VMk), -sgn * recv(RX, VM), -sgn * recv(RX, VMk)
            P_J, P_M = 0.5 * (L_J + nK_J), 0.5 * (L_M + nK_M)
            Q_J, Q_M = 0.5 * (nL_J - K_J), 0.5 * (nL_M - K_M)
            y = np.concatenate([-P_J - Q_M, Q_J - P_M])[rows_first]
            errs[sgn].append(float(np.linalg.norm(y - ref) / np.linalg.norm(ref)))
    assert max(errs[+1]) < 2e-3 and min(errs[+1]) < 1e-3, errs
    assert min(errs[-1]) > 0.1, errs
