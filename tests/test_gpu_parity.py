"""GPU parity tests: the CUDA path through the C-ABI against the CPU FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, icosphere, sample_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0 = 2 * np.pi


@pytest.fixture(scope="module")
def bi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_04892_gb300 import bi as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def sphere_c1():
    v, t = icosphere(8, 0.5)
    return v, t


@pytest.fixture(scope="module")
def Z_c1(sphere_c1):
    v, t = sphere_c1
    return {0: oracle.fill(v, t, K0, 0), 1: oracle.fill(v, t, K0, 1)}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_rwg_order_matches_oracle(bi, sphere_c1):
    v, t = sphere_c1
    op = bi.Operator(v, t, K0)
    assert np.array_equal(op.edges(), oracle.rwg(v, t)["edges"])
    op.close()


def test_invalid_mesh_rejected(bi):
    v, t = icosphere(2, 0.5)
    with pytest.raises(bi.BIError) as e:
        bi.Operator(v, t[:-1], K0)
    assert e.value.code == bi.BI_ERR_MESH
    t2 = t.copy()
    t2[3] = t2[3][[0, 2, 1]]
    with pytest.raises(bi.BIError) as e:
        bi.Operator(v, t2, K0)
    assert e.value.code == bi.BI_ERR_MESH


@pytest.mark.parametrize("mode", [0, 1])
def test_near_field_only_matches_dense_oracle(bi, sphere_c1, Z_c1, mode):
    """With a 0.5-wavelength leaf the 1-wavelength sphere has no far field: the product is
    the GPU's FP64 singular/near-singular Galerkin integrals alone."""
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, precision="fp64", op_mode=mode, leaf_box=0.5, max_rhs=2)
    assert op.info()["leaf_level"] < 2
    x = complex_gaussian(op.n_unknowns, 2, seed=SEED_BASE)
    y = op.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = x @ Z_c1[mode].T
    assert rel(y, ref) < 2e-5
    op.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", [0, 1])
def test_c1_mlfma_matches_dense_oracle(bi, sphere_c1, Z_c1, precision, mode):
    """PEC sphere r = 0.5 lambda, 1280 triangles, 3-level MLFMA at 3 digits; x = seeded
    complex Gaussian plus the plane wave along -z polarised along x (Eqs. 49-50)."""
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, digits=3, precision=precision, op_mode=mode, max_rhs=2)
    assert op.info()["levels"] == 3
    x0 = complex_gaussian(op.n_unknowns, 1, seed=SEED_BASE)
    b = oracle.rhs_planewave(v, t, K0, mode, [0, 0, -1.0], [1.0, 0, 0])
    x = np.concatenate([x0, b], 0)
    xt = torch.from_numpy(x.astype(op.np_cdtype)).cuda()
    y = op.matvec(xt).cpu().numpy()
    ref = x @ Z_c1[mode].T
    for r in range(2):
        assert rel(y[r], ref[r]) < 1e-3, (r, rel(y[r], ref[r]))
    op.close()


def test_c1b_small_leaf(bi, sphere_c1, Z_c1):
    """Same sphere with a 0.125-wavelength leaf (4 levels, interpolation between levels).
    Boxes this small sit at the low-frequency limit of the diagonal translation, so the
    4-digit sampling rule is needed to stay within 1e-3."""
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, digits=4, precision="fp64", op_mode=0, leaf_box=0.125, max_rhs=1)
    assert op.info()["levels"] == 4
    x = complex_gaussian(op.n_unknowns, 1, seed=SEED_BASE)
    y = op.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, x @ Z_c1[0].T) < 1e-3
    op.close()


def test_four_level_sphere_sampled_rows(bi):
    """Sphere r = 1 lambda (5120 triangles), 4 levels at the default 0.25-lambda leaf:
    interpolation 0.25 -> 0.5 lambda and anterpolation back; 192 sampled rows."""
    v, t = icosphere(16, 1.0)
    op = bi.Operator(v, t, K0, digits=3, precision="fp64", op_mode=0, max_rhs=1)
    assert op.info()["levels"] == 4
    x = complex_gaussian(op.n_unknowns, 1, seed=SEED_BASE + 3)
    y = op.matvec(torch.from_numpy(x).cuda()).cpu().numpy()[0]
    rows = sample_rows(op.n_unknowns, 192, seed=SEED_BASE + 13)
    ref = oracle.rows(v, t, K0, 0, rows) @ x[0]
    assert rel(y[rows], ref) < 1e-3
    op.close()


def test_translation_operators_vs_series(bi, sphere_c1):
    """Leaf translation operators T(khat; X) w(khat) for all 316 far offsets against the
    series evaluated with scipy's spherical Bessel functions."""
    from scipy import special
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, precision="fp64", max_rhs=1)
    inf = op.info()
    lf = inf["leaf_level"]
    L = inf["L"][lf]
    T = op.debug_buffer(2, lf)
    xg, wg = np.polynomial.legendre.leggauss(L + 1)
    o = np.argsort(-xg)
    th, wt = np.arccos(xg[o]), wg[o]
    nph = 2 * (L + 1)
    TH, PH = np.meshgrid(th, 2 * np.pi * np.arange(nph) / nph, indexing="ij")
    kh = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    W = (wt[:, None] * np.ones(nph)[None] * 2 * np.pi / nph).ravel()
    a = inf["root_size"] / 2 ** lf
    worst = 0.0
    for oi in range(343):
        off = np.array([oi // 49 - 3, (oi // 7) % 7 - 3, oi % 7 - 3])
        if np.abs(off).max() <= 1:
            assert np.abs(T[oi]).max() == 0
            continue
        X = off * a
        Xn = np.linalg.norm(X)
        cg = kh @ (X / Xn)
        ref = np.zeros(len(kh), complex)
        for l in range(L + 1):
            hl = special.spherical_jn(l, K0 * Xn) - 1j * special.spherical_yn(l, K0 * Xn)
            ref += (-1j) ** l * (2 * l + 1) * hl * special.eval_legendre(l, cg)
        worst = max(worst, rel(T[oi], ref * W))
    assert worst < 1e-10, worst
    op.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_rhs_planewave_matches_oracle(bi, sphere_c1, mode):
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, precision="fp64", op_mode=mode, max_rhs=2)
    kh = np.array([[0, 0, -1.0], [np.sin(1.0), 0, np.cos(1.0)]])
    ph = np.array([[1.0, 0, 0], [np.cos(1.0), 0, -np.sin(1.0)]])
    b = op.rhs_planewave(kh, ph).cpu().numpy()
    ref = oracle.rhs_planewave(v, t, K0, mode, kh, ph)
    assert rel(b, ref) < 1e-6
    op.close()


def test_matvec_host_equals_device(bi, sphere_c1):
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, max_rhs=3)
    x = complex_gaussian(op.n_unknowns, 3, seed=5).astype(np.complex64)
    yd = op.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    yh = op.matvec_host(x)
    assert np.array_equal(yd, yh)
    op.close()


# FP32 solves stop at 5e-4: the true residual of the FP32 product has a rounding floor near
# 1e-4 (FP32 noise of the patterns amplified through the translations), so a 1e-4 target sits
# on the floor; 5e-4 is clear of it and still half the 3-digit bar
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 5e-4)])
def test_pec_solve_matches_dense_solution(bi, sphere_c1, Z_c1, precision, tol):
    """GMRES on the PEC combined-field equation reaches tol (true residual) and agrees with
    the dense LU solution of the oracle's matrix within the MLFMA accuracy."""
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, precision=precision, op_mode=1, max_rhs=2)
    b = op.rhs_planewave([[0, 0, 1.0], [1.0, 0, 0]], [[1.0, 0, 0], [0, 0, 1.0]])
    x, its, relres = op.solve(b, tol=tol)
    assert np.all(relres <= tol * 1.001), relres
    assert np.all(its > 0)
    bb = b.cpu().numpy().astype(np.complex128)
    for r in range(2):
        xr = np.linalg.solve(Z_c1[1], bb[r])
        assert rel(x.cpu().numpy()[r], xr) < 2e-3
    op.close()


@pytest.mark.parametrize("precision,mode,tol", [("fp64", 1, 1e-6), ("fp64", 0, 1e-6), ("fp32", 1, 5e-4),
                                                ("fp32", 0, 5e-4)])
def test_sai_preconditioned_solve(bi, sphere_c1, Z_c1, precision, mode, tol):
    """Near-field SAI right preconditioner (Sec. III.B): the preconditioned solve reaches the
    same tolerance in fewer GMRES iterations and returns the solution of the unpreconditioned
    system (dense LU of the oracle's matrix, within the MLFMA accuracy)."""
    v, t = sphere_c1
    out = {}
    for pc in (0, 1):
        op = bi.Operator(v, t, K0, precision=precision, op_mode=mode, max_rhs=2, precond=pc)
        b = op.rhs_planewave([[0, 0, 1.0], [1.0, 0, 0]], [[1.0, 0, 0], [0, 0, 1.0]])
        x, its, relres = op.solve(b, tol=tol)
        op.status()
        out[pc] = (x.cpu().numpy().astype(np.complex128), its.copy(), relres.copy(), b.cpu().numpy())
        if pc == 1:
            assert op.info()["setup_sai_ms"] > 0
        op.close()
    x1, its1, rel1, bb = out[1]
    x0, its0, rel0, _ = out[0]
    assert np.all(rel1 <= tol * 1.001), rel1
    assert np.all(its1 < its0), (its0, its1)
    for r in range(2):
        xr = np.linalg.solve(Z_c1[mode], bb[r].astype(np.complex128))
        assert rel(x1[r], xr) < 2e-3
        assert rel(x1[r], x0[r]) < 50 * tol + 1e-9


def test_sai_preconditioned_server_request(bi):
    """A served request with the SAI preconditioner gives the direct preconditioned solve."""
    v, t = icosphere(8, 0.5)
    srv = bi.Server(max_active=2)
    rid = srv.submit(v, t, K0, [0, 0, 1.0], [1.0, 0, 0], tol=1e-3, op_mode=1, precond=1)
    r = srv.wait(rid)
    srv.close()
    assert r["status"] == bi.BI_OK
    assert np.all(r["relres"] <= 1e-3 * 1.001)
    op = bi.Operator(v, t, K0, op_mode=1, max_rhs=1, precond=1)
    b = op.rhs_planewave([0, 0, 1.0], [1.0, 0, 0])
    x, its, relres = op.solve(b, tol=1e-3)
    assert rel(r["x"][0], x.cpu().numpy()[0]) < 1e-2
    op.close()


def test_coupled_operator_eq52(bi, sphere_c1, Z_c1):
    """Eq. 52 through the coupling hook (steps 2(a)-(e)): with random sparse D blocks and a
    diagonal Q applied by a caller's callback, bi_matvec_coupled equals
    (C - D^{X Lambda} Q^{-1} D^{Lambda X}) x built from the oracle's dense C, bi_solve solves the
    reduced system, and clearing the coupling restores C."""
    sp = pytest.importorskip("scipy.sparse")
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, precision="fp64", op_mode=0, max_rhs=2)
    nun, n_int = op.n_unknowns, 400
    rng = np.random.default_rng(SEED_BASE + 51)

    def rand_csr(m, n, per_row, scale):
        rows = np.repeat(np.arange(m), per_row)
        cols = rng.integers(0, n, size=m * per_row)
        vals = scale * (rng.standard_normal(m * per_row) + 1j * rng.standard_normal(m * per_row))
        A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
        A.sum_duplicates()
        A.sort_indices()
        return A

    def dev(A):
        return (torch.from_numpy(A.indptr.astype(np.int32)).cuda(), torch.from_numpy(A.indices.astype(np.int32)).cuda(),
                torch.from_numpy(A.data.astype(np.complex128)).cuda())

    # a random rank-400 coupling is hard for restarted GMRES when it rivals C; a modest one
    # (checked below to move the product well beyond the tolerance) keeps the solve short
    Dlx, Dxl = rand_csr(n_int, nun, 4, 0.01), rand_csr(nun, n_int, 2, 0.01)
    q = 2.0 + 1.0j + 0.5 * rng.standard_normal(n_int)
    qt = torch.from_numpy(q).cuda()

    def qsolve(inp, out, stream):
        out.copy_(inp / qt)

    op.set_coupling(n_int, dev(Dlx), dev(Dxl), qsolve)
    Zr = Z_c1[0] - (Dxl @ sp.diags(1.0 / q) @ Dlx).toarray()
    x = complex_gaussian(nun, 2, seed=SEED_BASE + 52)
    y = op.matvec_coupled(torch.from_numpy(x).cuda()).cpu().numpy()
    for r in range(2):
        assert rel(y[r], Zr @ x[r]) < 1e-3
        assert rel(y[r], Z_c1[0] @ x[r]) > 5e-3      # the coupling term is resolved, not lost
    b = op.rhs_planewave([[0, 0, 1.0], [1.0, 0, 0]], [[1.0, 0, 0], [0, 0, 1.0]])
    xs, its, relres = op.solve(b, tol=1e-6)
    assert np.all(relres <= 1e-6 * 1.001), (relres, its)
    bb = b.cpu().numpy()
    for r in range(2):
        assert rel(xs.cpu().numpy()[r], np.linalg.solve(Zr, bb[r])) < 2e-3
    op.set_coupling(0, None, None, None)
    with pytest.raises(bi.BIError):
        op.matvec_coupled(torch.from_numpy(x).cuda())
    y0 = op.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y0[0], Z_c1[0] @ x[0]) < 1e-3
    op.close()


def test_cblock_solve_converges(bi, sphere_c1):
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, precision="fp32", op_mode=0, max_rhs=1)
    b = op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    x, its, relres = op.solve(b, tol=5e-4)
    assert relres[0] <= 5e-4 * 1.001
    r = op.matvec(x) - b
    assert float(r.norm() / b.norm()) <= 5.005e-4
    op.close()


def test_c2_sampled_rows(bi):
    """Coated-sphere outer surface r = 2 lambda (20480 triangles, 61440 unknowns), 5 levels,
    FP32, one RHS: 256 seeded sampled rows computed one by one by the oracle."""
    v, t = icosphere(32, 2.0)
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=1)
    assert op.info()["levels"] == 5
    x = complex_gaussian(op.n_unknowns, 1, seed=SEED_BASE + 1)
    y = op.matvec(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()[0]
    rows = sample_rows(op.n_unknowns, 256, seed=SEED_BASE + 11)
    Zr = oracle.rows(v, t, K0, 0, rows)
    ref = Zr @ x[0]
    assert rel(y[rows], ref) < 1e-3
    op.close()


@pytest.mark.parametrize("nu", [4, 8])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mode,nrhs", [(0, 3), (0, 8), (0, 13), (1, 4), (1, 6), (1, 16)])
def test_row_blocked_near_matches_per_row_kernel(bi, nu, precision, mode, nrhs, monkeypatch):
    """The row-pair near kernels (lanes split RHS and columns, two rows per warp; plain loads or
    cp.async-pipelined block entries) against the per-row kernel, on a one-level mesh (near
    field only, written to the user vector) and a multilevel one: the products agree to the
    rounding of the summation order."""
    v, t = icosphere(nu, 0.5)
    x = complex_gaussian(oracle.num_unknowns(v, t, mode), nrhs, seed=SEED_BASE + 71)
    ys = []
    for flag in ("0", "1", "2"):
        monkeypatch.setenv("BI_NEAR_RB", flag)
        op = bi.Operator(v, t, K0, precision=precision, op_mode=mode, max_rhs=nrhs)
        ys.append(op.matvec(torch.from_numpy(x.astype(op.np_cdtype)).cuda()).cpu().numpy())
        op.close()
    tol = 2e-6 if precision == "fp32" else 1e-13
    for r in range(nrhs):
        assert rel(ys[1][r], ys[0][r]) < tol
        assert rel(ys[2][r], ys[0][r]) < tol


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mode,nrhs", [(0, 2), (0, 8), (1, 3), (1, 16)])
def test_translation_variants_agree(bi, precision, mode, nrhs, monkeypatch):
    """Every form of the batched translation kernel (one or two pairs of entries per thread,
    all 8 child slots or 4 per thread, and the staged FP32 form) gives the same product on a
    5-level sphere, to the rounding of the summation order.  (A forced form that does not
    apply to E falls back to the tuned one.)"""
    v, t = icosphere(32, 2.0)
    x = complex_gaussian(oracle.num_unknowns(v, t, mode), nrhs, seed=SEED_BASE + 73)
    ys = {}
    variants = tuple(str(v) for v in range(1, 10)) if precision == "fp32" else ("1", "2", "3", "4", "6", "8")
    for var in variants:
        monkeypatch.setenv("BI_TRANSLATE_VARIANT", var)
        op = bi.Operator(v, t, K0, precision=precision, op_mode=mode, max_rhs=nrhs)
        ys[var] = op.matvec(torch.from_numpy(x.astype(op.np_cdtype)).cuda()).cpu().numpy()
        op.close()
    tol = 2e-6 if precision == "fp32" else 1e-13
    for var in variants[1:]:
        for r in range(nrhs):
            assert rel(ys[var][r], ys["1"][r]) < tol, (var, r)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mode,nrhs", [(0, 3), (0, 8), (1, 16)])
@pytest.mark.parametrize("variant", ["2", "3"])
def test_two_pass_level_forms_agree(bi, precision, mode, nrhs, variant, monkeypatch):
    """The two-pass interpolation and anterpolation forms (one entry per lane, and entry pairs
    with the zero taps of the padded lists skipped), forced on every level of a 5-level sphere,
    give the tuned product to the rounding of the summation order."""
    v, t = icosphere(32, 2.0)
    x = complex_gaussian(oracle.num_unknowns(v, t, mode), nrhs, seed=SEED_BASE + 75)
    ys = []
    for var in ("", variant):
        monkeypatch.setenv("BI_INTERP_VARIANT", var or "0")
        monkeypatch.setenv("BI_ANTERP_VARIANT", var or "0")
        op = bi.Operator(v, t, K0, precision=precision, op_mode=mode, max_rhs=nrhs)
        ys.append(op.matvec(torch.from_numpy(x.astype(op.np_cdtype)).cuda()).cpu().numpy())
        op.close()
    # the forms take theta and phi in different orders (anterpolation: phi first in the
    # two-pass forms, theta first in the row-block form), so their FP32 intermediates round
    # differently; the far part amplifies operand rounding about 400 times (the precision
    # study), which puts FP32 differences at a few 1e-6
    tol = 2e-5 if precision == "fp32" else 1e-13
    for r in range(nrhs):
        assert rel(ys[1][r], ys[0][r]) < tol, r


@pytest.mark.parametrize("mode,nrhs", [(0, 1), (0, 3), (1, 5), (0, 16), (1, 20)])
def test_fused_kernels_match_two_pass_kernels(bi, mode, nrhs, monkeypatch):
    """The fused/streaming kernels and the two-pass reference kernels give the same product
    (FP64; 4 levels so the interpolation and anterpolation kernels run)."""
    v, t = icosphere(16, 1.0)
    x = None
    ys = []
    for two_pass in ("0", "1"):
        monkeypatch.setenv("BI_TWO_PASS", two_pass)
        op = bi.Operator(v, t, K0, precision="fp64", op_mode=mode, max_rhs=nrhs)
        if x is None:
            x = complex_gaussian(op.n_unknowns, nrhs, seed=SEED_BASE + 5)
        ys.append(op.matvec(torch.from_numpy(x).cuda()).cpu().numpy())
        op.close()
    assert rel(ys[0], ys[1]) < 1e-12


@pytest.mark.parametrize("mode,nrhs", [(0, 3), (1, 8), (0, 16)])
def test_row_blocked_anterpolation_matches_two_pass_kernels(bi, mode, nrhs, monkeypatch):
    """The row-blocked anterpolation (transposed theta step first, on the parent's columns; the
    kernel of coarse levels whose shifted parent field does not fit one CTA), forced on every
    level, against the two-pass reference kernels in FP64."""
    v, t = icosphere(16, 1.0)
    x = None
    ys = []
    for env in ({"BI_ANTERP_ROWS": "1"}, {"BI_TWO_PASS": "1"}):
        for k2, v2 in env.items():
            monkeypatch.setenv(k2, v2)
        op = bi.Operator(v, t, K0, precision="fp64", op_mode=mode, max_rhs=nrhs)
        if x is None:
            x = complex_gaussian(op.n_unknowns, nrhs, seed=SEED_BASE + 15)
        ys.append(op.matvec(torch.from_numpy(x).cuda()).cpu().numpy())
        op.close()
        for k2 in env:
            monkeypatch.delenv(k2)
    assert rel(ys[0], ys[1]) < 1e-12


@pytest.mark.parametrize("precision,mode,nrhs", [("fp64", 0, 1), ("fp32", 0, 1), ("fp32", 0, 4), ("fp32", 1, 3),
                                                  ("fp64", 1, 7)])
def test_bulk_leaf_kernels_match_plain_kernels(bi, precision, mode, nrhs, monkeypatch):
    """Leaf aggregation and receive through the bulk-copy pipelines agree with the plain
    per-warp kernels (same sums in a different order), and the device status stays clean."""
    v, t = icosphere(16, 1.0)
    x = None
    ys = []
    for bulk in ("1", "0"):
        monkeypatch.setenv("BI_LEAF_BULK", bulk)
        op = bi.Operator(v, t, K0, precision=precision, op_mode=mode, max_rhs=nrhs)
        if x is None:
            x = complex_gaussian(op.n_unknowns, nrhs, seed=SEED_BASE + 6).astype(op.np_cdtype)
        y = op.matvec(torch.from_numpy(x).cuda())
        y2 = op.matvec(torch.from_numpy(x).cuda())   # second product: ring barriers re-initialised
        op.status()
        ys.append(y.cpu().numpy())
        # (the interpolation kernels sum children with atomics: the order may differ)
        assert rel(y2.cpu().numpy(), ys[-1]) < (1e-10 if precision == "fp64" else 1e-5)
        op.close()
    # FP64 shows the two orders compute the same sums; FP32 differs by rounding amplified
    # through the translations, well inside the 1e-3 bar
    assert rel(ys[0], ys[1]) < (1e-12 if precision == "fp64" else 1e-4)


def test_farfield_matches_oracle(bi, sphere_c1):
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, precision="fp64", op_mode=0, max_rhs=2)
    x = complex_gaussian(op.n_unknowns, 2, seed=SEED_BASE + 7)
    th = np.deg2rad(np.arange(0, 181, 3))
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    F = op.farfield(torch.from_numpy(x).cuda(), dirs).cpu().numpy()
    for r in range(2):
        ref = oracle.farfield(v, t, K0, 0, x[r], dirs)
        assert rel(F[r], ref) < 1e-5
    op.close()


@pytest.mark.parametrize("nu,radius,tol", [(8, 0.5, 5e-4), (32, 2.0, 5e-4)])
def test_pec_sphere_solve_rcs_vs_mie(bi, nu, radius, tol):
    """PEC combined-field solve (GMRES on the GPU, FP32 MLFMA) of a plane wave along +z
    polarised along x, RCS from the GPU far field against the Mie series (Sec. III.A
    metric): within 0.5 dB where sigma >= max - 20 dB.  radius 2 lambda is the 20,480-triangle
    sphere of the coated-sphere outer surface."""
    from oracle import mie
    v, t = icosphere(nu, radius)
    op = bi.Operator(v, t, K0, precision="fp32", op_mode=1, max_rhs=1)
    b = op.rhs_planewave([0, 0, 1.0], [1.0, 0, 0])
    x, its, relres = op.solve(b, tol=tol)
    assert relres[0] <= tol * 1.001
    th = np.deg2rad(np.arange(0, 181))
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    s = op.rcs(x, dirs)[0]
    sm = mie.rcs_pec(K0, radius, th)
    mask = 10 * np.log10(sm) >= 10 * np.log10(sm.max()) - 20
    assert np.abs(10 * np.log10(s / sm))[mask].max() < 0.5
    assert oracle.rcs_error(s, sm) < 0.1
    op.close()


@pytest.mark.parametrize("mode,tol", [(1, 1e-5), (0, 1e-4)])
def test_c2_refined_solve_below_the_fp32_floor(bi, mode, tol):
    """Iterative refinement on the 61,440-unknown sphere (r = 2 lambda): FP32 GMRES corrections,
    residuals from an FP64 operator of the same surface.  The true residual, recomputed here
    by the FP64 product, meets tol below the FP32 product's rounding floor; for the PEC
    operator the RCS still matches the Mie series."""
    from oracle import mie
    v, t = icosphere(32, 2.0)
    op = bi.Operator(v, t, K0, precision="fp32", op_mode=mode, max_rhs=1)
    ref = bi.Operator(v, t, K0, precision="fp64", op_mode=mode, max_rhs=1)
    b = ref.rhs_planewave([0, 0, 1.0], [1.0, 0, 0])
    x, its, relres = op.solve_refined(ref, b, tol=tol)
    assert relres[0] <= tol * 1.001
    r = ref.matvec(x) - b
    assert float(r.norm() / b.norm()) <= tol * 1.001
    if mode == 1:
        th = np.deg2rad(np.arange(0, 181))
        dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
        s = ref.rcs(x, dirs)[0]
        sm = mie.rcs_pec(K0, 2.0, th)
        mask = 10 * np.log10(sm) >= 10 * np.log10(sm.max()) - 20
        assert np.abs(10 * np.log10(s / sm))[mask].max() < 0.5
    op.close()
    ref.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_two_pass_near_fill_matches_single_pass(bi, mode, monkeypatch):
    """The default near-field fill (separated triangle pairs in FP32, the rest in FP64) against
    the single-pass all-FP64 fill: the products agree to FP32 rounding of the separated pairs."""
    v, t = icosphere(8, 0.5)
    ys = []
    for single in ("0", "1"):
        monkeypatch.setenv("BI_NEAR_FILL_SINGLE_PASS", single)
        op = bi.Operator(v, t, K0, precision="fp64", op_mode=mode, leaf_box=0.5, max_rhs=1)
        x = complex_gaussian(op.n_unknowns, 1, seed=SEED_BASE + 9)
        ys.append(op.matvec(torch.from_numpy(x).cuda()).cpu().numpy())
        if single == "0":
            assert op.info()["near_special_entries"] > 0
        op.close()
    assert rel(ys[0], ys[1]) < 2e-5


def _monostatic(nphi, dphi_deg=2.0):
    """Plane waves of a monostatic sweep over phi at theta = 90 deg (k = -(cos, sin, 0), p = z)."""
    ph = np.deg2rad(dphi_deg * np.arange(nphi))
    kh = -np.stack([np.cos(ph), np.sin(ph), 0 * ph], 1)
    pp = np.tile([0.0, 0.0, 1.0], (nphi, 1))
    return kh, pp


def test_c3_cube_cylinder_batched_sampled_rows(bi):
    """Cube 5 lambda (graded lambda/10.7 to lambda/16) with an embedded closed cylinder: two
    components, ~93k RWG, 6 levels.  The batched monostatic sweep exactly as the benchmark
    runs it: 64 plane-wave columns (right-hand sides of Eqs. 49-50 built by the oracle) in one
    product, every column checked on 256 seeded rows of the oracle's dense matrix, and a few
    columns against one-column products."""
    from paper_2210_04892_gb300.inputs import cube_with_cylinder
    v, t = cube_with_cylinder()
    R = 64
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=R)
    inf = op.info()
    assert inf["levels"] == 6
    kh, pp = _monostatic(R)
    xb = oracle.rhs_planewave(v, t, K0, 0, kh, pp)
    b = torch.from_numpy(xb.astype(np.complex64)).cuda()
    y = op.matvec(b)
    for r in (0, 31, 63):
        yr = op.matvec(b[r:r + 1].contiguous())
        assert rel(yr.cpu().numpy(), y[r:r + 1].cpu().numpy()) < 1e-4
    op.status()
    yy = y.cpu().numpy().astype(np.complex128)
    op.close()
    rows = sample_rows(len(xb[0]), 256, seed=SEED_BASE + 12)
    Zr = oracle.rows(v, t, K0, 0, rows)
    ref = (Zr @ xb.T).T
    errs = [rel(yy[r][rows], ref[r]) for r in range(R)]
    assert max(errs) < 1e-3, (int(np.argmax(errs)), max(errs))


# ------------------------------------------------------------------ failure paths
def test_bounded_wait_gives_up_and_the_handle_recovers(bi):
    """The leaf bulk-copy kernels' waits are bounded.  With a limit of one SM cycle a normal
    product gives up on its first copies (they still land: the kernel drains them with the
    default limit before leaving), the device status reports BI_ERR_TIMEOUT once, and with the
    default limit restored the next product on the same handle is clean and correct."""
    v, t = icosphere(16, 1.0)
    op = bi.Operator(v, t, K0, precision="fp32", op_mode=0, max_rhs=1)
    x = torch.from_numpy(complex_gaussian(op.n_unknowns, 1, seed=SEED_BASE + 60).astype(np.complex64)).cuda()
    y_ref = op.matvec(x).cpu().numpy()
    op.status()
    op.set_wait_limit(1)
    op.matvec(x)
    with pytest.raises(bi.BIError) as e:
        op.status()
    assert e.value.code == bi.BI_ERR_TIMEOUT
    op.status()                                    # the status word was cleared by the report
    with pytest.raises(bi.BIError) as e:
        op.matvec_host(x.cpu(), torch.empty_like(x.cpu()))   # the host entry point checks it too
    assert e.value.code == bi.BI_ERR_TIMEOUT
    op.set_wait_limit(0)
    y = op.matvec(x).cpu().numpy()
    op.status()
    assert rel(y, y_ref) < 1e-6
    op.close()


def test_gmres_iteration_cap_returns_the_best_iterate(bi, sphere_c1):
    """A solve stopped by gmres_maxit before tol returns BI_ERR_NOT_CONVERGED with the last
    iterate and its true relative residual filled in (the error contract of bi_solve)."""
    import ctypes
    v, t = sphere_c1
    op = bi.Operator(v, t, K0, precision="fp64", op_mode=1, max_rhs=1, gmres_maxit=3)
    b = op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    x = torch.zeros_like(b)
    its = np.zeros(1, np.int32)
    res = np.zeros(1, np.float64)
    rc = bi.load().bi_solve(op.h, b.data_ptr(), x.data_ptr(), 1, ctypes.c_double(1e-8), its.ctypes.data,
                            res.ctypes.data)
    assert rc == bi.BI_ERR_NOT_CONVERGED
    assert its[0] == 3
    r = op.matvec(x) - b
    true_res = float(r.norm() / b.norm())
    assert 1e-8 < res[0] < 1.0
    assert abs(true_res - res[0]) < 1e-6 * max(1.0, res[0])
    op.close()
