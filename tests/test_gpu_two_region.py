"""The two-region (PMCHWT) operator of a homogeneous body on the GPU (op_mode 2): the surface-only
form with which the paper's penetrable scatterers (Sec. III.A) are checked against the Mie
series without the HDG interior.  Each medium -- free space at k0 and the body at
k1 = k0 sqrt(eps_r) -- has its own octree, near field and multilevel product; the exterior
currents (J, M) are the unknowns.  Checked against the oracle's dense two_region matrix, and a
GPU GMRES solve of a dielectric sphere against the Mie series."""
import numpy as np
import pytest

import oracle
from oracle import mie
from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, icosphere

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("eps", [2 - 0.5j, 4.0], ids=["lossy", "lossless"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_two_region_product_matches_dense_oracle(bi, eps, precision, nrhs):
    """Sphere of radius 0.5 wavelength (1280 triangles, 3840 unknowns; edges of about a seventh
    of the body's wavelength at eps_r = 4): the GPU product of both media against the oracle's
    dense PMCHWT matrix.  Measured 1e-4 (lossy) and 3.4e-4 (eps_r = 4).  A mesh of 720
    triangles (edges of 0.18 of the body's wavelength) gives 8.8e-4 in FP64 and 1.2e-3 in FP32
    at eps_r = 4: the body's wavelength is then barely resolved for its quarter-wavelength
    boxes."""
    v, t = icosphere(8, 0.5)
    op = bi.Operator(v, t, K0, digits=3, precision=precision, op_mode=2, eps_r=eps, max_rhs=nrhs)
    assert op.n_unknowns == 2 * len(oracle.rwg(v, t)["edges"])
    x = complex_gaussian(op.n_unknowns, nrhs, seed=SEED_BASE + 74).astype(op.np_cdtype)
    y = op.matvec(torch.from_numpy(x).cuda())
    op.status()
    y = y.cpu().numpy().astype(np.complex128)
    op.close()
    Z = oracle.two_region(v, t, K0, eps)
    ref = x.astype(np.complex128) @ Z.T
    for r in range(nrhs):
        assert rel(y[r], ref[r]) < 1e-3, (r, rel(y[r], ref[r]))


def test_two_region_rhs_matches_oracle(bi):
    """[-<f, E_inc>; -<f, H_inc>] of two plane waves against the oracle."""
    v, t = icosphere(6, 0.5)
    kh, ph = np.array([[0, 0, 1.0], [0.6, 0, 0.8]]), np.array([[1.0, 0, 0], [0, 1.0, 0]])
    op = bi.Operator(v, t, K0, precision="fp64", op_mode=2, eps_r=4.0, max_rhs=2)
    b = op.rhs_planewave(kh, ph).cpu().numpy()
    op.close()
    ref = oracle.two_region_rhs(v, t, K0, kh, ph)
    assert rel(b, ref) < 1e-6


@pytest.mark.parametrize("nu,eps", [(7, 2 - 0.5j), (6, 4.0)])
def test_two_region_solve_rcs_vs_mie(bi, nu, eps):
    """Homogeneous sphere of radius 0.4 wavelength, plane wave along +z polarised along x: GMRES
    on the GPU (FP64 products), far field on the GPU, RCS within 0.5 dB of the Mie series where
    sigma >= max - 20 dB, and the error of Eq. 5-25 below 5%."""
    v, t = icosphere(nu, 0.4)
    op = bi.Operator(v, t, K0, digits=3, precision="fp64", op_mode=2, eps_r=eps, max_rhs=1)
    b = op.rhs_planewave([0, 0, 1.0], [1.0, 0, 0])
    x, its, relres = op.solve(b, tol=1e-5)
    assert relres[0] <= 1e-5 * 1.001
    th = np.deg2rad(np.arange(0, 181))
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    s = op.rcs(x, dirs)[0]
    op.close()
    sm = mie.rcs_dielectric(K0, 0.4, eps, th)
    mask = 10 * np.log10(sm) >= 10 * np.log10(sm.max()) - 20
    assert np.abs(10 * np.log10(s / sm))[mask].max() < 0.5
    assert oracle.rcs_error(s, sm) < 0.05


def test_two_region_rejects_unsupported_settings(bi):
    v, t = icosphere(4, 0.5)
    with pytest.raises(bi.BIError):
        bi.Operator(v, t, K0, op_mode=2, eps_r=4.0, precond=1)
    with pytest.raises(bi.BIError):
        bi.Operator(v, t, K0, op_mode=2, eps_r=4.0 + 1.0j)      # gain medium


def _coated_mesh(nu1, nu2):
    """Coat's outer surface (radius 0.4 wavelength) then the PEC core (radius 0.3), the core's
    vertices numbered after the outer surface's."""
    v1, t1 = icosphere(nu1, 0.4)
    v2, t2 = icosphere(nu2, 0.3)
    v = np.concatenate([v1, v2])
    t = np.concatenate([t1, t2 + len(v1)]).astype(np.int32)
    return (v1, t1), (v2, t2), v, t, len(t2)


@pytest.mark.parametrize("eps,precision", [(2 - 0.5j, "fp64"), (2 - 0.5j, "fp32"), (4.0, "fp32"), (8.0, "fp64")])
def test_coated_pec_product_matches_dense_oracle(bi, eps, precision):
    """The coated sphere of Sec. III.A (PEC radius 0.3 wavelength under a 0.1 wavelength coat):
    the GPU product of the outer medium on the coat's surface and of the coat on both surfaces,
    with the unknown and row maps of the coated system, against the oracle's dense matrix.  At
    the paper's eps_r = 8 the coat's wavelength spans about five edges of this mesh and FP32
    gives 1.1e-3 (FP64 stays inside 1e-3), so eps_r = 8 is checked in FP64."""
    (v1, t1), (v2, t2), v, t, nc = _coated_mesh(7, 6)
    Z, _, n1, n2 = oracle.coated_pec(v1, t1, v2, t2, K0, eps)
    op = bi.Operator(v, t, K0, digits=3, precision=precision, op_mode=4, eps_r=eps, core_tris=nc, max_rhs=2)
    assert op.n_unknowns == 2 * n1 + n2
    x = complex_gaussian(op.n_unknowns, 2, seed=SEED_BASE + 75).astype(op.np_cdtype)
    y = op.matvec(torch.from_numpy(x).cuda())
    op.status()
    y = y.cpu().numpy().astype(np.complex128)
    op.close()
    ref = x.astype(np.complex128) @ Z.T
    for r in range(2):
        assert rel(y[r], ref[r]) < 1e-3, (r, rel(y[r], ref[r]))


@pytest.mark.parametrize("eps", [2 - 0.5j, 8.0], ids=["lossy", "eps8"])
def test_coated_pec_solve_rcs_vs_mie(bi, eps):
    """The coated sphere solved on the GPU (GMRES, FP64 products) with a plane wave along +z
    polarised along x: RCS within 0.5 dB of the coated-sphere Mie series where sigma >=
    max - 20 dB, and the error of Eq. 5-25 below 5% (the paper's metric, Sec. III.A).  The
    core's row is of EFIE type, so GMRES converges slowly: restarts of 400 and a 1e-4 target
    (with restarts of 100 the eps_r = 8 solve stagnated near 2e-2)."""
    (v1, t1), (v2, t2), v, t, nc = _coated_mesh(7, 6)
    op = bi.Operator(v, t, K0, digits=3, precision="fp64", op_mode=4, eps_r=eps, core_tris=nc, max_rhs=1,
                     gmres_restart=400, gmres_maxit=4000)
    b = op.rhs_planewave([0, 0, 1.0], [1.0, 0, 0])
    _, rhs, _, _ = oracle.coated_pec(v1, t1, v2, t2, K0, eps)
    assert rel(b.cpu().numpy()[0], rhs([0, 0, 1.0], [1.0, 0, 0])[0]) < 1e-6
    x, its, relres = op.solve(b, tol=1e-4)
    assert relres[0] <= 1e-4 * 1.001
    th = np.deg2rad(np.arange(0, 181))
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    s = op.rcs(x, dirs)[0]
    op.close()
    sm = mie.rcs_coated_pec(K0, 0.3, 0.4, eps, th)
    mask = 10 * np.log10(sm) >= 10 * np.log10(sm.max()) - 20
    assert np.abs(10 * np.log10(s / sm))[mask].max() < 0.5
    assert oracle.rcs_error(s, sm) < 0.05
