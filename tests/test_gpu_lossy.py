"""Products at a complex wavenumber (a lossy medium, the coating of Sec. III.D with
eps_r = 2 - 0.5j: k1 = k0 sqrt(eps_r)) through the C-ABI, against the oracle's dense FP64
Galerkin matrices at the same k.  Every integral and expansion of the product is continued
to complex k: the near field (FP64 with singularity extraction), the leaf patterns (all
directions stored, R_n = F_n at the antipode), the shifts, and translation operators with
spherical Hankel functions of complex argument."""
import numpy as np
import pytest

import oracle
from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, icosphere, sample_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0 = 2 * np.pi
K1 = K0 * np.sqrt(2.0 - 0.5j)      # Re k > 0, Im k < 0 (exp(j w t))


@pytest.fixture(scope="module")
def bi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_04892_gb300 import bi as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def sphere():
    return icosphere(8, 0.5)


@pytest.fixture(scope="module")
def Z_lossy(sphere):
    v, t = sphere
    return {mode: oracle.fill(v, t, K1, mode) for mode in (0, 1)}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mode", [0, 1])
def test_lossy_near_field_only_matches_dense_oracle(bi, sphere, Z_lossy, mode):
    """A leaf of one wavelength (of Re k) leaves no far field on this sphere: the product is
    the GPU's complex-k near-field integrals alone."""
    v, t = sphere
    op = bi.Operator(v, t, K1, precision="fp64", op_mode=mode, leaf_box=1.0, max_rhs=2)
    assert op.info()["leaf_level"] < 2
    x = complex_gaussian(op.n_unknowns, 2, seed=SEED_BASE + 70)
    y = op.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, x @ Z_lossy[mode].T) < 2e-5
    op.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 3, 8])
def test_lossy_multilevel_product_matches_dense_oracle(bi, sphere, Z_lossy, precision, mode, nrhs):
    """Quarter-wavelength leaves (of Re k) and 3 digits: 4 levels on the 1280-triangle sphere,
    so interpolation, translation and anterpolation all run at complex k; one, three and
    eight right-hand sides (the one-RHS and batched kernel families of the level passes)."""
    v, t = sphere
    op = bi.Operator(v, t, K1, digits=3, precision=precision, op_mode=mode, max_rhs=nrhs)
    assert op.info()["levels"] >= 4
    x = complex_gaussian(op.n_unknowns, nrhs, seed=SEED_BASE + 71).astype(op.np_cdtype)
    y = op.matvec(torch.from_numpy(x).cuda())
    op.status()
    y = y.cpu().numpy().astype(np.complex128)
    op.close()
    ref = x.astype(np.complex128) @ Z_lossy[mode].T
    for r in range(nrhs):
        assert rel(y[r], ref[r]) < 1e-3, (r, rel(y[r], ref[r]))


def test_lossy_larger_sphere_sampled_rows(bi):
    """Sphere of radius 1 wavelength (of k0; 5120 triangles, 15,360 unknowns) at k1: 5 levels,
    FP32, 4 right-hand sides, on 192 seeded rows of the oracle's dense C block."""
    v, t = icosphere(16, 1.0)
    op = bi.Operator(v, t, K1, digits=3, precision="fp32", op_mode=0, max_rhs=4)
    assert op.info()["levels"] >= 5
    x = complex_gaussian(op.n_unknowns, 4, seed=SEED_BASE + 72)
    y = op.matvec(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    op.close()
    rows = sample_rows(len(x[0]), 192, seed=SEED_BASE + 73)
    Zr = oracle.rows(v, t, K1, 0, rows)
    for r in range(4):
        assert rel(y[r][rows], Zr @ x[r]) < 1e-3


def test_lossy_handle_rejects_free_space_only_calls(bi, sphere):
    """Plane-wave right-hand sides and far fields are defined for free space only."""
    v, t = sphere
    op = bi.Operator(v, t, K1, precision="fp32", op_mode=1, max_rhs=1)
    with pytest.raises(bi.BIError) as e:
        op.rhs_planewave([0, 0, 1.0], [1.0, 0, 0])
    assert e.value.code == bi.BI_ERR_ARG
    x = torch.zeros((1, op.n_unknowns), dtype=torch.complex64, device="cuda")
    with pytest.raises(bi.BIError):
        op.farfield(x, np.array([[0, 0, 1.0]]))
    op.close()
    with pytest.raises(bi.BIError):
        bi.Operator(v, t, K0 * (1 - 2j), precision="fp32")      # |Im k| > Re k
