"""The coupling blocks of Eqs. 40a/b, 47, 48 assembled on the GPU against the oracle's
quadrature, and the reduced operator of Eq. 52 built from them."""
import numpy as np
import pytest

import oracle
from oracle import coupling
from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, ellipsoid, icosphere

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

K0 = 2 * np.pi


@pytest.fixture(scope="module")
def bi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_04892_gb300 import bi as mod
    mod.load()
    return mod


def _csr(ptr, col, val, shape):
    return sp.csr_matrix((val.cpu().numpy(), col.cpu().numpy(), ptr.cpu().numpy()), shape=shape)


@pytest.mark.parametrize("conforming", [False, True])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 3e-7)])
@pytest.mark.parametrize("mesh", ["sphere", "ellipsoid"])
def test_coupling_blocks_match_oracle(bi, conforming, precision, tol, mesh):
    v, t = icosphere(5, 0.5) if mesh == "sphere" else ellipsoid(5, (1.0, 0.7, 0.45))
    op = bi.Operator(v, t, K0, precision=precision, op_mode=0, max_rhs=1)
    nL, lx, xl = op.coupling_blocks(conforming=conforming)
    N = op.n_unknowns // 2
    assert nL == (N if conforming else 3 * len(t))
    # every row holds the edge functions of both triangles (face layout: 6, conforming: 5
    # distinct edges); every Lambda row the J and M columns of the RWG functions it touches
    per_row = 5 if conforming else 6
    assert xl[1].numel() == 2 * N * per_row
    assert lx[1].numel() == nL * (10 if conforming else 6)
    Dxl = _csr(*xl, (op.n_unknowns, nL))
    Dlx = _csr(*lx, (nL, op.n_unknowns))
    for A in (Dxl, Dlx):
        assert A.has_sorted_indices
        assert np.all(np.abs(A.data.imag) == 0)
    Rxl, Rlx = coupling.coupling_matrices(v, t, conforming=conforming)
    sc = np.abs(Rxl).max()
    assert np.abs(Dxl.toarray() - Rxl).max() < tol * sc
    assert np.abs(Dlx.toarray() - Rlx).max() < 2 * tol * sc
    op.close()


def test_eq52_operator_with_assembled_blocks(bi):
    """Eq. 52 with the GPU-assembled D blocks (face layout) and a diagonal Q applied by the
    caller: matches C - D^{X Lambda} Q^{-1} D^{Lambda X} from the oracle's dense C and its
    quadrature of the blocks; the solve of the reduced system matches a dense solve."""
    v, t = icosphere(6, 0.5)
    op = bi.Operator(v, t, K0, precision="fp64", op_mode=0, max_rhs=2)
    nL, lx, xl = op.coupling_blocks(conforming=False)
    rng = np.random.default_rng(SEED_BASE + 61)
    q = 0.02 * (1.0 + 0.5j + 0.2 * rng.standard_normal(nL))
    qt = torch.from_numpy(q).cuda()

    def qsolve(inp, out, stream):
        out.copy_(inp / qt)

    op.set_coupling(nL, lx, xl, qsolve)
    Z = oracle.fill(v, t, K0, 0)
    Rxl, Rlx = coupling.coupling_matrices(v, t, conforming=False)
    Zr = Z - Rxl @ np.diag(1.0 / q) @ Rlx
    x = complex_gaussian(op.n_unknowns, 2, seed=SEED_BASE + 62)
    y = op.matvec_coupled(torch.from_numpy(x).cuda()).cpu().numpy()
    for r in range(2):
        assert np.linalg.norm(y[r] - Zr @ x[r]) < 1e-3 * np.linalg.norm(Zr @ x[r])
        assert np.linalg.norm(y[r] - Z @ x[r]) > 1e-2 * np.linalg.norm(Z @ x[r])
    b = op.rhs_planewave([0, 0, 1.0], [1.0, 0, 0])
    xs, its, relres = op.solve(b, tol=1e-6)
    assert relres[0] <= 1e-6 * 1.001
    xd = np.linalg.solve(Zr, b.cpu().numpy()[0])
    assert np.linalg.norm(xs.cpu().numpy()[0] - xd) < 2e-3 * np.linalg.norm(xd)
    op.close()


def test_coupling_blocks_reject_other_modes(bi):
    v, t = icosphere(4, 0.5)
    op = bi.Operator(v, t, K0, precision="fp64", op_mode=1, max_rhs=1)
    with pytest.raises(bi.BIError):
        op.coupling_blocks()
    op.close()
