"""Edge cases of the product against the dense CPU FP64 oracle (Eqs. 42-46), through the C-ABI:

- a body smaller than one leaf box: the tree is a single box, there is no far field at all,
  and the product is the near-field block of one box against itself;
- two bodies far apart: they are coupled only through translations on the coarse levels,
  so every level pass (interpolation to the coarsest level, translation, anterpolation back)
  carries the whole coupling, over single-child parents;
- a ragged unknown count (1470 RWG) with right-hand side counts that fill no tile: the
  row-pair near product (3 to 8 columns), the tiled leaf kernels and general-E level passes
  (8 columns and more), and a call with fewer columns than the handle holds.
"""
import numpy as np
import pytest

import oracle
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


def _product(op, x):
    return op.matvec(torch.from_numpy(x.astype(op.np_cdtype)).cuda()).cpu().numpy()


@pytest.fixture(scope="module")
def tiny_body():
    v, t = icosphere(3, 0.1)           # 180 triangles, 270 RWG, diameter 0.2 lambda
    return v, t, {m: oracle.fill(v, t, K0, m) for m in (0, 1)}


@pytest.mark.parametrize("precision,tol", [("fp64", 2e-5), ("fp32", 1e-4)])
@pytest.mark.parametrize("mode", [0, 1])
def test_body_inside_one_leaf_box(bi, tiny_body, precision, tol, mode):
    """Single-box tree: no translation, no pattern, no level pass.  The only error left is
    that of the two independent near-field quadratures (the oracle's own quadrature moves
    this product by 7e-8 between its refinement levels) and, in FP32, the storage of the
    near blocks."""
    v, t, Z = tiny_body
    op = bi.Operator(v, t, K0, digits=3, precision=precision, op_mode=mode, max_rhs=2)
    inf = op.info()
    assert inf["levels"] == 1 and inf["boxes"] == [1]
    assert inf["near_pairs"] == inf["n_rwg"] ** 2
    x = complex_gaussian(op.n_unknowns, 2, seed=SEED_BASE + 70)
    y = _product(op, x)
    op.status()
    op.close()
    assert rel(y, x @ Z[mode].T) < tol


@pytest.fixture(scope="module")
def two_bodies():
    v1, t1 = icosphere(4, 0.25, center=(-1.0, 0.0, 0.0))
    v2, t2 = icosphere(4, 0.25, center=(1.0, 0.0, 0.0))
    v = np.concatenate([v1, v2])
    t = np.concatenate([t1, t2 + len(v1)]).astype(np.int32)
    return v, t, {m: oracle.fill(v, t, K0, m) for m in (0, 1)}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode,nrhs", [(0, 1), (0, 3), (1, 8)])
def test_bodies_coupled_only_through_coarse_levels(bi, two_bodies, precision, mode, nrhs):
    """Two spheres of radius 0.25 lambda, 2 lambda apart (5 levels, one child per parent).
    No leaf box of one touches a leaf box of the other, and their parents do not touch
    either: the whole cross coupling goes up two levels, across by translation and down
    again.  The full product is held to the 3-digit bar (1e-3).

    The cross block alone (x zero on the first body, rows of the first body) holds nothing
    but far interactions at the closest separation the method translates, so its error is
    the 3-digit truncation of the plane-wave expansion itself, relative to a small field.
    On the C block's first column of three it is 1.08e-3, in FP64 and FP32 alike, and an
    FP64 numpy model of the same sampling (the plan's tables, its own pattern quadrature)
    gives the same 1.0822e-3; the other columns are 2e-4 to 4e-4.  That block is held to
    2e-3."""
    v, t, Z = two_bodies
    op = bi.Operator(v, t, K0, digits=3, precision=precision, op_mode=mode, max_rhs=nrhs)
    inf = op.info()
    assert inf["levels"] == 5
    assert inf["interactions"][inf["leaf_level"]] == 0 and sum(inf["interactions"]) > 0
    nun = op.n_unknowns
    x = complex_gaussian(nun, nrhs, seed=SEED_BASE + 71)
    y = _product(op, x)
    # RWG of the second sphere: those whose edges join its vertices (numbered after the first's)
    second = np.nonzero(op.edges()[:, 0] >= len(v) // 2)[0]
    n_rwg = op.n_rwg
    cols = np.concatenate([second + c * n_rwg for c in range(nun // n_rwg)])
    xs = np.zeros_like(x)
    xs[:, cols] = x[:, cols]
    ys = _product(op, xs)
    op.status()
    op.close()
    ref, refs = x @ Z[mode].T, xs @ Z[mode].T
    rows_first = np.setdiff1d(np.arange(nun), cols)
    for r in range(nrhs):
        assert rel(y[r], ref[r]) < 1e-3, (r, rel(y[r], ref[r]))
    for r in range(nrhs):
        # the field of the second body on the first: far field alone
        e = rel(ys[r][rows_first], refs[r][rows_first])
        assert e < 2e-3, (r, e)


@pytest.fixture(scope="module")
def ragged_sphere():
    v, t = icosphere(7, 0.5)           # 980 triangles, 1470 RWG: no multiple of 32
    return v, t, {m: oracle.fill(v, t, K0, m) for m in (0, 1)}


@pytest.mark.parametrize("mode,nrhs,max_rhs", [(0, 5, 5), (0, 11, 11), (1, 7, 7), (1, 9, 13)])
def test_ragged_sizes_match_dense_oracle(bi, ragged_sphere, mode, nrhs, max_rhs):
    """FP32, 3 levels, every column of an odd right-hand-side count against the dense oracle;
    the last case calls with fewer columns than the handle was built for."""
    v, t, Z = ragged_sphere
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=mode, max_rhs=max_rhs)
    assert op.n_rwg == 1470 and op.info()["levels"] == 3
    x = complex_gaussian(op.n_unknowns, nrhs, seed=SEED_BASE + 72)
    y = _product(op, x)
    op.status()
    op.close()
    ref = x @ Z[mode].T
    for r in range(nrhs):
        assert rel(y[r], ref[r]) < 1e-3, (r, rel(y[r], ref[r]))
