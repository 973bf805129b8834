"""Full-size parity of the large-scatterer configuration: a sphere of radius 20 wavelengths
(1,161,620 triangles, 1,742,430 RWG, 3,484,860 unknowns in the C block of Eq. 42), 9-level
product in FP32 with 8 right-hand sides in one call, against rows of the dense FP64 operator
that the oracle computes one by one."""
import numpy as np
import pytest

import oracle
from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, sample_rows, workload

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

K0 = 2 * np.pi


@pytest.fixture(scope="module")
def bi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_04892_gb300 import bi as mod
    mod.load()
    return mod


def test_large_sphere_sampled_rows_eight_rhs(bi):
    v, t, meta = workload("sphere_r20_nu241")
    R = 8
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=R)
    info = op.info()
    assert info["levels"] == 9
    nun = op.n_unknowns
    x = complex_gaussian(nun, R, seed=meta["seed"]).astype(np.complex64)
    y = op.matvec(torch.from_numpy(x).cuda())
    op.status()
    y = y.cpu().numpy()
    op.close()
    rows = sample_rows(nun, 8, seed=SEED_BASE + 41)
    Z = oracle.rows(v, t, K0, 0, rows)
    for r in range(R):
        ref = Z @ x[r].astype(np.complex128)
        err = float(np.linalg.norm(y[r][rows] - ref) / np.linalg.norm(ref))
        assert err < 1e-3, (r, err)
