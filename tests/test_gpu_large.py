"""Full-size parity of the large-scatterer configuration: a sphere of radius 20 wavelengths
(1,161,620 triangles, 1,742,430 RWG, 3,484,860 unknowns in the C block of Eq. 42), 9-level
product in FP32 with 8 right-hand sides in one call (the benchmark's call), against 256 rows
of the dense FP64 operator times the same columns.  The oracle's rows cost minutes each on the
host at this size, so tests/golden/make_c5_rows.py (which calls only the oracle) stored them."""
import numpy as np
import pytest

from paper_2210_04892_gb300.inputs import complex_gaussian

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_c5_large_sphere_stored_oracle_rows(bi):
    """The large scatterer (geodesic sphere nu = 241, radius 20 wavelengths, 3,484,860
    unknowns, 9 levels), FP32, the benchmark's 8 columns in one product, against 256 rows of
    the dense FP64 operator times the same columns, stored by tests/golden/make_c5_rows.py
    (the oracle alone computed them)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c5_rows.json")
    g = json.load(open(path))
    from paper_2210_04892_gb300.inputs import workload
    v, t, meta = workload(g["workload"])
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=g["nrhs"])
    assert op.info()["levels"] == 9
    x = complex_gaussian(op.n_unknowns, g["nrhs"], seed=g["x_seed"])
    idx = np.arange(0, x.shape[1], 9973)
    fp = np.array(g["x_fingerprint"])
    assert np.allclose(x[:, idx].sum(1), fp[:, 0] + 1j * fp[:, 1], rtol=0, atol=1e-9), \
        "the seeded columns differ from those the stored rows were computed with"
    y = op.matvec(torch.from_numpy(x.astype(np.complex64)).cuda())
    op.status()
    y = y.cpu().numpy()
    op.close()
    ref = np.array(g["y"])
    ref = ref[..., 0] + 1j * ref[..., 1]
    rows = np.array(g["rows"])
    for r in range(g["nrhs"]):
        assert rel(y[r][rows], ref[r]) < 1e-3, (r, rel(y[r][rows], ref[r]))
