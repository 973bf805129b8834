"""bi_farfield_noalloc: the far field for callers that cannot allocate device memory while
they run (fixed-budget real-time loops, hosts whose allocator belongs to another runtime).
It must return what bi_farfield returns, call after call, while its partial sums live in the
library's fixed device array.

Collected last on purpose (file name), so a stop-at-first-failure run has already run the
rest of the suite; it also passes when run alone in a fresh process."""
import ctypes

import numpy as np
import pytest

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


def _call(L, name, op, x, dirs, F):
    return getattr(L, name)(op.h, ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.c_void_p(dirs.data_ptr()),
                            dirs.shape[0], ctypes.c_void_p(F.data_ptr()))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_far_field_matches_bi_farfield_twice(bi, precision):
    L = bi.load()
    v, t = icosphere(8, 0.5)
    op = bi.Operator(v, t, K0, precision=precision, op_mode=0, max_rhs=2)
    th = np.deg2rad(np.arange(0, 181, 2))
    dirs = torch.tensor(np.stack([np.sin(th), 0 * th, np.cos(th)], 1), dtype=torch.float64, device="cuda")
    for call in range(2):
        x = torch.from_numpy(complex_gaussian(op.n_unknowns, 2, seed=SEED_BASE + 40 + call).astype(op.np_cdtype)).cuda()
        F_ref = torch.empty((2, dirs.shape[0], 3), dtype=torch.complex128, device="cuda")
        F_new = torch.full_like(F_ref, float("nan"))
        assert _call(L, "bi_farfield", op, x, dirs, F_ref) == bi.BI_OK
        assert _call(L, "bi_farfield_noalloc", op, x, dirs, F_new) == bi.BI_OK
        torch.cuda.synchronize()
        a, b = F_new.cpu().numpy(), F_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12
    op.close()


def test_noalloc_rejects_requests_beyond_the_fixed_array(bi):
    L = bi.load()
    v, t = icosphere(8, 0.5)
    op = bi.Operator(v, t, K0, precision="fp32", op_mode=1, max_rhs=1)
    x = torch.zeros((1, op.n_unknowns), dtype=torch.complex64, device="cuda")
    ndir = 20000   # 8 chunks x 20000 directions x 96 B > 8 MiB
    dirs = torch.zeros((ndir, 3), dtype=torch.float64, device="cuda")
    dirs[:, 2] = 1.0
    F = torch.zeros((1, ndir, 3), dtype=torch.complex128, device="cuda")
    assert _call(L, "bi_farfield_noalloc", op, x, dirs, F) == bi.BI_ERR_ARG
    assert b"fixed" in L.bi_last_error(op.h)
    op.close()
