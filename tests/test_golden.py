"""Provenance of the stored expected values under tests/golden/: they are reproduced here from
the CPU oracle alone, so none of them can have come from the CUDA path."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, sample_rows, workload

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.slow
def test_stored_large_sphere_rows_are_the_oracles():
    """tests/golden/c5_rows.json (rows of the dense FP64 C block of the 3,484,860-unknown
    sphere times eight seeded columns): the stored row indices and column fingerprint follow
    from their seeds, and two of the stored rows, recomputed by the oracle, agree to rounding."""
    g = json.load(open(os.path.join(HERE, "golden", "c5_rows.json")))
    v, t, meta = workload(g["workload"])
    nun = oracle.num_unknowns(v, t, g["op_mode"])
    assert nun == 3484860 and g["nrhs"] == 8 and g["x_seed"] == meta["seed"]
    rows = np.array(g["rows"])
    assert np.array_equal(rows, sample_rows(nun, len(rows), seed=g["row_seed"]))
    x = complex_gaussian(nun, g["nrhs"], seed=g["x_seed"])
    idx = np.arange(0, nun, 9973)
    fp = np.array(g["x_fingerprint"])
    assert np.allclose(x[:, idx].sum(1), fp[:, 0] + 1j * fp[:, 1], rtol=0, atol=1e-9)
    y = np.array(g["y"])
    y = y[..., 0] + 1j * y[..., 1]
    pick = np.array([0, len(rows) // 2 + 1])
    Z = oracle.rows(v, t, g["k0"], g["op_mode"], rows[pick])
    got = (Z @ x.T).T
    assert np.linalg.norm(got - y[:, pick]) / np.linalg.norm(y[:, pick]) < 1e-12
