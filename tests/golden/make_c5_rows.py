"""Write tests/golden/c5_rows.json: rows of the dense FP64 C block (Eqs. 43-46) of the
large-scatterer workload (geodesic sphere nu = 241, radius 20 wavelengths, 1,161,620
triangles, 3,484,860 unknowns, k = 2 pi) times eight seeded complex-Gaussian columns.

Only the CPU oracle computes the stored values; the GPU tests compare their sampled rows
with them.  The columns x are regenerated from their seed by the tests, which check the
stored fingerprint of x first (sum of x over a fixed index set) so that a different random
stream is reported instead of compared.

  python tests/golden/make_c5_rows.py      (about half an hour on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, sample_rows, workload  # noqa: E402

NAME = "sphere_r20_nu241"
NRHS = 8
NROWS = 256
ROW_SEED = SEED_BASE + 41
K0 = 2 * np.pi
OUT = os.path.join(HERE, "c5_rows.json")


def fingerprint(x):
    idx = np.arange(0, x.shape[1], 9973)
    return [[float(v.real), float(v.imag)] for v in x[:, idx].sum(1)]


def main():
    v, t, meta = workload(NAME)
    nun = oracle.num_unknowns(v, t, 0)
    x = complex_gaussian(nun, NRHS, seed=meta["seed"])
    rows = sample_rows(nun, NROWS, seed=ROW_SEED)
    y = np.zeros((NRHS, NROWS), np.complex128)
    t0 = time.time()
    for i in range(0, NROWS, 16):
        Z = oracle.rows(v, t, K0, 0, rows[i:i + 16])
        y[:, i:i + 16] = (Z @ x.T).T
        print("%d/%d rows, %.0f s" % (i + 16, NROWS, time.time() - t0), flush=True)
    out = {"workload": NAME, "k0": K0, "op_mode": 0, "nrhs": NRHS, "x_seed": int(meta["seed"]),
           "row_seed": ROW_SEED, "rows": [int(r) for r in rows], "x_fingerprint": fingerprint(x),
           "y": [[[float(c.real), float(c.imag)] for c in yr] for yr in y],
           "oracle_threads": oracle.threads(), "seconds": time.time() - t0}
    with open(OUT, "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
