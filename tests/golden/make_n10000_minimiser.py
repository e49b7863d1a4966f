"""Writes n10000_minimiser.json: the FP64 oracle's minimiser of the n = 10000
sparse-Theta workload (m = 5000 samples, seed 3000, lambda = 0.08; the
samples rounded to FP32, as the workload hands them to the device, then S
formed from them in FP64), solved to relative KKT 1e-9, as upper-triangle triplets (i <= j, both triangles hold
the value), with its objective, log det and KKT residual, and the pairs whose
|(S - W)_ij| lies within 1e-7 of lambda (the support-border pairs, where the
support of a solution that meets the entry bar may differ).

The minimiser of eq. MLE_l1_prior is unique (Section 5), so every correct
solver reaches these entries.  Calls only oracle/ and the seeded generators.

    python tests/golden/make_n10000_minimiser.py   (hours: the oracle is plain
    single-threaded C and each relaxation factors and inverts a 10000 x 10000 matrix)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1607_00315_gb300 import synth  # noqa: E402

TOL = 1e-9
BORDER = 1e-7


def main():
    oracle.build()
    p = synth.config_problem(3)
    S = oracle.form_S(p.X.astype(np.float32).astype(np.float64))
    t0 = time.perf_counter()
    A, W, info, _ = oracle.solve(S, p.lam, tol=TOL)
    wall = time.perf_counter() - t0
    assert info["status"] == oracle.OK, info
    iu, ju = np.nonzero(np.triu(A))
    G = np.abs(S - W)
    bi, bj = np.nonzero(np.triu(np.abs(G - p.lam) <= BORDER))
    out = {
        "workload": "sparse-Theta n=10000 m=5000 seed 3000 lambda=0.08, S in FP64 from the FP32 samples",
        "n": p.n, "m": p.m, "lambda": p.lam, "tol": TOL, "border": BORDER,
        "objective": info["objective"], "logdet": info["logdet"], "rel_kkt": info["rel_kkt"],
        "cycles": info["cycles"], "relaxations": info["relaxations"],
        "nnz": int(np.count_nonzero(A)), "oracle_seconds": round(wall, 1),
        "i": iu.tolist(), "j": ju.tolist(), "a": [float(x) for x in A[iu, ju]],
        "border_i": bi.tolist(), "border_j": bj.tolist(),
    }
    with open(os.path.join(HERE, "n10000_minimiser.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print({k: v for k, v in out.items() if not isinstance(v, list)})


if __name__ == "__main__":
    main()
