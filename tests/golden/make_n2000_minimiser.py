"""Writes n2000_minimiser.json: the FP64 oracle's minimiser of the n = 2000
sparse-Theta workload (m = 1000 samples, seed 2000, lambda = 0.1), solved to
relative KKT 1e-10, as upper-triangle triplets (i <= j, both triangles hold
the value), with its objective, log det and KKT residual, and the pairs whose
|(S - W)_ij| lies within 1e-7 of lambda (the support-border pairs, where the
support of a solution that meets the entry bar may differ).

The minimiser of eq. MLE_l1_prior is unique (Section 5), so every correct
solver reaches these entries.  Calls only oracle/ and the seeded generators.

    python tests/golden/make_n2000_minimiser.py
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

TOL = 1e-10
BORDER = 1e-7


def main():
    oracle.build()
    p = synth.config_problem(2)
    S = oracle.form_S(p.X)
    t0 = time.perf_counter()
    A, W, info, _ = oracle.solve(S, p.lam, tol=TOL)
    wall = time.perf_counter() - t0
    assert info["status"] == oracle.OK, info
    iu, ju = np.nonzero(np.triu(A))
    G = np.abs(S - W)
    bi, bj = np.nonzero(np.triu(np.abs(G - p.lam) <= BORDER))
    out = {
        "workload": "sparse-Theta n=2000 m=1000 seed 2000 lambda=0.1 (the headline workload's S)",
        "n": p.n, "m": p.m, "lambda": p.lam, "tol": TOL, "border": BORDER,
        "objective": info["objective"], "logdet": info["logdet"], "rel_kkt": info["rel_kkt"],
        "cycles": info["cycles"], "relaxations": info["relaxations"],
        "nnz": int(np.count_nonzero(A)), "oracle_seconds": round(wall, 1),
        "i": iu.tolist(), "j": ju.tolist(), "a": [float(x) for x in A[iu, ju]],
        "border_i": bi.tolist(), "border_j": bj.tolist(),
    }
    with open(os.path.join(HERE, "n2000_minimiser.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print({k: v for k, v in out.items() if not isinstance(v, list)})


if __name__ == "__main__":
    main()
