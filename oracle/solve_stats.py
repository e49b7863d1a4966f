"""Runs the FP64 oracle's full solve of the n = 2000 sparse-Theta workload
(m = 1000, lambda = 0.1, rel. KKT 1e-5) and stores its statistics in
solve_stats_n2000.json.  The CPU-baseline legs of the benchmark use the
relaxation count to turn a timed sample of relaxations into a per-solve time.
Calls only oracle/ (and the seeded input generators)."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_1607_00315_gb300 import synth  # noqa: E402


def main():
    p = synth.config_problem(2)
    S = oracle.form_S(p.X)
    t0 = time.perf_counter()
    _, _, info, trace = oracle.solve(S, p.lam, tol=p.tol, trace_cap=1000)
    info["wall_s"] = time.perf_counter() - t0
    info["levels"] = [int(x) for x in trace[:, 1]]
    info["workload"] = "sparse-Theta n=2000 m=1000 lambda=0.1 tol=1e-5, seed 2000"
    with open(os.path.join(HERE, "solve_stats_n2000.json"), "w") as f:
        json.dump(info, f, indent=1)
    print(json.dumps(info))


if __name__ == "__main__":
    main()
