"""Writes mixed_cone_c1_seed0.json: the oracle's solve of the mixed-cone QP
(n = 2000, m = 6600: 500 zero, 3000 nonneg rows, 500 SOC(5), 100 exp, 100
pow(0.3) cones; P = diag + rank 10; seed 0) at eps_feas = 1e-8.

Calls only the oracle (and the seeded input generator).  The stored x is the
primal optimum, unique because P is positive definite (diag U(0.1, 1) plus a
rank-10 PSD term); s = b - A x follows from it, and the dual z is not unique
(3300+ active rows against 2000 variables), so only its validity is checked
by the tests.  Run from the repository root:

    python tests/golden/make_mixed_cone_c1.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2412_19027_gb300 import workloads as W  # noqa: E402


def main():
    prob = W.mixed_cone(0)
    t0 = time.time()
    r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones)
    out = {
        "source": "oracle.solve (FP64, dense Bunch-Kaufman LDL^T + refinement), default settings, eps_feas 1e-8",
        "workload": "mixed_cone(seed=0): n=2000, m=6600 (500 zero, 3000 nonneg, 500 SOC5, 100 exp, 100 pow0.3)",
        "status": r.status_name, "iterations": int(r.iterations),
        "objective": float(prob.objective(r.x)), "obj_primal": float(r.obj_primal), "obj_dual": float(r.obj_dual),
        "res_primal": float(r.res_primal), "res_dual": float(r.res_dual), "gap_abs": float(r.gap_abs),
        "gap_rel": float(r.gap_rel), "seconds": time.time() - t0,
        "x": [float(v) for v in r.x],
    }
    with open(os.path.join(HERE, "mixed_cone_c1_seed0.json"), "w") as f:
        json.dump(out, f, indent=0)
    print(out["status"], out["iterations"], out["objective"], "%.1f s" % out["seconds"])


if __name__ == "__main__":
    main()
