"""Write tests/golden/oracle_L11.json: full-size reference values computed by
the oracle alone (nothing here touches the CUDA path).

Workload: Poisson control on the unit square at h = 2^-11 (2049 x 2049 nodes,
8.4M unknowns), y_D = sin(2 pi x) sin(2 pi y) + 0.1 N(0,1) (seed 1), W-cycle
with 2+2 smoothing steps down to h = 1/2, for alpha in {1, 1e-2, 1e-4, 1e-6,
1e-8} and the NE and LSGS smoothers.  Each solve runs to a relative residual of
1e-10 (at this size FP64 rounding stalls the residual near 3e-11 for alpha = 1);
the file keeps the residual history (so the iteration count to any tolerance
above 1e-10 can be read off), and the solution at 256 seeded node indices.

Usage: python oracle/make_golden.py [L]   (takes tens of minutes on one core)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1502_03917_gb300 import inputs  # noqa: E402

ALPHAS = [1.0, 1e-2, 1e-4, 1e-6, 1e-8]


def main():
    L = int(sys.argv[1]) if len(sys.argv) > 1 else 11
    out = os.path.join(ROOT, "tests", "golden", f"oracle_L{L}.json")
    yD = inputs.yd_sine_noise(L, 1)
    nn = ((1 << L) + 1) ** 2
    sample = np.sort(np.random.default_rng(12345).choice(nn, size=256, replace=False))
    res = {"level": L, "workload": "y_D = sin(2 pi x) sin(2 pi y) + 0.1 N(0,1), seed 1; W(2,2) to h=1/2",
           "sample_nodes": sample.tolist(), "runs": []}
    for smoother in ("lsgs", "ne"):
        for a in ALPHAS:
            t0 = time.time()
            o = oracle.Oracle(L, a, smoother=smoother)
            f = o.rhs(yD)
            x, it, rr, hist = o.solve(f, tol=1e-10, max_iter=60)
            res["runs"].append({
                "smoother": smoother, "alpha": a, "iterations_to_1e-10": it, "relres": rr,
                "history": hist.tolist(),
                "y": x[sample].tolist(), "lambda": x[nn + sample].tolist(),
                "seconds": time.time() - t0,
            })
            o.close()
            print(smoother, a, it, rr, f"{time.time() - t0:.1f}s", flush=True)
            json.dump(res, open(out, "w"), indent=1)


if __name__ == "__main__":
    main()
