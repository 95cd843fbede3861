"""Write tests/golden/oracle_L{L}.json: full-size reference values computed by
the oracle alone (nothing here touches the CUDA path).

Workloads (W-cycle with 2+2 smoothing steps down to h = 1/2):

* L = 11 (default), the scaling workload at its largest size: h = 2^-11
  (2049 x 2049 nodes, 8.4M unknowns), y_D = sin(2 pi x) sin(2 pi y) +
  0.1 N(0,1) (seed 1), alpha in {1, 1e-2, 1e-4, 1e-6, 1e-8}, LSGS, NE, sLSGS
  and CGS.
* L = 12, the largest single instance: h = 2^-12 (4097 x 4097 nodes, 33.6M
  unknowns), y_D = +1 on [0.25, 0.75]^2, -1 elsewhere, plus U(-0.05, 0.05)
  noise (seed 5), alpha = 1e-6, LSGS.

Each solve runs to a relative residual of 1e-10 (at these sizes FP64 rounding
stalls the residual a little below that); the file keeps the residual history
(so the iteration count to any tolerance above 1e-10 can be read off), and the
solution at 256 seeded node indices.

Usage: python oracle/make_golden.py [L [smoother ...]]   (minutes per solve on one core)
With smoothers named, only their runs are computed and merged into an existing
file (sLSGS with 1+1 smoothing steps, the paper's choice; the others 2+2).
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

WORKLOADS = {
    11: {"workload": "y_D = sin(2 pi x) sin(2 pi y) + 0.1 N(0,1), seed 1; W(2,2) to h=1/2",
         "yd": lambda L: inputs.yd_sine_noise(L, 1),
         "alphas": [1.0, 1e-2, 1e-4, 1e-6, 1e-8], "smoothers": ("lsgs", "ne", "slsgs", "cgs")},
    12: {"workload": "y_D = +1 on [0.25,0.75]^2, -1 elsewhere, + U(-0.05,0.05), seed 5; W(2,2) to h=1/2",
         "yd": lambda L: inputs.yd_piecewise(L, 5),
         "alphas": [1e-6], "smoothers": ("lsgs",)},
}


def main():
    L = int(sys.argv[1]) if len(sys.argv) > 1 else 11
    w = WORKLOADS[L]
    out = os.path.join(ROOT, "tests", "golden", f"oracle_L{L}.json")
    yD = w["yd"](L)
    nn = ((1 << L) + 1) ** 2
    sample = np.sort(np.random.default_rng(12345).choice(nn, size=256, replace=False))
    smoothers = tuple(sys.argv[2:]) or w["smoothers"]
    res = {"level": L, "workload": w["workload"], "sample_nodes": sample.tolist(), "runs": []}
    if sys.argv[2:] and os.path.exists(out):
        res = json.load(open(out))
        assert res["sample_nodes"] == sample.tolist()
        res["runs"] = [r for r in res["runs"] if r["smoother"] not in smoothers]
    for smoother in smoothers:
        nu = 1 if smoother == "slsgs" else 2
        for a in w["alphas"]:
            t0 = time.time()
            o = oracle.Oracle(L, a, smoother=smoother, nu_pre=nu, nu_post=nu)
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
