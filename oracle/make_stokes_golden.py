"""Write tests/golden/stokes_L{L}.json: reference values of the Stokes control
problem computed by the oracle alone (nothing here touches the CUDA path).

Workloads (W-cycle, LSGS with 2+2 steps in the multicolour order, coarsest
h = 1/2; desired velocity: the divergence-free vortex of
inputs.stokes_vd_vortex with 0.1 N(0,1) noise, seed 1):

* L = 8 (h = 2^-8, 1,176,582 unknowns): alpha in {1e-2, 1e-6};
* L = 9 (h = 2^-9, 4,712,454 unknowns): alpha = 1e-4.

Each solve runs from x = 0 to a relative residual of 1e-10 in ||.||_{L^-1};
the file keeps the residual history and the solution (means of p and mu
removed) at 256 seeded indices.

Usage: python oracle/make_stokes_golden.py [L]   (about a minute per solve at L = 8,
five at L = 9, on one core)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle.stokes import StokesOracle  # noqa: E402
from paper_1502_03917_gb300 import inputs  # noqa: E402

WORKLOADS = {8: [1e-2, 1e-6], 9: [1e-4]}


def main():
    L = int(sys.argv[1]) if len(sys.argv) > 1 else 8
    out = os.path.join(ROOT, "tests", "golden", f"stokes_L{L}.json")
    vD = inputs.stokes_vd_vortex(L, 1)
    m = inputs.stokes_sizes(L)[2]
    sample = np.sort(np.random.default_rng(2024).choice(m, size=256, replace=False))
    res = {"level": L, "workload": "v_D = curl(sin(pi x)^2 sin(pi y)^2) + 0.1 N(0,1), seed 1; LSGS W(2,2) to h=1/2",
           "sample": sample.tolist(), "runs": []}
    for a in WORKLOADS[L]:
        t0 = time.time()
        o = StokesOracle(L, a, smoother="lsgs")
        f = o.rhs(vD)
        x, it, rr, hist = o.solve(f, tol=1e-10, max_iter=60)
        x = o.normalize(x)
        res["runs"].append({"alpha": a, "iterations_to_1e-10": it, "relres": rr, "history": hist.tolist(),
                            "x": x[sample].tolist(), "seconds": time.time() - t0})
        o.close()
        print(L, a, it, rr, f"{time.time() - t0:.1f}s", flush=True)
        json.dump(res, open(out, "w"), indent=1)


if __name__ == "__main__":
    main()
