"""Full-size parity at h = 2^-11 (2049 x 2049 nodes, 8.4M unknowns), the size
the benchmark runs: GPU solutions against the FP64 oracle's, read from
tests/golden/oracle_L11.json (written by oracle/make_golden.py, oracle only).

* FP64 path: the iterates are the oracle's up to rounding, so it needs exactly
  the oracle's number of cycles to reach a relative residual of 1e-10 and its
  solution agrees with the oracle's at the sampled nodes to 1e-9.
* FP32 cycles in FP64 refinement: a different iteration towards the same
  discrete solution; both solutions are within 1e-8 of each other.
"""
import json
import os

import numpy as np
import pytest

from paper_1502_03917_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_L11.json")


@pytest.fixture(scope="module")
def golden():
    return json.load(open(GOLDEN))


def runs(g, smoother):
    return {r["alpha"]: r for r in g["runs"] if r["smoother"] == smoother}


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("alpha", [1.0, 1e-4, 1e-8])
def test_lsgs_solution_L11(golden, alpha, precision):
    import paper_1502_03917_gb300.aaomg as mg

    L = golden["level"]
    ref = runs(golden, "lsgs")[alpha]
    idx = np.array(golden["sample_nodes"])
    yD = torch.tensor(inputs.yd_sine_noise(L, 1), dtype=torch.float64, device="cuda")
    with mg.Solver(L, alpha, smoother="lsgs", precision=precision, max_iter=60) as s:
        f = s.rhs_from_yd(yD)
        x = torch.zeros_like(f)
        it, rr, _ = s.solve(f, x, tol=1e-10)
        xh = x.cpu().numpy()
    N = s.N
    y, lam = xh[idx], xh[N + idx]
    yo, lo = np.array(ref["y"]), np.array(ref["lambda"])
    ey = np.abs(y - yo).max() / np.abs(yo).max()
    el = np.abs(lam - lo).max() / np.abs(lo).max()
    if precision == "fp64":
        assert it == ref["iterations_to_1e-10"], (it, ref["iterations_to_1e-10"])
        assert max(ey, el) <= 1e-9, (ey, el)
    else:
        assert max(ey, el) <= 1e-8, (ey, el)


@pytest.mark.parametrize("alpha", [1e-2, 1e-6])
def test_iteration_counts_L11(golden, alpha):
    """GPU FP64 LSGS and NE need the oracle's number of W-cycles to 1e-8."""
    import paper_1502_03917_gb300.aaomg as mg

    L = golden["level"]
    yD = torch.tensor(inputs.yd_sine_noise(L, 1), dtype=torch.float64, device="cuda")
    for smoother in ("lsgs", "ne"):
        hist = runs(golden, smoother)[alpha]["history"]
        it_o = next(i for i, v in enumerate(hist) if v <= 1e-8)
        with mg.Solver(L, alpha, smoother=smoother, max_iter=80) as s:
            f = s.rhs_from_yd(yD)
            x = torch.zeros_like(f)
            it, rr, _ = s.solve(f, x, tol=1e-8)
        assert it == it_o, (smoother, it, it_o)
