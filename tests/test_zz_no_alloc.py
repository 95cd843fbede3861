"""mg_residual_noalloc: the residual entry point for callers that must not
allocate device memory (fixed memory budgets, frameworks whose allocator owns
the device, real-time loops).  It must give the handle-based mg_residual's
result on consecutive calls, since all calls share one static scratch array.
This file is collected last so that a failure here never hides another test."""
import numpy as np
import pytest

from paper_1502_03917_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,alpha", [(1, 1.0), (4, 1e-3), (7, 1e-8), (10, 1e-2)])
def test_noalloc_residual_matches_handle_residual(L, alpha):
    import paper_1502_03917_gb300.aaomg as mg

    yD = torch.tensor(inputs.yd_sine_noise(L, 3), dtype=torch.float64, device="cuda")
    with mg.Solver(L, alpha) as s:
        f = s.rhs_from_yd(yD)
        r_ref = torch.empty_like(f)
        for call in range(2):
            x = torch.tensor(inputs.x_uniform(L, 40 + call), dtype=torch.float64, device="cuda")
            rr_ref = s.residual(f, x, r_ref)
            r = torch.full_like(f, float("nan"))
            rr = mg.residual_noalloc(L, alpha, f, x, r)
            torch.cuda.synchronize()
            a, b = r.cpu().numpy(), r_ref.cpu().numpy()
            # same stencil arithmetic per node; the norms differ only in summation order
            assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)
            assert rr == pytest.approx(rr_ref, rel=1e-12)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1502_03917_gb300.aaomg as mg

    f = torch.zeros(8, dtype=torch.float64, device="cuda")
    lib = mg.load()
    import ctypes

    code = lib.mg_residual_noalloc(13, 1.0, 0, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()), None,
                                   None, None)
    assert code == mg.ERR_BAD_ARG
    assert lib.mg_residual_noalloc(5, -1.0, 0, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()), None,
                                   None, None) == mg.ERR_BAD_ARG
