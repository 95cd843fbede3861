"""GPU adjoint, autograd and batched solves.

* autograd gradients of L = 1/2 ||u - u_t||^2 (u = lambda / alpha) equal the
  direct-solve gradient built from the oracle's matrices at h = 2^-5;
* they agree with central finite differences of the GPU solve (FP64, step 1e-6);
* mg_solve_batch on independent problems of mixed size and precision gives
  every instance the oracle's solution (and bitwise its own mg_solve's).
"""
import numpy as np
import pytest

from paper_1502_03917_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def direct_gradient(oracle_mod, L, alpha, yD, ut):
    o = oracle_mod.Oracle(L, alpha)
    A, M = o.scipy(L, "A").tocsc(), o.scipy(L, "M")
    import scipy.sparse.linalg as spla

    n = M.shape[0]
    x = spla.spsolve(A, np.concatenate([M @ yD, np.zeros(n)]))
    lam = x[n:]
    r = lam / alpha - ut
    z = spla.spsolve(A, np.concatenate([np.zeros(n), r / alpha]))
    return M @ z[:n], -(r @ lam + z[n:] @ (M @ lam)) / alpha ** 2, lam / alpha


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-6])
def test_autograd_matches_direct_solve_gradient(oracle_mod, alpha, precision):
    from paper_1502_03917_gb300.autograd import control

    L = 5
    yD_np, ut_np = inputs.yd_uniform(L, 4), inputs.u_target(L, 3)
    yD = dev(yD_np).requires_grad_(True)
    la = torch.tensor(np.log(alpha), dtype=torch.float64, requires_grad=True)
    u = control(yD, la, L, tol=1e-12, precision=precision)
    loss = 0.5 * ((u - dev(ut_np)) ** 2).sum()
    loss.backward()
    g_yD, g_alpha, u_ref = direct_gradient(oracle_mod, L, alpha, yD_np, ut_np)
    np.testing.assert_allclose(u.detach().cpu().numpy(), u_ref, rtol=1e-8, atol=1e-8 * np.abs(u_ref).max())
    gy = yD.grad.cpu().numpy()
    assert np.linalg.norm(gy - g_yD) <= 1e-8 * np.linalg.norm(g_yD)
    assert la.grad.item() == pytest.approx(alpha * g_alpha, rel=1e-8)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_batched_autograd_matches_direct_solve_gradient(oracle_mod, precision):
    """Several desired states at one alpha through the batched Function (one
    batch graph forward, one batched adjoint backward): each instance's dL/dyD
    and the summed dL/dlog(alpha) equal the direct-solve gradients built from
    the oracle's matrices."""
    from paper_1502_03917_gb300.autograd import control

    L, alpha, B = 5, 1e-2, 3
    rng = np.random.default_rng(21)
    yD_np = rng.uniform(-1.0, 1.0, (B, ((1 << L) + 1) ** 2))
    ut_np = rng.standard_normal(yD_np.shape)
    yD = dev(yD_np).requires_grad_(True)
    la = torch.tensor(np.log(alpha), dtype=torch.float64, requires_grad=True)
    u = control(yD, la, L, tol=1e-12, precision=precision)
    assert u.shape == yD.shape
    loss = 0.5 * ((u - dev(ut_np)) ** 2).sum()
    loss.backward()
    g_alpha = 0.0
    for k in range(B):
        g_yD, ga, u_ref = direct_gradient(oracle_mod, L, alpha, yD_np[k], ut_np[k])
        np.testing.assert_allclose(u[k].detach().cpu().numpy(), u_ref, rtol=1e-8, atol=1e-8 * np.abs(u_ref).max())
        gy = yD.grad[k].cpu().numpy()
        assert np.linalg.norm(gy - g_yD) <= 1e-8 * np.linalg.norm(g_yD)
        g_alpha += ga
    assert la.grad.item() == pytest.approx(alpha * g_alpha, rel=1e-8)


def test_autograd_finite_differences():
    import paper_1502_03917_gb300.aaomg as mg

    L, alpha = 5, 1e-2
    yD, ut = dev(inputs.yd_uniform(L, 6)), dev(inputs.u_target(L, 7))
    v = dev(np.random.default_rng(8).standard_normal(yD.numel()))

    def loss(y, a):
        with mg.Solver(L, a, smoother="lsgs", max_iter=300) as s:
            f = s.rhs_from_yd(y)
            x = torch.zeros_like(f)
            s.solve(f, x, tol=1e-13)
            return 0.5 * float(((s.control(x) - ut) ** 2).sum())

    from paper_1502_03917_gb300.autograd import control

    y = yD.clone().requires_grad_(True)
    la = torch.tensor(np.log(alpha), dtype=torch.float64, requires_grad=True)
    lval = 0.5 * ((control(y, la, L, tol=1e-13, precision="fp64") - ut) ** 2).sum()
    lval.backward()
    h = 1e-6
    fd_y = (loss(yD + h * v, alpha) - loss(yD - h * v, alpha)) / (2 * h)
    fd_a = (loss(yD, alpha * np.exp(h)) - loss(yD, alpha * np.exp(-h))) / (2 * h)
    assert float((y.grad * v).sum()) == pytest.approx(fd_y, rel=1e-6)
    assert la.grad.item() == pytest.approx(fd_a, rel=1e-6)


def test_batch_solve_against_oracle(oracle_mod):
    """Every instance of a mixed batch (levels 3..8, alpha log-uniform in
    [1e-8, 1], both precisions) solved through mg_solve_batch equals the FP64
    oracle's multigrid solution to 1e-8 (the L norm of the error and the
    element-wise maximum of y and of u = lambda / alpha); it is also bitwise the
    result of the instance's own mg_solve."""
    import paper_1502_03917_gb300.aaomg as mg

    levels, alphas, yds = inputs.batch_instances(10, 2, lmin=3, lmax=8)
    precs = ["fp32_refine", "fp64"] * 5
    solvers = [mg.Solver(L, a, smoother="lsgs", precision=p, max_iter=200) for L, a, p in zip(levels, alphas, precs)]
    fs = [s.rhs_from_yd(dev(y)) for s, y in zip(solvers, yds)]
    xs = [torch.zeros_like(f) for f in fs]
    its, rrs, code = mg.solve_batch(solvers, fs, xs, tol=1e-11)
    assert code == mg.OK and all(r <= 1e-11 for r in rrs)
    for s, L, a, y, f, x, it in zip(solvers, levels, alphas, yds, fs, xs, its):
        o = oracle_mod.Oracle(L, a, smoother="lsgs")
        xo, _, _, _ = o.solve(o.rhs(y), tol=1e-13, max_iter=400)
        xg = x.cpu().numpy()
        n = o.nn()
        eL = o.norm_L(xg - xo) / o.norm_L(xo)
        ey = np.abs(xg[:n] - xo[:n]).max() / np.abs(xo[:n]).max()
        eu = np.abs(xg[n:] - xo[n:]).max() / np.abs(xo[n:]).max()
        assert max(eL, ey, eu) <= 1e-8, (L, a, s.precision, eL, ey, eu)
        o.close()
        x1 = torch.zeros_like(f)
        it1, rr1, _ = s.solve(f, x1, tol=1e-11)
        assert it1 == it
        assert torch.equal(x1, x)
    for s in solvers:
        s.close()


def test_batch_graph_repeated_solves_and_statuses():
    """A recorded batch (one CUDA graph, convergence tests on the device) can be
    solved again with new initial guesses and tolerances; each instance gives
    bitwise its own mg_solve's iterate, iteration count and residual history,
    and an instance that runs out of iterations reports NOT_CONVERGED without
    stopping the others."""
    import paper_1502_03917_gb300.aaomg as mg

    levels, alphas, yds = inputs.batch_instances(5, 9, lmin=4, lmax=7)
    cfg = [("lsgs", "fp32_refine", 0), ("ne", "fp64", 0), ("cgs", "fp32_refine", 0), ("lsgs", "fp64", 2),
           ("slsgs", "fp64", 0)]
    solvers = [mg.Solver(L, a, smoother=sm, precision=p, max_iter=mi if mi else 200)
               for (L, a, (sm, p, mi)) in zip(levels, alphas, cfg)]
    fs = [s.rhs_from_yd(dev(y)) for s, y in zip(solvers, yds)]
    with mg.Batch(solvers) as b:
        for rep, tol in enumerate((1e-9, 1e-11)):
            x0 = [dev(inputs.x_uniform(L, 50 + rep + k)) for k, L in enumerate(levels)]
            xs = [x.clone() for x in x0]
            its, rrs, sts, code = b.solve(fs, xs, tol=tol, raise_on_fail=False)
            assert code == mg.ERR_NOT_CONVERGED
            assert sts == [mg.OK, mg.OK, mg.OK, mg.ERR_NOT_CONVERGED, mg.OK]
            assert its[3] == 2
            hists = [s.history() for s in solvers]
            for k, s in enumerate(solvers):
                x1 = x0[k].clone()
                it1, rr1, code1 = s.solve(fs[k], x1, tol=tol, raise_on_fail=False)
                assert it1 == its[k] and rr1 == rrs[k]
                assert torch.equal(x1, xs[k])
                assert s.history() == hists[k]
                if sts[k] == mg.OK:
                    assert rrs[k] <= tol
    for s in solvers:
        s.close()


def test_batch_rejects_bad_handles():
    import paper_1502_03917_gb300.aaomg as mg

    with mg.Solver(4, 1e-2) as a, mg.Solver(4, 1e-2, profile=True) as p:
        with pytest.raises(mg.MGError) as e:
            mg.Batch([a, a])
        assert e.value.code == mg.ERR_BAD_ARG
        with pytest.raises(mg.MGError) as e:
            mg.Batch([a, p])
        assert e.value.code == mg.ERR_BAD_ARG


def test_batch_solve_host_equals_device():
    """mg_batch_solve_host (host vectors, copies inside the call) gives bitwise
    the iterates, counts and residuals of mg_batch_solve on device vectors."""
    import paper_1502_03917_gb300.aaomg as mg

    levels, alphas, yds = inputs.batch_instances(3, 11, lmin=4, lmax=7)
    solvers = [mg.Solver(L, a, smoother="lsgs", precision="fp32_refine") for L, a in zip(levels, alphas)]
    fs = [s.rhs_from_yd(dev(y)) for s, y in zip(solvers, yds)]
    with mg.Batch(solvers) as b:
        xs = [torch.zeros_like(f) for f in fs]
        its, rrs, sts, code = b.solve(fs, xs, tol=1e-10)
        hf = [f.cpu().numpy().copy() for f in fs]
        hx = [np.zeros(f.numel()) for f in fs]
        its_h, rrs_h, sts_h, code_h = b.solve_host(hf, hx, tol=1e-10)
    assert code == code_h == mg.OK and its == its_h and rrs == rrs_h and sts == sts_h
    for x, xh in zip(xs, hx):
        assert np.array_equal(x.cpu().numpy(), xh)
    for s in solvers:
        s.close()
