"""GPU parity: every step of the CUDA path against the FP64 oracle, through the
C ABI, element by element, on seeded inputs: every comparison bounds both the
normwise relative difference of each field and its element-wise maximum
relative to the field's largest entry.

Tolerances: FP64 path 1e-12 relative difference per step (sum-order rounding
only), FP32 path 1e-5 per step (single-precision rounding of a handful of
operations per unknown), solutions 1e-8 relative error (solved to a relative
residual of 1e-11 so that the error bound holds for every alpha).
"""
import numpy as np
import pytest

from paper_1502_03917_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32_refine": 1e-5}


@pytest.fixture(scope="module")
def mg():
    import paper_1502_03917_gb300.aaomg as m

    m.load()
    return m


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def field_reldiff(a, b, n):
    """max over the two fields of ||a - b|| / ||b||"""
    out = 0.0
    for s in (slice(0, n), slice(n, 2 * n)):
        nb = np.linalg.norm(b[s])
        out = max(out, np.linalg.norm(a[s] - b[s]) / (nb if nb > 0 else 1.0))
    return out


def field_maxrel(a, b, n):
    """max over the two fields of max_i |a_i - b_i| / max_i |b_i|: element by
    element, so that a few wrong nodes (a boundary row, a tile edge) cannot
    hide in a norm over millions of correct ones"""
    out = 0.0
    for s in (slice(0, n), slice(n, 2 * n)):
        nb = np.abs(b[s]).max()
        out = max(out, np.abs(a[s] - b[s]).max() / (nb if nb > 0 else 1.0))
    return out


def field_diff(a, b, n):
    """both measures at once: a test's tolerance bounds the normwise and the
    element-wise relative difference"""
    return max(field_reldiff(a, b, n), field_maxrel(a, b, n))


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("smoother", ["ne", "lsgs", "slsgs", "cgs"])
@pytest.mark.parametrize("L", [2, 3, 5, 7, 9])
@pytest.mark.parametrize("alpha", [1.0, 1e-4, 1e-8])
def test_smoother_step_parity(mg, oracle_mod, L, alpha, smoother, precision):
    x0 = inputs.f32_exact(inputs.x_uniform(L, 100 + L))
    f = inputs.f32_exact(inputs.x_uniform(L, 200 + L))
    o = oracle_mod.Oracle(L, alpha, smoother=smoother)
    n = o.nn()
    with mg.Solver(L, alpha, smoother=smoother, precision=precision) as s:
        for steps in (1, 2):
            x = dev(x0)
            s.smooth(dev(f), x, steps)
            got = host(x)
            want = o.smooth(f, x0, steps)
            d = field_diff(got, want, n)
            assert d <= TOL[precision], (steps, d)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("smoother", ["ne", "lsgs", "slsgs", "cgs"])
@pytest.mark.parametrize("L,small_max", [(6, 0), (8, 0), (10, 0), (6, -1), (8, -1), (9, 300)])
def test_smoothing_call_kernels(mg, oracle_mod, L, small_max, smoother, precision):
    """The one-launch smoothing call (one block with the residual in shared
    memory, or one cluster with x and the residual in its blocks' shared
    memory) and the per-phase launches (small_max = -1) give the oracle's
    steps."""
    alpha = 1e-2
    x0 = inputs.f32_exact(inputs.x_uniform(L, 500 + L))
    f = inputs.f32_exact(inputs.x_uniform(L, 600 + L))
    o = oracle_mod.Oracle(L, alpha, smoother=smoother)
    with mg.Solver(L, alpha, smoother=smoother, precision=precision, small_max=small_max) as s:
        for steps in (1, 2):
            x = dev(x0)
            s.smooth(dev(f), x, steps)
            d = field_diff(host(x), o.smooth(f, x0, steps), o.nn())
            assert d <= TOL[precision], (steps, d)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("smoother", ["ne", "lsgs", "slsgs", "cgs"])
@pytest.mark.parametrize("L,cs", [(6, 2), (6, 3), (6, 16), (7, 5), (7, 16), (8, 12), (8, 16)])
def test_cluster_smoothing_call(mg, oracle_mod, L, cs, smoother, precision):
    """The one-launch smoothing call on a cluster of cs blocks (grid rows split
    into cs strips, uneven ones included; neighbouring strips reached through
    distributed shared memory) gives the oracle's steps."""
    alpha = 1e-2
    x0 = inputs.f32_exact(inputs.x_uniform(L, 700 + L))
    f = inputs.f32_exact(inputs.x_uniform(L, 800 + L))
    o = oracle_mod.Oracle(L, alpha, smoother=smoother)
    with mg.Solver(L, alpha, smoother=smoother, precision=precision, cluster_size=cs) as s:
        for steps in (1, 2):
            x = dev(x0)
            s.smooth(dev(f), x, steps)
            d = field_diff(host(x), o.smooth(f, x0, steps), o.nn())
            assert d <= TOL[precision], (steps, d)


@pytest.mark.parametrize("L", [9, 10])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("smoother", ["lsgs", "cgs"])
def test_autotuned_kernels(mg, oracle_mod, smoother, precision, L):
    """With autotune the set-up picks each level's kernel by timing (strips
    cluster sizes; per-phase launches or the band kernel in one of three
    tilings); whatever it picks, a smoothing call still gives the oracle's
    steps and a solve the oracle's solution."""
    alpha = 1e-2
    x0 = inputs.f32_exact(inputs.x_uniform(L, 900))
    f = inputs.f32_exact(inputs.x_uniform(L, 901))
    o = oracle_mod.Oracle(L, alpha, smoother=smoother)
    with mg.Solver(L, alpha, smoother=smoother, precision=precision, autotune=True) as s:
        x = dev(x0)
        s.smooth(dev(f), x, 2)
        d = field_diff(host(x), o.smooth(f, x0, 2), o.nn())
        assert d <= TOL[precision], d
        yD = inputs.yd_uniform(L, 0)
        fs = s.rhs_from_yd(dev(yD))
        xs = torch.zeros_like(fs)
        it, rr, code = s.solve(fs, xs, tol=1e-10)
        assert code == 0 and rr <= 1e-10
        kinds = s.level_kernels()
        assert all(kinds[l][0] == "coarse" for l in range(1, 6))
        assert all(kinds[l][0] in ("strips", "band", "phases") for l in range(6, L + 1))
    with mg.Solver(L, alpha, smoother=smoother, precision=precision) as s:
        xd = torch.zeros_like(fs)
        s.solve(s.rhs_from_yd(dev(yD)), xd, tol=1e-10)
    assert field_diff(host(xs), host(xd), o.nn()) <= 1e-8


@pytest.mark.parametrize("L,cs", [(8, 2), (7, 17), (6, 64)])
def test_cluster_size_that_cannot_run(mg, L, cs):
    """A forced cluster size whose strips do not fit in shared memory, or that
    exceeds the cluster limit, is refused at set-up."""
    with pytest.raises(mg.MGError) as e:
        mg.Solver(L, 1e-2, smoother="lsgs", precision="fp32_refine", cluster_size=cs)
    assert e.value.code == -1


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("tile", [(0, 0), (20, 9), (1, 1), (57, 130), (3, 40)])
@pytest.mark.parametrize("L", [2, 4, 8])
def test_lsgs_step_kernel_tiling(mg, oracle_mod, L, tile, precision):
    """The one-launch LSGS step (wavefront over bands of columns and segments
    of rows, with recomputed halos) equals the sequential multicolour sweep for
    every tiling, including one-node tiles and an odd number of steps."""
    alpha = 1e-3
    x0 = inputs.f32_exact(inputs.x_uniform(L, 300 + L))
    f = inputs.f32_exact(inputs.x_uniform(L, 400 + L))
    o = oracle_mod.Oracle(L, alpha, smoother="lsgs")
    with mg.Solver(L, alpha, smoother="lsgs", precision=precision, tile_w=tile[0], tile_h=tile[1]) as s:
        for steps in (1, 3):
            x = dev(x0)
            s.smooth(dev(f), x, steps)
            d = field_diff(host(x), o.smooth(f, x0, steps), o.nn())
            assert d <= TOL[precision], (steps, d)


@pytest.mark.parametrize("tile", [(0, 0), (0, 700), (100, 0)])
@pytest.mark.parametrize("alpha", [1.0, 1e-8])
def test_band_step_parity_L10(mg, oracle_mod, alpha, tile):
    """The one-launch LSGS step at h = 2^-10 (1025^2 nodes, the size from which
    the FP32 cycles use it), in the default tiling (bands of columns, one row
    segment per block of a full wave), with tall segments and with narrow
    bands, equals the oracle's multicolour sweep element by element."""
    L = 10
    x0 = inputs.f32_exact(inputs.x_uniform(L, 1000))
    f = inputs.f32_exact(inputs.x_uniform(L, 1001))
    o = oracle_mod.Oracle(L, alpha, smoother="lsgs")
    with mg.Solver(L, alpha, smoother="lsgs", precision="fp32_refine", tile_w=tile[0], tile_h=tile[1]) as s:
        assert s.level_kernels()[L][0] == "band"
        for steps in (1, 2):
            x = dev(x0)
            s.smooth(dev(f), x, steps)
            d = field_diff(host(x), o.smooth(f, x0, steps), o.nn())
            assert d <= TOL["fp32_refine"], (steps, d)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("L", [2, 4, 7])
def test_transfer_parity(mg, oracle_mod, L, precision):
    alpha = 1e-3
    o = oracle_mod.Oracle(L, alpha)
    n, nc = o.nn(L), o.nn(L - 1)
    x = inputs.f32_exact(inputs.x_uniform(L, 7))
    f = inputs.f32_exact(inputs.x_uniform(L, 8))
    xc = inputs.f32_exact(inputs.x_uniform(L - 1, 9))
    with mg.Solver(L, alpha, precision=precision) as s:
        fc = host(s.restrict(dev(f), dev(x)))
        want = o.restrict(o.residual(f, x))
        assert field_diff(fc, want, nc) <= TOL[precision]
        xg = dev(x)
        s.prolong_add(dev(xc), xg)
        assert field_diff(host(xg), o.prolong_add(xc, x), n) <= TOL[precision]


@pytest.mark.parametrize("L", [1, 3, 6])
def test_residual_and_rhs_parity(mg, oracle_mod, L):
    alpha = 1e-5
    o = oracle_mod.Oracle(L, alpha)
    n = o.nn()
    yD = inputs.yd_sine_noise(L, 1)
    x = inputs.x_uniform(L, 3)
    with mg.Solver(L, alpha) as s:
        f = s.rhs_from_yd(dev(yD))
        fo = o.rhs(yD)
        assert np.linalg.norm(host(f)[:n] - fo[:n]) / np.linalg.norm(fo[:n]) <= 1e-13
        assert np.all(host(f)[n:] == 0.0)
        r = torch.empty_like(f)
        rr = s.residual(f, dev(x), r)
        ro = o.residual(fo, x)
        assert np.linalg.norm(host(r) - ro) / np.linalg.norm(ro) <= 1e-13
        assert rr == pytest.approx(o.norm_Linv(ro) / o.norm_Linv(fo), rel=1e-12)


@pytest.mark.parametrize("coarse_level", [-1, 0, 3])
@pytest.mark.parametrize("cycle", ["W", "V"])
@pytest.mark.parametrize("smoother", ["ne", "lsgs", "slsgs", "cgs"])
@pytest.mark.parametrize("L", [1, 2, 4, 7])
def test_cycle_parity_fp64(mg, oracle_mod, L, smoother, cycle, coarse_level):
    """coarse_level -1: default single-block coarse kernel (levels <= 5 in
    FP64); 0: grid-wide kernels on every level; 3: a mix.  Per sweep the two
    sides differ by summation order only (1e-12); a cycle then solves the
    coarse problem from a defect carrying that rounding, which the condition
    number of the operator, O(h^-2) = O(4^L), amplifies: tol = max(1e-12,
    2^-52 4^L) (CGS recomputes each node's residual where the oracle carries
    it, which shows this at L = 7)."""
    alpha = 1e-2
    nu = 1 if smoother == "slsgs" else 2
    o = oracle_mod.Oracle(L, alpha, smoother=smoother, gamma=2 if cycle == "W" else 1, nu_pre=nu, nu_post=nu)
    f = o.rhs(inputs.yd_uniform(L, 0))
    x0 = inputs.x_uniform(L, 4)
    with mg.Solver(L, alpha, smoother=smoother, cycle=cycle, coarse_level=coarse_level) as s:
        x = dev(x0)
        s.cycle(dev(f), x)
        want = o.cycle(f, x0)
        assert field_diff(host(x), want, o.nn()) <= max(1e-12, 2.0 ** -52 * 4.0 ** L)


@pytest.mark.parametrize("coarse_level", [-1, 0])
@pytest.mark.parametrize("smoother", ["ne", "lsgs", "cgs"])
@pytest.mark.parametrize("L", [3, 6, 8])
def test_refinement_step_parity_fp32(mg, oracle_mod, L, smoother, coarse_level):
    """One FP32 cycle inside the refinement step: its correction matches one
    FP64 oracle cycle on the same defect to single-precision accuracy.  A
    cycle is more than a sweep: the coarse-grid correction of the smooth modes
    is solved from a defect rounded to FP32, which amplifies the unit roundoff
    2^-24 by up to the condition number of the scaled operator, O(h^-2) = O(4^L).
    Hence tol = max(1e-4, 2^-24 4^L); the FP64 refinement removes this error."""
    alpha = 1e-3
    o = oracle_mod.Oracle(L, alpha, smoother=smoother)
    f = o.rhs(inputs.yd_uniform(L, 5))
    x0 = inputs.x_uniform(L, 6)
    with mg.Solver(L, alpha, smoother=smoother, precision="fp32_refine", inner_cycles=1,
                   coarse_level=coarse_level) as s:
        x = dev(x0)
        s.cycle(dev(f), x)
        # FP64 reference: x0 + one cycle on A d = f - A x0 from d = 0
        r = o.residual(f, x0)
        d = o.cycle(r, np.zeros_like(r))
        want = x0 + d
        dg = host(x) - x0
        assert field_diff(dg, d, o.nn()) <= max(1e-4, 2.0 ** -24 * 4.0 ** L)


def solution_errors(o, x, xo):
    n = o.nn()
    eL = o.norm_L(x - xo) / o.norm_L(xo)
    ey = np.abs(x[:n] - xo[:n]).max() / np.abs(xo[:n]).max()
    eu = np.abs(x[n:] - xo[n:]).max() / np.abs(xo[n:]).max()  # u = lambda / alpha: same relative error
    return max(eL, ey, eu)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("smoother", ["ne", "lsgs", "cgs"])
@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-4, 1e-6, 1e-8])
def test_solve_parity_L5(mg, oracle_mod, alpha, smoother, precision):
    L = 5
    yD = inputs.yd_uniform(L, 0)
    o = oracle_mod.Oracle(L, alpha, smoother=smoother)
    fo = o.rhs(yD)
    xo, ito, _, _ = o.solve(fo, tol=1e-13, max_iter=400)
    with mg.Solver(L, alpha, smoother=smoother, precision=precision, max_iter=200) as s:
        f = s.rhs_from_yd(dev(yD))
        x = torch.zeros_like(f)
        it, rr, _ = s.solve(f, x, tol=1e-11)
        assert rr <= 1e-11
        assert solution_errors(o, host(x), xo) <= 1e-8
        if precision == "fp64":
            # same iterates as the oracle: identical iteration count to the same tolerance
            _, it_o, _, _ = o.solve(fo, tol=1e-11)
            assert it == it_o


def test_solve_host_and_history(mg, oracle_mod):
    L, alpha = 4, 1e-3
    o = oracle_mod.Oracle(L, alpha, smoother="lsgs")
    f = o.rhs(inputs.yd_uniform(L, 1))
    xo, _, _, hist_o = o.solve(f, tol=1e-10)
    with mg.Solver(L, alpha, smoother="lsgs") as s:
        x = np.zeros_like(f)
        it, rr, _ = s.solve_host(np.ascontiguousarray(f), x, tol=1e-10)
        assert solution_errors(o, x, xo) <= 1e-8
        h = s.history()
        assert len(h) == it + 1
        # residual norms below ~1e-8 sit at the cancellation floor of f - A x
        # (absolute differences ~1e-16 of ||f||), hence the absolute term
        np.testing.assert_allclose(h, hist_o, rtol=1e-7, atol=1e-14)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("alpha", [1.0, 1e-6])
def test_norms_match_oracle(mg, oracle_mod, alpha, precision):
    """mg_norms: ||x||_L and ||x||_{L^-1} with the paper's L = diag(Q)."""
    L = 5
    o = oracle_mod.Oracle(L, alpha)
    x0 = inputs.x_uniform(L, 11)
    with mg.Solver(L, alpha, precision=precision) as s:
        nl, ninv = s.norms(dev(x0))
    assert nl == pytest.approx(o.norm_L(x0), rel=1e-13)
    assert ninv == pytest.approx(o.norm_Linv(x0), rel=1e-13)


@pytest.mark.parametrize("smoother", ["ne", "lsgs", "slsgs", "cgs"])
@pytest.mark.parametrize("k", [5, 6])
@pytest.mark.parametrize("alpha", [1.0, 1e-6, 1e-12])
def test_protocol_iterations_match_oracle(mg, oracle_mod, k, alpha, smoother):
    """Section 3's protocol (zero right-hand side, random start, W-cycles until
    the error in the L norm has dropped by 1e-6; 2+2 steps, sLSGS 1+1) on the
    GPU in FP64 takes exactly the oracle's iteration count in the same colour
    order: the iterates agree to rounding."""
    nu = 1 if smoother == "slsgs" else 2
    o = oracle_mod.Oracle(k, alpha, smoother=smoother, nu_pre=nu, nu_post=nu)
    x0 = inputs.x_uniform(k, 7)
    want = o.protocol_iterations(x0, 1e-6, 300)
    with mg.Solver(k, alpha, smoother=smoother, precision="fp64", nu_pre=nu, nu_post=nu) as s:
        got = s.protocol_iterations(dev(x0), 1e-6, 300)
    assert got == want > 0


def test_default_level_kernels(mg):
    """The per-level kernels of the default FP32 LSGS configuration at
    h = 2^-11: the dense level-5 map below, one block on level 6, clusters of
    16 blocks on levels 7 and 8 (x and residual on chip) and on level 9 (the
    residual on chip, x in global memory), the band kernel on levels 10 and
    11; FP64 keeps one launch per colour phase on level 9."""
    with mg.Solver(11, 1e-2, smoother="lsgs", precision="fp32_refine") as s:
        k = s.level_kernels()
    assert [k[l][0] for l in range(1, 6)] == ["coarse"] * 5
    assert k[6] == ("strips", 1) and k[7] == ("strips", 16) and k[8] == ("strips", 16)
    assert k[9] == ("strips", 16)
    assert all(k[l][0] == "band" and k[l][1] > 0 for l in (10, 11))
    with mg.Solver(10, 1e-2, smoother="lsgs", precision="fp64") as s:
        assert s.level_kernels()[9] == ("phases", 0)
    with mg.Solver(10, 1e-2, smoother="cgs", precision="fp32_refine") as s:
        assert s.level_kernels()[9] == ("phases", 0)


@pytest.mark.parametrize("smoother", ["lsgs", "slsgs"])
@pytest.mark.parametrize("alpha", [1.0, 1e-8])
def test_level_513_cluster_kernel(mg, oracle_mod, smoother, alpha):
    """The 513 x 513 cluster kernel (residual in the 16 blocks' shared memory,
    iterate updated in global memory) gives the oracle's smoothing steps, one
    step and a call of three, and a W-cycle of a h = 2^-10 problem that visits
    it matches one with per-phase launches there (small_max = 257)."""
    L = 9
    x0 = inputs.f32_exact(inputs.x_uniform(L, 1100))
    f = inputs.f32_exact(inputs.x_uniform(L, 1101))
    o = oracle_mod.Oracle(L, alpha, smoother=smoother)
    with mg.Solver(L, alpha, smoother=smoother, precision="fp32_refine") as s:
        assert s.level_kernels()[L] == ("strips", 16)
        for steps in (1, 3):
            x = dev(x0)
            s.smooth(dev(f), x, steps)
            d = field_diff(host(x), o.smooth(f, x0, steps), o.nn())
            assert d <= TOL["fp32_refine"], (steps, d)
    yD = dev(inputs.yd_uniform(10, 3))
    out = []
    for small_max in (0, 257):
        with mg.Solver(10, alpha, smoother=smoother, precision="fp32_refine", small_max=small_max) as s:
            assert s.level_kernels()[9] == (("strips", 16) if small_max == 0 else ("phases", 0))
            fs = s.rhs_from_yd(yD)
            x = torch.zeros_like(fs)
            s.solve(fs, x, tol=1e-10)
            out.append(host(x))
    n = out[0].size // 2
    assert field_diff(out[0], out[1], n) <= 1e-8


def test_profile_of_one_level(mg):
    """profile_level times the smoothing calls of that level: a W-cycle from
    level 8 visits level 6 four times, with nu_pre + nu_post = 4 steps a visit,
    in each of the 3 inner cycles of every refinement step."""
    L = 8
    with mg.Solver(L, 1e-2, smoother="lsgs", precision="fp32_refine", profile=True, profile_level=6,
                   inner_cycles=3) as s:
        f = s.rhs_from_yd(dev(inputs.yd_sine_noise(L, 1)))
        x = torch.zeros_like(f)
        it, rr, code = s.solve(f, x, tol=1e-6)
        ms, sweeps = s.profile()
        assert code == 0 and ms > 0.0
        assert sweeps == it * 3 * 4 * 4


def test_determinism(mg):
    L, alpha = 6, 1e-4
    yD = dev(inputs.yd_uniform(L, 3))
    outs = []
    for _ in range(2):
        with mg.Solver(L, alpha, smoother="lsgs", precision="fp32_refine") as s:
            f = s.rhs_from_yd(yD)
            x = torch.zeros_like(f)
            s.solve(f, x, tol=1e-10)
            outs.append(host(x))
    assert np.array_equal(outs[0], outs[1])


def test_bad_arguments(mg):
    for args in ((0, 1.0), (14, 1.0), (5, 0.0), (5, -1.0), (5, float("nan")), (5, float("inf"))):
        with pytest.raises(mg.MGError) as e:
            mg.Solver(*args)
        assert e.value.code == mg.ERR_BAD_ARG
    with mg.Solver(3, 1.0) as s:
        lib = mg.load()
        assert lib.mg_solve(s._h, None, None, 1e-8, None, None, None) == mg.ERR_BAD_ARG
        assert lib.mg_smooth(None, None, None, 1, None) == mg.ERR_BAD_ARG


def test_not_converged_and_nan(mg):
    L = 5
    with mg.Solver(L, 1e-2, smoother="ne", max_iter=2) as s:
        f = s.rhs_from_yd(dev(inputs.yd_uniform(L, 0)))
        x = torch.zeros_like(f)
        it, rr, code = s.solve(f, x, tol=1e-12, raise_on_fail=False)
        assert code == mg.ERR_NOT_CONVERGED and it == 2
        x[5] = float("nan")
        it, rr, code = s.solve(f, x, tol=1e-12, raise_on_fail=False)
        assert code == mg.ERR_DIVERGED


def test_constant_desired_state(mg):
    L, alpha, c = 6, 1e-3, -0.4
    with mg.Solver(L, alpha, smoother="lsgs", precision="fp32_refine") as s:
        f = s.rhs_from_yd(torch.full((s.N,), c, dtype=torch.float64, device="cuda"))
        x = torch.zeros_like(f)
        s.solve(f, x, tol=1e-12)
        xh = host(x)
        np.testing.assert_allclose(xh[: s.N], c / (1 + alpha), rtol=1e-9)
        np.testing.assert_allclose(xh[s.N:], alpha * c / (1 + alpha), rtol=1e-8)


def test_device_peaks_are_plausible(mg):
    """The microbenchmarks behind the roofline report rates in the order the
    hardware has them: packed FP32 far above FP64, L2-resident reads above the
    HBM copy, and an HBM copy bandwidth of a few TB/s."""
    p = mg.device_peaks()
    assert p["fp32_tflops"] > 10 * p["fp64_tflops"] > 0
    assert p["l2_gbs"] > p["hbm_copy_gbs"] > 1000
