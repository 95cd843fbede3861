"""Pins for the oracle's smoothers and transfers (section 2, Algorithms 1 and 2).

The algorithms update x and carry the residual along; the paper also states
each smoother in compact matrix form.  These tests evaluate the compact forms
with dense linear algebra (a textbook triangular solve, not the residual
trick), so a wrong index, sign or visiting order in the oracle's loops fails.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1502_03917_gb300 import inputs


def setup_case(oracle_mod, L, alpha, smoother, seed=11, **kw):
    o = oracle_mod.Oracle(L, alpha, smoother=smoother, **kw)
    A = o.scipy(L, "A").toarray()
    Ld = o.ldiag()
    x = inputs.x_uniform(L, seed)
    f = inputs.x_uniform(L, seed + 1)
    return o, A, Ld, x, f


@pytest.mark.parametrize("alpha", [1.0, 1e-3, 1e-8])
@pytest.mark.parametrize("L", [2, 3, 4])
def test_ne_step_is_damped_normal_equation_richardson(oracle_mod, L, alpha):
    o, A, Ld, x, f = setup_case(oracle_mod, L, alpha, "ne")
    Li = 1.0 / Ld
    expect = x.copy()
    for _ in range(2):
        expect = expect + 0.4 * Li * (A.T @ (Li * (f - A @ expect)))
    got = o.smooth(f, x, steps=2)
    np.testing.assert_allclose(got, expect, rtol=1e-11, atol=1e-11 * np.abs(expect).max())


def colour_perm(o):
    order = o.order()
    P = np.zeros((order.size, order.size))
    P[np.arange(order.size), order] = 1.0  # (P v)_s = v[order[s]]
    return order, P


@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-6])
@pytest.mark.parametrize("L", [2, 3, 4])
def test_lsgs_step_is_forward_substitution(oracle_mod, L, alpha):
    """x <- x + P^T trig(P N P^T)^{-1} P A^T L^{-1} (f - A x), N = A^T L^{-1} A,
    P the visiting-order permutation (the compact form of the LSGS step)."""
    o, A, Ld, x, f = setup_case(oracle_mod, L, alpha, "lsgs")
    Li = 1.0 / Ld
    N = A.T @ (Li[:, None] * A)
    _, P = colour_perm(o)
    T = np.tril(P @ N @ P.T)
    expect = x.copy()
    for _ in range(2):
        g = P @ (A.T @ (Li * (f - A @ expect)))
        expect = expect + P.T @ sla.solve_triangular(T, g, lower=True)
    got = o.smooth(f, x, steps=2)
    np.testing.assert_allclose(got, expect, rtol=1e-9, atol=1e-10 * np.abs(expect).max())


@pytest.mark.parametrize("L", [2, 3])
def test_lsgs_lexicographic_order(oracle_mod, L):
    """The natural order y_1..y_N, lambda_1..lambda_N of Algorithm 2: trig(N)."""
    o, A, Ld, x, f = setup_case(oracle_mod, L, 1e-2, "lsgs", lexicographic=True)
    Li = 1.0 / Ld
    N = A.T @ (Li[:, None] * A)
    expect = x + sla.solve_triangular(np.tril(N), A.T @ (Li * (f - A @ x)), lower=True)
    np.testing.assert_allclose(o.smooth(f, x, steps=1), expect, rtol=1e-9, atol=1e-10 * np.abs(expect).max())


@pytest.mark.parametrize("L", [2, 3])
def test_slsgs_compact_form(oracle_mod, L):
    """One sLSGS step equals x + Nhat^{-1} A^T L^{-1}(f - A x) with
    Nhat = trig(N) diag(N)^{-1} trig(N)^T, in the permuted order."""
    o, A, Ld, x, f = setup_case(oracle_mod, L, 1e-4, "slsgs")
    Li = 1.0 / Ld
    _, P = colour_perm(o)
    Np = P @ (A.T @ (Li[:, None] * A)) @ P.T
    T = np.tril(Np)
    Nhat = T @ np.diag(1.0 / np.diag(Np)) @ T.T
    expect = x + P.T @ np.linalg.solve(Nhat, P @ (A.T @ (Li * (f - A @ x))))
    np.testing.assert_allclose(o.smooth(f, x, steps=1), expect, rtol=1e-8, atol=1e-9 * np.abs(expect).max())


@pytest.mark.parametrize("L", [2, 3])
def test_cgs_block_gauss_seidel(oracle_mod, L):
    """CGS: block Gauss-Seidel with the 2x2 node blocks (y_i, lambda_i) in the
    colour order (i + j) mod 3."""
    alpha = 1e-3
    o, A, Ld, x, f = setup_case(oracle_mod, L, alpha, "cgs")
    n = o.nn()
    nodes = [j * ((1 << L) + 1) + i for c in range(3) for j in range((1 << L) + 1) for i in range((1 << L) + 1)
             if (i + j) % 3 == c]
    perm = np.array([u for node in nodes for u in (node, n + node)])
    Ap = A[np.ix_(perm, perm)]
    B = np.tril(Ap)
    for b in range(n):  # keep the full 2x2 diagonal blocks
        B[2 * b, 2 * b + 1] = Ap[2 * b, 2 * b + 1]
    expect = x.copy()
    expect[perm] += np.linalg.solve(B, (f - A @ x)[perm])
    np.testing.assert_allclose(o.smooth(f, x, steps=1), expect, rtol=1e-9, atol=1e-10 * np.abs(expect).max())


@pytest.mark.parametrize("L", [3, 5, 7])
def test_colouring_is_distance_two(oracle_mod, L):
    """The visiting order is field-major, colours 0,6,5,4,3,2,1 of
    (i + 2j) mod 7, and two nodes of one colour never share a neighbour in A
    (so the updates within a colour are independent)."""
    o = oracle_mod.Oracle(L, 1.0)
    n1 = (1 << L) + 1
    nn = n1 * n1
    order = o.order()
    assert sorted(order.tolist()) == list(range(2 * nn))
    assert (order[:nn] < nn).all() and (order[nn:] >= nn).all()
    col = lambda u: ((u % nn) % n1 + 2 * ((u % nn) // n1)) % 7
    seq = [col(u) for u in order[:nn]]
    runs = [seq[0]] + [c for a, c in zip(seq, seq[1:]) if c != a]
    assert runs == [0, 6, 5, 4, 3, 2, 1]
    M = o.scipy(L, "M")
    N2 = (M @ M).tocoo()  # nonzero iff graph distance <= 2
    for p, q in zip(N2.row, N2.col):
        if p != q:
            ip, jp, iq, jq = p % n1, p // n1, q % n1, q // n1
            assert (ip + 2 * jp) % 7 != (iq + 2 * jq) % 7


@pytest.mark.parametrize("L", [3, 5, 7])
def test_cgs_colouring_is_distance_one(oracle_mod, L):
    """The CGS colours (i + j) mod 3 never couple two nodes of one colour in A
    (so the 2x2 block solves of a colour are independent and each can gather
    its residual from the current iterate), while (i - j) mod 3 would: its
    colour is shared by the diagonal neighbours (i+1, j+1) of the "/" mesh."""
    o = oracle_mod.Oracle(L, 1.0)
    n1 = (1 << L) + 1
    A = o.scipy(L, "M").tocoo()  # the coupling pattern of every block of A
    bad_minus = 0
    for p, q in zip(A.row, A.col):
        if p != q:
            ip, jp, iq, jq = p % n1, p // n1, q % n1, q // n1
            assert (ip + jp) % 3 != (iq + jq) % 3
            bad_minus += (ip - jp) % 3 == (iq - jq) % 3
    assert bad_minus > 0


@pytest.mark.parametrize("smoother", ["lsgs", "slsgs", "cgs"])
def test_least_squares_functional_decreases(oracle_mod, smoother):
    """Each LSGS update minimises Phi(x) = 1/2 ||L^{-1/2}(f - A x)||^2 along one
    coordinate, so Phi never increases from step to step."""
    L = 4
    o, A, Ld, x, f = setup_case(oracle_mod, L, 1e-5, smoother)
    phi = lambda v: 0.5 * np.sum((f - A @ v) ** 2 / Ld)
    prev = phi(x)
    for _ in range(4):
        x = o.smooth(f, x, steps=1)
        cur = phi(x)
        if smoother != "cgs":
            assert cur <= prev * (1 + 1e-12)
        prev = cur
    assert np.isfinite(prev)


def test_transfers_match_exported_P(oracle_mod):
    L = 5
    o = oracle_mod.Oracle(L, 1e-2)
    P = o.scipy(L, "P")
    nf, nc = o.nn(L), o.nn(L - 1)
    rng = np.random.default_rng(3)
    rf, xc, xf = rng.standard_normal(2 * nf), rng.standard_normal(2 * nc), rng.standard_normal(2 * nf)
    np.testing.assert_allclose(o.restrict(rf), np.concatenate([P.T @ rf[:nf], P.T @ rf[nf:]]), rtol=1e-14,
                               atol=1e-14)
    np.testing.assert_allclose(o.prolong_add(xc, xf), xf + np.concatenate([P @ xc[:nc], P @ xc[nc:]]),
                               rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("alpha", [1.0, 1e-8])
def test_coarse_solve_matches_library_solve(oracle_mod, alpha):
    o = oracle_mod.Oracle(3, alpha)
    A1 = o.scipy(1, "A").toarray()
    assert A1.shape == (18, 18)
    f = np.random.default_rng(5).standard_normal(18)
    np.testing.assert_allclose(o.coarse_solve(f), np.linalg.solve(A1, f), rtol=1e-12,
                               atol=1e-12 * np.abs(np.linalg.solve(A1, f)).max())
