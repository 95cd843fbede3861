"""Pins for the Stokes control oracle (section 1, second model problem,
eq. (mp3); section 2; Algorithms 1 and 2; section 3, Table 2).

Each check compares the oracle with something other than itself: exact
integrals of polynomials the Taylor-Hood spaces reproduce, the P1 mass matrix
of the (separately pinned) Poisson oracle, the Galerkin identities of nested
spaces, the compact matrix forms of the smoothers evaluated with dense linear
algebra, a sparse direct solve, and the iteration counts the paper prints.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_1502_03917_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_iterations.txt")


def half_grid(L):
    n = 1 << L
    t = np.arange(2 * n + 1, dtype=np.float64) / (2 * n)
    X, Y = np.meshgrid(t, t, indexing="xy")
    return X.ravel(), Y.ravel()


def vertices(L):
    n = 1 << L
    t = np.arange(n + 1, dtype=np.float64) / n
    X, Y = np.meshgrid(t, t, indexing="xy")
    return X.ravel(), Y.ravel()


def interior_of_half_grid(L):
    """half-step grid index of every velocity unknown"""
    n = 1 << L
    ng = 2 * n + 1
    b, a = np.divmod(np.arange((2 * n - 1) ** 2), 2 * n - 1)
    return (b + 1) * ng + (a + 1)


def square_integral(poly):
    """int over [0,1]^2 of sum c x^a y^b, poly = {(a, b): c}"""
    return sum(c / ((a + 1) * (b + 1)) for (a, b), c in poly.items())


# ----------------------------------------------------------- assembly --


@pytest.mark.parametrize("L", [1, 2, 4])
def test_p2_mass_integrates_quadratics_exactly(stokes_mod, L):
    o = stokes_mod.StokesOracle(L, 1.0)
    Mf = o.scipy(L, "Mf")
    X, Y = half_grid(L)
    one = np.ones_like(X)
    assert abs(one @ Mf @ one - 1.0) < 1e-13
    # P2 interpolants of x^2 and y^2 are exact; their product has degree 4
    assert abs((X * X) @ Mf @ (Y * Y) - 1.0 / 9.0) < 1e-13
    assert abs((X * X) @ Mf @ (X * Y) - 1.0 / 8.0) < 1e-13
    assert abs(o.pweights().sum() - 1.0) < 1e-13


@pytest.mark.parametrize("L", [1, 3])
def test_p2_stiffness_integrates_gradients_exactly(stokes_mod, L):
    o = stokes_mod.StokesOracle(L, 1.0)
    Kf = o.scipy(L, "Kf")
    X, Y = half_grid(L)
    q = X * X + 3 * X * Y - 2 * Y * Y + X
    # grad q = (2x + 3y + 1, 3x - 4y)
    g2 = {(2, 0): 4 + 9, (0, 2): 9 + 16, (0, 0): 1, (1, 1): 12 - 24, (1, 0): 4, (0, 1): 6}
    assert abs(q @ Kf @ q - square_integral(g2)) < 1e-12
    assert np.abs(Kf @ np.ones_like(X)).max() < 1e-12


@pytest.mark.parametrize("L", [1, 2, 4])
def test_divergence_against_p1_mass(stokes_mod, oracle_mod, L):
    """(D v)_q = -int psi_q div v: for v = (x^2 + y, xy - 3y^2) (in P2),
    div v = 3x - 6y, and int psi_q g = (M_P1 g)_q for linear g, with M_P1 the
    Poisson oracle's P1 mass matrix."""
    o = stokes_mod.StokesOracle(L, 1.0)
    X, Y = half_grid(L)
    v1, v2 = X * X + Y, X * Y - 3 * Y * Y
    Dv = o.scipy(L, "Dxf") @ v1 + o.scipy(L, "Dyf") @ v2
    M1 = oracle_mod.Oracle(L, 1.0).scipy(L, "M")
    Xv, Yv = vertices(L)
    np.testing.assert_allclose(Dv, -(M1 @ (3 * Xv - 6 * Yv)), atol=1e-13)


@pytest.mark.parametrize("L", [1, 3])
def test_gradient_on_interior_velocities(stokes_mod, L):
    """D^T is the discrete gradient: for velocities vanishing on the boundary,
    -int p d_c phi_i = int (d_c p) phi_i, so p = 2x + 5y gives
    D_x^T p = 2 int phi_i and D_y^T p = 5 int phi_i."""
    o = stokes_mod.StokesOracle(L, 1.0)
    Xv, Yv = vertices(L)
    p = 2 * Xv + 5 * Yv
    ints = (o.scipy(L, "Mf") @ np.ones(half_grid(L)[0].size))[interior_of_half_grid(L)]
    np.testing.assert_allclose(o.scipy(L, "Dx").T @ p, 2 * ints, atol=1e-14)
    np.testing.assert_allclose(o.scipy(L, "Dy").T @ p, 5 * ints, atol=1e-14)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_galerkin_identities(stokes_mod, L):
    """Nested spaces: the coarse matrices are the fine ones seen through the
    canonical embeddings (P2 for velocities, P1 for pressures)."""
    o = stokes_mod.StokesOracle(L, 1.0)
    P2, P1 = o.scipy(L, "P2"), o.scipy(L, "P1")
    for w in ("M", "K"):
        d = (P2.T @ o.scipy(L, w) @ P2 - o.scipy(L - 1, w)).toarray()
        assert np.abs(d).max() < 1e-13 * max(1.0, np.abs(o.scipy(L - 1, w).toarray()).max()), w
    for w in ("Dx", "Dy"):
        d = (P1.T @ o.scipy(L, w) @ P2 - o.scipy(L - 1, w)).toarray()
        assert np.abs(d).max() < 1e-14, w
    # the P1 embedding reproduces linear functions
    Xc, Yc = vertices(L - 1)
    Xf, Yf = vertices(L)
    np.testing.assert_allclose(P1 @ (2 * Xc - Yc + 1), 2 * Xf - Yf + 1, atol=1e-14)


@pytest.mark.parametrize("alpha", [1.0, 1e-6])
@pytest.mark.parametrize("L", [1, 2, 3])
def test_kernel_is_the_constant_pressures(stokes_mod, L, alpha):
    """A of eq. (mp3) is symmetric with exactly the two constant modes of p and
    mu in its kernel (inf-sup stable Taylor-Hood pair)."""
    o = stokes_mod.StokesOracle(L, alpha)
    s = o.sizes()
    A = o.scipy(L, "A")
    assert abs(A - A.T).max() == 0.0
    for off in (s["p"], s["mu"]):
        e = np.zeros(s["m"])
        e[off: off + s["np"]] = 1.0
        assert np.abs(A @ e).max() < 1e-12 * abs(A).max()
    if L <= 2:
        # in the L-scaled form L^{-1/2} A L^{-1/2}, whose spectrum is bounded
        # independently of alpha and h (section 2)
        d = 1.0 / np.sqrt(o.ldiag())
        sv = np.linalg.svd(d[:, None] * A.toarray() * d[None, :], compute_uv=False)
        assert sv[-1] < 1e-12 * sv[0] and sv[-2] < 1e-12 * sv[0] and sv[-3] > 1e-4 * sv[0]


# ---------------------------------------------------------- smoothers --


def case(stokes_mod, L, alpha, smoother, seed=21, **kw):
    o = stokes_mod.StokesOracle(L, alpha, smoother=smoother, **kw)
    A = o.scipy(L, "A").toarray()
    Ld = o.ldiag()
    x = inputs.stokes_x_uniform(L, seed)
    f = inputs.stokes_x_uniform(L, seed + 1)
    return o, A, Ld, x, f


@pytest.mark.parametrize("alpha", [1.0, 1e-6])
@pytest.mark.parametrize("L", [1, 2])
def test_ne_step_compact_form(stokes_mod, L, alpha):
    o, A, Ld, x, f = case(stokes_mod, L, alpha, "ne")
    Li = 1.0 / Ld
    expect = x.copy()
    for _ in range(2):
        expect = expect + 0.35 * Li * (A.T @ (Li * (f - A @ expect)))
    np.testing.assert_allclose(o.smooth(f, x, 2), expect, rtol=1e-10, atol=1e-10 * np.abs(expect).max())


def perm(order):
    P = np.zeros((order.size, order.size))
    P[np.arange(order.size), order] = 1.0
    return P


@pytest.mark.parametrize("lexicographic", [False, True])
@pytest.mark.parametrize("alpha", [1.0, 1e-6])
@pytest.mark.parametrize("L", [1, 2])
def test_lsgs_and_slsgs_compact_forms(stokes_mod, L, alpha, lexicographic):
    """LSGS: x + P^T trig(P N P^T)^{-1} P A^T L^{-1} r; sLSGS: x + P^T Nhat^{-1}
    P A^T L^{-1} r with Nhat = trig D^{-1} trig^T (eq. (eqmcNhat)), N = A^T
    L^{-1} A, P the visiting order."""
    for smoother in ("lsgs", "slsgs"):
        o, A, Ld, x, f = case(stokes_mod, L, alpha, smoother, lexicographic=lexicographic)
        Li = 1.0 / Ld
        N = A.T @ (Li[:, None] * A)
        P = perm(o.order())
        T = np.tril(P @ N @ P.T)
        Dg = np.diag(np.diag(T))
        expect = x.copy()
        for _ in range(2):
            g = P @ (A.T @ (Li * (f - A @ expect)))
            if smoother == "lsgs":
                d = sla.solve_triangular(T, g, lower=True)
            else:
                d = sla.solve_triangular(T.T, Dg @ sla.solve_triangular(T, g, lower=True), lower=False)
            expect = expect + P.T @ d
        got = o.smooth(f, x, 2)
        np.testing.assert_allclose(got, expect, rtol=1e-8, atol=1e-9 * np.abs(expect).max())


@pytest.mark.parametrize("L", [2, 3, 4])
def test_multicolour_classes_have_disjoint_rows(stokes_mod, L):
    """The multicolour order is block by block (v_1, v_2, p, lambda_1,
    lambda_2, mu), colours (a + 7b) mod 19 on the P2 half-step grid and
    (i + 2j) mod 7 on the vertices, ascending; the unknowns of one class touch
    disjoint rows of A, so their Algorithm 2 updates commute."""
    o = stokes_mod.StokesOracle(L, 1e-2)
    s = o.sizes()
    n, nv, npn = s["n"], s["nv"], s["np"]
    idx = np.arange(nv)
    b, a = np.divmod(idx, 2 * n - 1)
    vcol = (a + 1 + 7 * (b + 1)) % 19
    j, i = np.divmod(np.arange(npn), n + 1)
    pcol = (i + 2 * j) % 7
    blocks = [(0, vcol), (nv, vcol), (2 * nv, pcol), (2 * nv + npn, vcol), (3 * nv + npn, vcol),
              (4 * nv + npn, pcol)]
    key = np.empty(s["m"], np.int64)
    for bi, (off, col) in enumerate(blocks):
        key[off: off + col.size] = bi * 100 + col
    order = o.order()
    assert sorted(order.tolist()) == list(range(s["m"]))
    k = key[order]
    assert np.all(np.diff(k) >= 0)
    A = abs(o.scipy(L, "A")).tocsc()
    A.data[:] = 1.0
    for c in np.unique(key):
        cols = np.nonzero(key == c)[0]
        hits = np.asarray(A[:, cols].sum(axis=1)).ravel()
        assert hits.max() <= 1.0, c


# --------------------------------------------------- solves, Table 2 --


@pytest.mark.parametrize("alpha", [1.0, 1e-8])
def test_coarse_solve_picks_zero_mean_pressures(stokes_mod, alpha):
    o = stokes_mod.StokesOracle(1, alpha)
    A = o.scipy(1, "A")
    xr = inputs.stokes_x_uniform(1, 5)
    x = o.coarse_solve(A @ xr)
    xn = o.normalize(xr, 1)
    assert o.norm_L(x - xn, 1) <= 1e-11 * o.norm_L(xn, 1)


def bordered_direct(o, f):
    L = o.L
    s = o.sizes()
    A = o.scipy(L, "A")
    w = o.pweights()
    C = sp.lil_matrix((s["m"], 2))
    C[s["p"]: s["p"] + s["np"], 0] = w[:, None]
    C[s["mu"]: s["mu"] + s["np"], 1] = w[:, None]
    C = C.tocsr()
    B = sp.bmat([[A, C], [C.T, None]]).tocsc()
    return spla.spsolve(B, np.concatenate([f, [0.0, 0.0]]))[: s["m"]]


@pytest.mark.parametrize("smoother", ["ne", "lsgs", "slsgs"])
@pytest.mark.parametrize("alpha", [1.0, 1e-4, 1e-8])
@pytest.mark.parametrize("L", [3, 4])
def test_solve_matches_sparse_direct_solve(stokes_mod, L, alpha, smoother):
    nu = 1 if smoother == "slsgs" else 2
    o = stokes_mod.StokesOracle(L, alpha, smoother=smoother, nu_pre=nu, nu_post=nu)
    f = o.rhs(inputs.stokes_vd_vortex(L, 3))
    x, it, rr, hist = o.solve(f, tol=1e-11, max_iter=300)
    assert rr <= 1e-11
    xd = bordered_direct(o, f)
    err = o.norm_L(o.normalize(x) - xd) / o.norm_L(xd)
    assert err < 1e-8, err
    assert hist[-1] < hist[0]


def load_table2():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            s, k, a, it = line.split()
            rows.append((s, int(k), float(a), int(it)))
    return rows


def test_table2_iteration_counts(stokes_mod):
    """Section 3 protocol in the natural order of Algorithm 2 (the order of x),
    W-cycle, coarsest h = 1/2: Table 2 for k = 4, 5 at alpha = 1 and 1e-6
    within 4 iterations (the paper states neither the mesh nor the cycle).  At
    alpha = 1e-12 the counts of this discretisation stay near their alpha = 1e-6
    values for LSGS and grow for NE and sLSGS, where the paper's fall with k:
    that column is not reproduced (a reading recorded with the design); only
    convergence is checked there."""
    for (s, k, a, it_paper) in load_table2():
        if k > 5:
            continue
        nu = 1 if s == "slsgs" else 2
        o = stokes_mod.StokesOracle(k, a, smoother=s, nu_pre=nu, nu_post=nu, lexicographic=True)
        x0 = np.random.default_rng(7).uniform(-1.0, 1.0, o.m())
        it = o.protocol_iterations(x0, 1e-6, 300)
        if a >= 1e-6:
            assert abs(it - it_paper) <= 4, (s, k, a, it, it_paper)
        else:
            assert 0 < it <= 100, (s, k, a, it)


def test_lsgs_halves_ne_and_is_robust(stokes_mod):
    """LSGS needs about half the NE iterations (section 3, Table 2) and its
    counts are bounded independently of h and alpha in [1e-6, 1]."""
    ne, ls = [], []
    for k in (3, 4, 5):
        for a in (1.0, 1e-3, 1e-6):
            x0 = np.random.default_rng(9).uniform(-1.0, 1.0, inputs.stokes_sizes(k)[2])
            ne.append(stokes_mod.StokesOracle(k, a, smoother="ne").protocol_iterations(x0, 1e-6, 300))
            ls.append(stokes_mod.StokesOracle(k, a, smoother="lsgs").protocol_iterations(x0, 1e-6, 300))
    assert max(ls) <= 18 and max(ne) <= 45
    assert np.mean(ls) < 0.6 * np.mean(ne)
