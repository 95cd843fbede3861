"""Pins for the oracle's discretisation (section 1, eq. (mp2); section 2).

Each check compares the oracle with something it does not compute itself:
hand-derived P1 stencils, exact integrals of linear functions, a brute-force
quadrature assembly from the global hat-function formula, the Galerkin
identities of nested P1 spaces, and the closed-form spectrum of the pencil
(A_k, Q_k) behind the stability estimate (a1).
"""
import numpy as np
import pytest
import scipy.linalg as sla


def dense(o, level, which):
    return o.scipy(level, which).toarray()


# ---------------------------------------------------------------- helpers --
def hat(n, a, b, x, y):
    """Global P1 hat function of node (a, b) on the '/' mesh (cells split by
    the SW-NE diagonal): 1 - max(|u|, |v|, |u - v|), clipped at zero, with
    (u, v) the offset from the node in units of h."""
    u = x * n - a
    v = y * n - b
    return max(0.0, 1.0 - max(abs(u), abs(v), abs(u - v)))


def brute_force_mass_stiffness(n):
    """Assemble M and the bare stiffness matrix by quadrature: the edge-midpoint
    rule is exact for the quadratic phi_a*phi_b; gradients by central
    differences at the centroid (exact for functions linear on the triangle)."""
    h = 1.0 / n
    nn = (n + 1) ** 2
    M = np.zeros((nn, nn))
    K = np.zeros((nn, nn))
    nodes = [(i, j) for j in range(n + 1) for i in range(n + 1)]
    for cj in range(n):
        for ci in range(n):
            for tri in (((ci, cj), (ci + 1, cj), (ci + 1, cj + 1)), ((ci, cj), (ci + 1, cj + 1), (ci, cj + 1))):
                P = np.array(tri, float) * h
                area = 0.5 * h * h
                mids = [(P[a] + P[(a + 1) % 3]) / 2 for a in range(3)]
                cen = P.mean(axis=0)
                d = 1e-4 * h
                vals, grads = {}, {}
                for (a, b) in nodes:
                    vals[(a, b)] = [hat(n, a, b, m[0], m[1]) for m in mids]
                    gx = (hat(n, a, b, cen[0] + d, cen[1]) - hat(n, a, b, cen[0] - d, cen[1])) / (2 * d)
                    gy = (hat(n, a, b, cen[0], cen[1] + d) - hat(n, a, b, cen[0], cen[1] - d)) / (2 * d)
                    grads[(a, b)] = (gx, gy)
                for p, (a, b) in enumerate(nodes):
                    for q, (c, e) in enumerate(nodes):
                        M[(b * (n + 1) + a), (e * (n + 1) + c)] += area / 3 * sum(
                            vals[(a, b)][k] * vals[(c, e)][k] for k in range(3))
                        K[(b * (n + 1) + a), (e * (n + 1) + c)] += area * (
                            grads[(a, b)][0] * grads[(c, e)][0] + grads[(a, b)][1] * grads[(c, e)][1])
    return M, K


def nodal(L, fn):
    n = 1 << L
    t = np.arange(n + 1) / n
    X, Y = np.meshgrid(t, t, indexing="xy")
    return fn(X.ravel(), Y.ravel())


# ------------------------------------------------------------------ tests --
@pytest.mark.parametrize("n_level", [1, 2])
def test_brute_force_assembly(oracle_mod, n_level):
    o = oracle_mod.Oracle(n_level, 1e-2, kvariant=1)
    o0 = oracle_mod.Oracle(n_level, 1e-2, kvariant=0)
    Mb, Kb = brute_force_mass_stiffness(1 << n_level)
    M, K = dense(o, n_level, "M"), dense(o, n_level, "K")
    np.testing.assert_allclose(M, Mb, rtol=0, atol=1e-13)
    np.testing.assert_allclose(K, Kb, rtol=0, atol=1e-9)
    # kvariant 0: K is the matrix of (grad y, grad v) + (y, v)
    np.testing.assert_allclose(dense(o0, n_level, "K"), Kb + Mb, rtol=0, atol=1e-9)


def test_interior_stencils(oracle_mod):
    L = 4
    n = 1 << L
    h2 = (1.0 / n) ** 2
    o = oracle_mod.Oracle(L, 1.0, kvariant=1)
    M, K = o.scipy(L, "M"), o.scipy(L, "K")
    i, j = 7, 9
    p = j * (n + 1) + i
    off = {(0, 0): None, (1, 0): None, (-1, 0): None, (0, 1): None, (0, -1): None, (1, 1): None, (-1, -1): None}
    for (di, dj) in off:
        q = (j + dj) * (n + 1) + (i + di)
        m_expect = h2 / 2 if (di, dj) == (0, 0) else h2 / 12
        k_expect = 4.0 if (di, dj) == (0, 0) else (-1.0 if abs(di) + abs(dj) == 1 else 0.0)
        assert M[p, q] == pytest.approx(m_expect, rel=1e-14)
        assert K[p, q] == pytest.approx(k_expect, abs=1e-14)
    assert M.getrow(p).nnz == 7
    # corners: (0,0) and (n,n) touch two triangles, (n,0) and (0,n) touch one
    for (ci, cj, ntri) in [(0, 0, 2), (n, n, 2), (n, 0, 1), (0, n, 1)]:
        q = cj * (n + 1) + ci
        assert M[q, q] == pytest.approx(ntri * h2 / 12, rel=1e-14)


@pytest.mark.parametrize("L", [2, 4, 6])
def test_integrals_of_linear_functions(oracle_mod, L):
    """v^T M w = int u w and v^T K v = int |grad u|^2 (+ int u^2) exactly for
    linear u, w, which P1 reproduces."""
    o1 = oracle_mod.Oracle(L, 1.0, kvariant=1)
    o0 = oracle_mod.Oracle(L, 1.0, kvariant=0)
    a, b, c = 0.3, -1.7, 2.2
    d, e, g = -0.4, 0.9, 0.5
    u = nodal(L, lambda X, Y: a + b * X + c * Y)
    w = nodal(L, lambda X, Y: d + e * X + g * Y)
    M, Kd, K = o1.scipy(L, "M"), o1.scipy(L, "K"), o0.scipy(L, "K")
    # int_0^1 int_0^1 (a+bx+cy)(d+ex+gy)
    exact_uw = a * d + (a * e + b * d) / 2 + (a * g + c * d) / 2 + b * e / 3 + c * g / 3 + (b * g + c * e) / 4
    assert u @ (M @ w) == pytest.approx(exact_uw, rel=1e-12)
    assert np.ones_like(u) @ (M @ np.ones_like(u)) == pytest.approx(1.0, rel=1e-13)
    assert u @ (Kd @ u) == pytest.approx(b * b + c * c, rel=1e-12)
    np.testing.assert_allclose(Kd @ np.ones_like(u), 0.0, atol=1e-12)
    assert u @ (K @ u) == pytest.approx(b * b + c * c + u @ (M @ u), rel=1e-12)


@pytest.mark.parametrize("L", [3, 5])
def test_block_structure_and_symmetry(oracle_mod, L):
    alpha = 3e-3
    o = oracle_mod.Oracle(L, alpha)
    A = o.scipy(L, "A")
    M, K = o.scipy(L, "M"), o.scipy(L, "K")
    n = o.nn()
    Ad = A.toarray()
    np.testing.assert_array_equal(Ad, Ad.T)  # symmetric, bitwise
    np.testing.assert_allclose(Ad[:n, :n], M.toarray(), rtol=0, atol=0)
    np.testing.assert_allclose(Ad[:n, n:], K.toarray(), rtol=0, atol=0)
    np.testing.assert_allclose(Ad[n:, :n], K.toarray(), rtol=0, atol=0)
    np.testing.assert_allclose(Ad[n:, n:], -M.toarray() / alpha, rtol=1e-15, atol=0)
    # L = diag(Q_k)
    Ld = o.ldiag()
    np.testing.assert_allclose(Ld[:n], M.diagonal() + np.sqrt(alpha) * K.diagonal(), rtol=1e-15)
    np.testing.assert_allclose(Ld[n:], M.diagonal() / alpha + K.diagonal() / np.sqrt(alpha), rtol=1e-15)
    # N_ii = sum_j A_ij^2 / L_jj
    np.testing.assert_allclose(o.ndiag(), (Ad ** 2) @ (1.0 / Ld), rtol=1e-13)


def a1_spectrum_ok(A, M, K, alpha, rtol=1e-9):
    """Generalized eigenvalues of (A, Q) must be exactly +-sqrt(1+s^2)/(1+s)
    with s = sqrt(alpha) mu, mu in spec(K, M): the closed form behind eq. (a1)
    (|eig| in [2^-1/2, 1] for every h and alpha)."""
    n = M.shape[0]
    if not np.array_equal(A, A.T):
        return False, None
    W = M + np.sqrt(alpha) * K
    Q = np.block([[W, np.zeros((n, n))], [np.zeros((n, n)), W / alpha]])
    theta = np.sort(sla.eigh(A, Q, eigvals_only=True))
    mu = sla.eigh(K, M, eigvals_only=True)
    s = np.sqrt(alpha) * mu
    mag = np.sqrt(1 + s * s) / (1 + s)
    expect = np.sort(np.concatenate([mag, -mag]))
    return np.allclose(theta, expect, rtol=rtol, atol=1e-12), theta


@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-6, 1e-8])
@pytest.mark.parametrize("L", [2, 3, 4])
def test_a1_closed_form_spectrum(oracle_mod, L, alpha):
    o = oracle_mod.Oracle(L, alpha)
    A, M, K = dense(o, L, "A"), dense(o, L, "M"), dense(o, L, "K")
    ok, theta = a1_spectrum_ok(A, M, K, alpha)
    assert ok
    assert np.abs(theta).min() >= 2 ** -0.5 - 1e-10
    assert np.abs(theta).max() <= 1 + 1e-10


def test_a1_pin_rejects_planted_mistakes(oracle_mod):
    """The spectrum pin is sharp: a flipped sign, a dropped alpha or a
    transposed off-diagonal block or a dropped mass term in K each fail it."""
    L, alpha = 3, 1e-2
    o = oracle_mod.Oracle(L, alpha)
    A, M, K = dense(o, L, "A"), dense(o, L, "M"), dense(o, L, "K")
    n = M.shape[0]
    bad_sign = A.copy()
    bad_sign[n:, n:] *= -1
    bad_alpha = A.copy()
    bad_alpha[n:, n:] *= alpha
    bad_block = A.copy()
    bad_block[:n, n:] = M
    dropped = A.copy()
    dropped[:n, n:] -= M
    dropped[n:, :n] -= M
    for bad in (bad_sign, bad_alpha, bad_block, dropped):
        assert not a1_spectrum_ok(bad, M, K, alpha)[0]


@pytest.mark.parametrize("alpha", [1.0, 1e-4, 1e-8])
def test_tau_bound(oracle_mod, alpha):
    """rho(tau L^-1 A L^-1 A) stays below 2 for tau = 0.4 (section 2: the NE
    smoother's damping must keep the spectral radius away from 2)."""
    for L in (2, 3, 4):
        o = oracle_mod.Oracle(L, alpha)
        A = dense(o, L, "A")
        Li = 1.0 / o.ldiag()
        T = 0.4 * (Li[:, None] * A) @ (Li[:, None] * A)
        rho = np.max(np.abs(np.linalg.eigvals(T)))
        assert rho < 1.8


@pytest.mark.parametrize("L", [2, 3, 5])
def test_galerkin_nested_spaces(oracle_mod, L):
    """P^T M_k P = M_{k-1} and P^T K_k P = K_{k-1}: the canonical embedding of
    nested P1 spaces (section 2)."""
    o = oracle_mod.Oracle(L, 0.1)
    P = o.scipy(L, "P")
    for which in ("M", "K"):
        fine, coarse = o.scipy(L, which), o.scipy(L - 1, which)
        np.testing.assert_allclose((P.T @ fine @ P).toarray(), coarse.toarray(), rtol=0, atol=1e-13)
    # P reproduces linear functions: prolongated coarse nodal values equal fine nodal values
    u = lambda X, Y: 0.7 - 1.3 * X + 2.1 * Y
    np.testing.assert_allclose(P @ nodal(L - 1, u), nodal(L, u), atol=1e-14)
    # every row of P sums to one (constants are reproduced), weights are 1 or 1/2
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-15)
    assert set(np.round(P.data, 12)) <= {0.5, 1.0}
