"""Pin for the adjoint gradient formulas used by the autograd wrapper.

For the loss L = 1/2 ||u - u_t||^2 of the control u = lambda / alpha (eq. (mp2)
and u = alpha^{-1} lambda), with A x = (M y_D, 0):
  dL/dy_D   = M z_y,                       A z = (0, (u - u_t) / alpha),
  dL/dalpha = -alpha^{-2} ((u - u_t) . lambda + z_lambda^T M lambda).
Checked here against central finite differences of dense solves built from the
oracle's matrices (independent of the formula)."""
import numpy as np
import pytest

from paper_1502_03917_gb300 import inputs


def dense_setup(oracle_mod, L, alpha):
    o = oracle_mod.Oracle(L, alpha)
    return o, o.scipy(L, "A").toarray(), o.scipy(L, "M").toarray()


def loss_and_grad(oracle_mod, L, alpha, yD, ut, grad=True):
    o, A, M = dense_setup(oracle_mod, L, alpha)
    n = M.shape[0]
    f = np.concatenate([M @ yD, np.zeros(n)])
    x = np.linalg.solve(A, f)
    lam = x[n:]
    u = lam / alpha
    r = u - ut
    loss = 0.5 * r @ r
    if not grad:
        return loss
    z = np.linalg.solve(A, np.concatenate([np.zeros(n), r / alpha]))
    g_yD = M @ z[:n]
    g_alpha = -(r @ lam + z[n:] @ (M @ lam)) / alpha ** 2
    return loss, g_yD, g_alpha


@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-4])
def test_adjoint_gradient_matches_finite_differences(oracle_mod, alpha):
    L = 3
    yD = inputs.yd_uniform(L, 4)
    ut = inputs.u_target(L, 3)
    loss, g_yD, g_alpha = loss_and_grad(oracle_mod, L, alpha, yD, ut)
    v = np.random.default_rng(9).standard_normal(yD.size)
    h = 1e-6
    fd = (loss_and_grad(oracle_mod, L, alpha, yD + h * v, ut, False) -
          loss_and_grad(oracle_mod, L, alpha, yD - h * v, ut, False)) / (2 * h)
    assert g_yD @ v == pytest.approx(fd, rel=1e-6)
    # derivative in log(alpha): dL/dlog(alpha) = alpha dL/dalpha
    fa = (loss_and_grad(oracle_mod, L, alpha * np.exp(h), yD, ut, False) -
          loss_and_grad(oracle_mod, L, alpha * np.exp(-h), yD, ut, False)) / (2 * h)
    assert alpha * g_alpha == pytest.approx(fa, rel=1e-6)


@pytest.mark.parametrize("alpha", [1.0, 1e-4])
def test_symmetric_adjoint_identity(oracle_mod, alpha):
    """The backward pass solves with A itself because A is symmetric: for any
    right-hand sides f, g the oracle's multigrid solutions satisfy
    g . A^{-1} f = f . A^{-1} g (to the solves' tolerance)."""
    L = 4
    o = oracle_mod.Oracle(L, alpha)
    rng = np.random.default_rng(21)
    n2 = 2 * o.nn()
    f, g = rng.standard_normal(n2), rng.standard_normal(n2)
    xf, _, rf, _ = o.solve(f, tol=1e-13, max_iter=400)
    xg, _, rg, _ = o.solve(g, tol=1e-13, max_iter=400)
    assert rf <= 1e-13 and rg <= 1e-13
    assert g @ xf == pytest.approx(f @ xg, rel=1e-9)
