"""Pins for the oracle's exact solve and the adjoint of the posterior means (Eq. 3), each
against something other than the function's own arithmetic: the diagonal special case in
closed form, the oracle's CG with refinement (Alg. 1, a different algorithm), and central
finite differences of the loss."""
import numpy as np
import pytest

from oracle import cofem

BETA = 50.0


def _problem(D, N, seed):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((N, D)) / np.sqrt(N)
    y = rng.standard_normal(N)
    alpha = rng.uniform(0.2, 3.0, size=D)
    return P, y, alpha


def test_solve_exact_diagonal_closed_form():
    """Phi = I (N = D): A = diag(beta + alpha), so Sigma B = B / (beta + alpha)."""
    D = 12
    rng = np.random.default_rng(1)
    alpha = rng.uniform(0.1, 5.0, size=D)
    B = rng.standard_normal((D, 3))
    X = cofem.solve_exact(np.eye(D), BETA, alpha, B)
    np.testing.assert_allclose(X, B / (BETA + alpha)[:, None], rtol=1e-13)


def test_solve_exact_matches_refined_cg():
    P, y, alpha = _problem(D=40, N=28, seed=2)
    B = np.random.default_rng(3).standard_normal((40, 4))
    op = lambda V, idx: cofem.apply_A(P, BETA, alpha, V)
    X0 = cofem.cg(op, B, 1e-10, 400).x
    X, _ = cofem.refine(op, B, X0, 1e-10, 400, 1e-14, 20)
    Xe = cofem.solve_exact(P, BETA, alpha, B)
    assert np.linalg.norm(X - Xe) <= 1e-9 * np.linalg.norm(Xe)
    # and it solves the system: the residual is at rounding level
    R = B - cofem.apply_A(P, BETA, alpha, Xe)
    assert np.linalg.norm(R) <= 1e-11 * np.linalg.norm(B)


def test_mean_adjoint_diagonal_closed_form():
    """Phi = I: mu_d = beta y_d / (beta + alpha_d), so dL/dy_d = g_d beta / (beta + alpha_d) and
    dL/dalpha_d = -g_d beta y_d / (beta + alpha_d)^2."""
    D = 10
    rng = np.random.default_rng(4)
    y = rng.standard_normal(D)
    alpha = rng.uniform(0.1, 5.0, size=D)
    g = rng.standard_normal(D)
    a = cofem.mean_adjoint(np.eye(D), y, BETA, alpha, g)
    np.testing.assert_allclose(a["mu"], BETA * y / (BETA + alpha), rtol=1e-13)
    np.testing.assert_allclose(a["dy"], g * BETA / (BETA + alpha), rtol=1e-12)
    np.testing.assert_allclose(a["dalpha"], -g * BETA * y / (BETA + alpha) ** 2, rtol=1e-12)


@pytest.mark.parametrize("shape", [(24, 16), (16, 30)])
def test_mean_adjoint_matches_finite_differences(shape):
    """Central differences of L = g^T mu(Phi, y, alpha) along random directions, every input
    at once and each input alone (so a wrong sign or a transposed term in any one fails)."""
    D, N = shape
    P, y, alpha = _problem(D, N, seed=5 + D)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(D)
    a = cofem.mean_adjoint(P, y, BETA, alpha, g)
    loss = lambda P_, y_, al_: float(g @ cofem.solve_exact(P_, BETA, al_, cofem.rhs_mean(P_, y_, BETA)))
    h = 1e-6
    for which in ("all", "Phi", "y", "alpha"):
        for _ in range(3):
            vP = rng.standard_normal(P.shape) if which in ("all", "Phi") else np.zeros_like(P)
            vy = rng.standard_normal(N) if which in ("all", "y") else np.zeros(N)
            va = rng.standard_normal(D) if which in ("all", "alpha") else np.zeros(D)
            fd = (loss(P + h * vP, y + h * vy, alpha + h * va) -
                  loss(P - h * vP, y - h * vy, alpha - h * va)) / (2 * h)
            terms = [np.sum(a["dPhi"] * vP), np.sum(a["dy"] * vy), np.sum(a["dalpha"] * va)]
            ad = float(np.sum(terms))
            assert abs(ad - fd) <= 1e-7 * max(1.0, float(np.sum(np.abs(terms)))), (which, ad, fd)
