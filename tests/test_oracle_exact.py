"""Pins for the oracle's exact E-step, likelihood, responsibilities and M-step.

Each check reaches the value by a route other than the oracle's own: the Gaussian marginal
density of y_t (Eq. 1 integrated over z_t) through scipy's multivariate normal, the
matrix-determinant lemma on the N x N side, an LU-based inverse, brute force over all
cluster assignments, EM monotonicity (Sec. 2) and stationarity of the Q-function (Eq. 2)."""
import itertools

import numpy as np
import pytest
from scipy.stats import multivariate_normal

from oracle import cofem


def _problem(T=3, C=2, D=12, N=5, seed=0, beta=50.0):
    rng = np.random.default_rng(seed)
    Phi = [rng.standard_normal((N, D)) / np.sqrt(N) for _ in range(T)]
    y = [rng.standard_normal(N) for _ in range(T)]
    alpha = rng.uniform(0.2, 3.0, size=(C, D))
    pi = rng.dirichlet(np.ones(C))
    return Phi, y, alpha, pi, beta


def _marginal_logpdf(Phi_t, y_t, alpha_c, beta):
    """log p(y_t | alpha_c) = log N(y_t; 0, I/beta + Phi diag(1/alpha) Phi^T)  (Eq. 1)."""
    cov = np.eye(len(y_t)) / beta + (Phi_t / alpha_c) @ Phi_t.T
    return multivariate_normal(mean=np.zeros(len(y_t)), cov=cov).logpdf(y_t)


def test_exact_estep_mean_and_covariance():
    Phi, y, alpha, pi, beta = _problem()
    est = cofem.exact_estep(Phi, y, alpha, pi, beta)
    for t in range(3):
        for c in range(2):
            A = beta * Phi[t].T @ Phi[t] + np.diag(alpha[c])
            b0 = beta * Phi[t].T @ y[t]
            assert np.linalg.norm(A @ est["mu"][t, c] - b0) <= 1e-12 * np.linalg.norm(b0)
            Sig = np.linalg.inv(A)                  # LU-based, not the oracle's Cholesky
            np.testing.assert_allclose(est["s"][t, c], np.diag(Sig), rtol=1e-10)


def test_logdet_by_matrix_determinant_lemma():
    """log det A = sum log alpha + log det(I_N + beta Phi diag(alpha)^-1 Phi^T)."""
    Phi, y, alpha, pi, beta = _problem(N=4, D=9)
    est = cofem.exact_estep(Phi, y, alpha, pi, beta)
    for t in range(3):
        for c in range(2):
            M = np.eye(4) + beta * (Phi[t] / alpha[c]) @ Phi[t].T
            logdetA = np.sum(np.log(alpha[c])) + np.linalg.slogdet(M)[1]
            assert abs(est["logdet"][t, c] - (-logdetA)) <= 1e-10 * abs(logdetA)


def test_ell_is_twice_marginal_loglik_plus_task_constant():
    """Eq. 3's ell equals 2 log p(y|alpha) + N log 2pi - N log beta + beta ||y||^2."""
    Phi, y, alpha, pi, beta = _problem()
    est = cofem.exact_estep(Phi, y, alpha, pi, beta)
    for t in range(3):
        N = len(y[t])
        for c in range(2):
            lp = _marginal_logpdf(Phi[t], y[t], alpha[c], beta)
            want = 2 * lp + N * np.log(2 * np.pi) - N * np.log(beta) + beta * y[t] @ y[t]
            assert abs(est["ell"][t, c] - want) <= 1e-9 * max(1.0, abs(want))
            assert abs(lp - (0.5 * est["ell"][t, c] - cofem.task_const(y[t], beta))) < 1e-9


def test_responsibilities_are_bayes_posteriors():
    Phi, y, alpha, pi, beta = _problem(C=3)
    est = cofem.exact_estep(Phi, y, alpha, pi, beta)
    for t in range(3):
        lp = np.array([_marginal_logpdf(Phi[t], y[t], alpha[c], beta) for c in range(3)])
        w = np.log(pi) + lp
        post = np.exp(w - w.max())
        post /= post.sum()
        np.testing.assert_allclose(est["q"][t], post, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(est["q"].sum(axis=1), 1.0, atol=1e-15)


def test_mixture_likelihood_brute_force_over_assignments():
    """sum over all C^T assignments of prod_t pi_{a_t} p(y_t|alpha_{a_t}) = exp(T * L)."""
    T, C = 4, 3
    Phi, y, alpha, pi, beta = _problem(T=T, C=C, D=8, N=4)
    est = cofem.exact_estep(Phi, y, alpha, pi, beta)
    lp = np.array([[_marginal_logpdf(Phi[t], y[t], alpha[c], beta) for c in range(C)]
                   for t in range(T)])
    terms = []
    for a in itertools.product(range(C), repeat=T):
        terms.append(sum(np.log(pi[a[t]]) + lp[t, a[t]] for t in range(T)))
    terms = np.array(terms)
    brute = terms.max() + np.log(np.exp(terms - terms.max()).sum())
    assert abs(T * est["loglik"] - brute) <= 1e-9 * abs(brute)


def test_exact_em_is_monotone():
    """Sec. 2: every EM iteration does not decrease L(theta)."""
    Phi, y, alpha, pi, beta = _problem(T=4, C=2, D=16, N=6, seed=3, beta=200.0)
    out = cofem.em(Phi, y, pi, beta, 12, method="exact", alpha0=alpha)
    tr = out["loglik_trace"]
    assert np.all(np.diff(tr) >= -1e-9 * np.abs(tr[1:])), tr


def _Q(alpha_c, q_c, mu_c, s_c):
    """The alpha_c-dependent part of Eq. 2 for one cluster (q_c [T], mu_c and s_c [T, D])."""
    return float(np.sum(q_c[:, None] * (0.5 * np.log(alpha_c)[None, :]
                                         - 0.5 * alpha_c[None, :] * (mu_c ** 2 + s_c))))


def test_m_step_maximises_q_function():
    Phi, y, alpha, pi, beta = _problem(T=4, C=2, D=10, N=4, seed=5)
    est = cofem.exact_estep(Phi, y, alpha, pi, beta)
    new = cofem.m_step(est["q"], est["mu"], est["s"], alpha)
    for c in range(2):
        q0 = _Q(new[c], est["q"][:, c], est["mu"][:, c], est["s"][:, c])
        for d in range(10):
            for h in (1e-3, -1e-3):
                a = new[c].copy()
                a[d] *= (1 + h)
                assert _Q(a, est["q"][:, c], est["mu"][:, c], est["s"][:, c]) <= q0 + 1e-15


def test_m_step_clamps_and_empty_cluster():
    q = np.array([[1.0, 0.0], [1.0, 0.0]])
    mu = np.zeros((2, 2, 3))
    s = np.zeros((2, 2, 3))
    s[:, 0, 0] = 1e-30        # den ~ 0     -> alpha_max
    s[:, 0, 1] = -5.0         # negative s  -> term clipped to 0 -> alpha_max
    s[:, 0, 2] = 1e20         # huge den    -> alpha_min
    prev = np.full((2, 3), 7.0)
    new = cofem.m_step(q, mu, s, prev, alpha_min=1e-10, alpha_max=1e10)
    assert new[0, 0] == 1e10 and new[0, 1] == 1e10 and new[0, 2] == 1e-10
    np.testing.assert_array_equal(new[1], prev[1])      # zero responsibility keeps alpha


@pytest.mark.parametrize("C", [1])
def test_single_cluster_reduces_to_multitask_update(C):
    """C = 1 (the multi-task model the paper's Eq. 1 reduces to): q == 1 and the update is
    alpha_d = T / sum_t (mu_td^2 + Sigma_t,dd)."""
    Phi, y, alpha, pi, beta = _problem(T=3, C=1, D=7, N=3, seed=2)
    pi = np.array([1.0])
    est = cofem.exact_estep(Phi, y, alpha, pi, beta)
    np.testing.assert_array_equal(est["q"], 1.0)
    new = cofem.m_step(est["q"], est["mu"], est["s"], alpha)
    want = 3.0 / np.sum(est["mu"][:, 0] ** 2 + est["s"][:, 0], axis=0)
    np.testing.assert_allclose(new[0], want, rtol=1e-13)
