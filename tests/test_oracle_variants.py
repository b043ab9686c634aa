"""Pins for the oracle's E-step and M-step variants: learned cluster priors, probes shared
across clusters and Jacobi-preconditioned CG.

Routes independent of the oracle's own formulas: a numerical optimiser over the simplex and
EM monotonicity (learned pi, Sec. 2); exact equality of the estimates of two identical
clusters and the variance of their difference over many seeds (shared probes); dense solves,
exhaustive averaging over all 2^D Rademacher probes, plain CG on the explicitly scaled
matrix and the case M = c I (Jacobi preconditioning)."""
import itertools

import numpy as np
from scipy.optimize import minimize

from oracle import cofem, philox


def _problem(T=3, C=2, D=12, N=5, seed=0, beta=50.0):
    rng = np.random.default_rng(seed)
    Phi = [rng.standard_normal((N, D)) / np.sqrt(N) for _ in range(T)]
    y = [rng.standard_normal(N) for _ in range(T)]
    alpha = rng.uniform(0.2, 3.0, size=(C, D))
    pi = rng.dirichlet(np.ones(C))
    return Phi, y, alpha, pi, beta


# ---- learned pi ------------------------------------------------------------------------

def test_pi_update_maximises_expected_log_prior():
    """pi_update(q) maximises sum_tc q_tc log pi_c over the simplex: compare with a generic
    optimiser on the softmax parameterisation."""
    rng = np.random.default_rng(0)
    q = rng.dirichlet(np.ones(4), size=7)
    pi = cofem.pi_update(q)
    assert abs(pi.sum() - 1.0) <= 1e-15

    def neg(v):
        p = np.exp(v - v.max())
        p /= p.sum()
        return -float(np.sum(q * np.log(p)[None, :]))

    res = minimize(neg, np.zeros(4), method="Nelder-Mead",
                   options=dict(xatol=1e-10, fatol=1e-14, maxiter=20000))
    p = np.exp(res.x - res.x.max())
    np.testing.assert_allclose(pi, p / p.sum(), atol=1e-5)
    assert neg(np.log(pi)) <= res.fun + 1e-12


def test_pi_update_keeps_empty_cluster_finite():
    q = np.array([[1.0, 0.0, 0.0], [0.25, 0.75, 0.0]])
    pi = cofem.pi_update(q)
    assert np.all(np.isfinite(np.log(pi)))
    np.testing.assert_allclose(pi[:2], [0.625, 0.375], rtol=1e-15)
    assert 0.0 < pi[2] <= 1e-299


def test_exact_em_with_learned_pi_is_monotone():
    """Sec. 2: with pi learned too, every EM iteration still does not decrease L(theta)."""
    Phi, y, alpha, pi, beta = _problem(T=5, C=3, D=14, N=6, seed=3, beta=200.0)
    out = cofem.em(Phi, y, pi, beta, 12, method="exact", alpha0=alpha, learn_pi=True)
    tr = out["loglik_trace"]
    assert np.all(np.diff(tr) >= -1e-9 * np.abs(tr[1:])), tr
    np.testing.assert_allclose(out["pi"], cofem.pi_update(out["last"]["q"]), rtol=1e-15)


# ---- probes shared across clusters -------------------------------------------------------

def test_shared_probes_make_identical_clusters_agree_exactly():
    """Two clusters with the same alpha: with shared probes their s and nu are identical;
    with independent probes they are not."""
    Phi, y, alpha, pi, beta = _problem(T=2, C=2, D=16, N=7, seed=4)
    alpha[1] = alpha[0]
    kw = dict(K=6, seed=5, em_iter=0, tol=1e-12, max_iter=40)
    sh = cofem.cofem_estep(Phi, y, alpha, pi, beta, probe_share=True, **kw)
    ind = cofem.cofem_estep(Phi, y, alpha, pi, beta, **kw)
    np.testing.assert_array_equal(sh["s"][:, 0], sh["s"][:, 1])
    np.testing.assert_array_equal(sh["logdet"][:, 0], sh["logdet"][:, 1])
    assert np.abs(ind["logdet"][:, 0] - ind["logdet"][:, 1]).max() > 1e-6
    # cluster 0 draws the same probes either way
    np.testing.assert_array_equal(sh["logdet"][:, 0], ind["logdet"][:, 0])
    p0 = philox.probes(5, 0, 1, 0, 2, 6, 16)
    np.testing.assert_array_equal(p0, philox.probes(5, 0, 1, 0, 2, 6, 16))


def test_shared_probes_reduce_variance_of_ell_differences():
    """Common random numbers: for two nearby alphas the variance over seeds of
    nu_t1 - nu_t0 is much smaller with shared probes."""
    Phi, y, alpha, pi, beta = _problem(T=1, C=2, D=20, N=8, seed=6)
    alpha[1] = alpha[0] * 1.05
    diffs = {False: [], True: []}
    for seed in range(40):
        for share in (False, True):
            e = cofem.cofem_estep(Phi, y, alpha, pi, beta, 4, seed, 0, 1e-12, 60,
                                  probe_share=share)
            diffs[share].append(e["logdet"][0, 1] - e["logdet"][0, 0])
    v_ind, v_sh = np.var(diffs[False]), np.var(diffs[True])
    assert v_sh < 0.05 * v_ind, (v_sh, v_ind)


# ---- Jacobi-preconditioned CG ----------------------------------------------------------

def _spread_problem(D=30, N=12, seed=0, beta=1e3):
    rng = np.random.default_rng(seed)
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    alpha = 10.0 ** rng.uniform(-2, 6, size=D)           # pruned and active coefficients
    A = beta * Phi.T @ Phi + np.diag(alpha)
    op = lambda V, idx=None: cofem.apply_A(Phi, beta, alpha, V)
    return Phi, alpha, beta, A, op


def test_pcg_matches_dense_solve_and_needs_fewer_steps():
    Phi, alpha, beta, A, op = _spread_problem()
    B = np.random.default_rng(1).standard_normal((30, 3))
    m = cofem.jacobi_diag(Phi, beta, alpha)
    np.testing.assert_allclose(m, np.diag(A), rtol=1e-14)
    r = cofem.pcg(op, B, 1.0 / m, 1e-12, 200)
    np.testing.assert_allclose(r.x, np.linalg.solve(A, B), rtol=1e-8)
    plain = cofem.cg(op, B, 1e-12, 200)
    assert r.steps.max() < plain.steps.max()


def test_pcg_coefficients_are_cg_on_the_scaled_system():
    """gamma_u and xi_u of pcg equal those of plain CG on Ah = M^-1/2 A M^-1/2 with
    bh = M^-1/2 b, the matrix formed explicitly."""
    Phi, alpha, beta, A, op = _spread_problem(D=20, N=9, seed=2)
    m = np.diag(A)
    S = np.diag(1.0 / np.sqrt(m))
    Ah = S @ A @ S
    b = np.random.default_rng(3).standard_normal((20, 2))
    r = cofem.pcg(op, b, 1.0 / m, 0.0, 12)
    h = cofem.cg(lambda V, idx=None: Ah @ V, S @ b, 0.0, 12)
    np.testing.assert_allclose(r.gamma, h.gamma, rtol=1e-9)
    np.testing.assert_allclose(r.xi, h.xi, rtol=1e-9)
    np.testing.assert_allclose(r.x, S @ h.x, rtol=1e-9, atol=1e-14)


def test_pcg_exhaustive_probes_give_exact_diagonal_and_logdet():
    """With every Rademacher probe and U = D, the preconditioned estimates are exact:
    s = diag(Sigma) and nu = log det Sigma (the sum_d log m_d term restores log det M)."""
    D, N = 8, 5
    rng = np.random.default_rng(4)
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    y = rng.standard_normal(N)
    alpha = 10.0 ** rng.uniform(-1, 3, size=(1, D))
    beta = 30.0
    allp = np.array(list(itertools.product([1.0, -1.0], repeat=D)))
    est = cofem.cofem_estep([Phi], [y], alpha, np.array([1.0]), beta, len(allp), 0, 0,
                            0.0, D, probe_fn=lambda t, c: allp, precond=True)
    A = beta * Phi.T @ Phi + np.diag(alpha[0])
    Sig = np.linalg.inv(A)
    np.testing.assert_allclose(est["s"][0, 0], np.diag(Sig), rtol=1e-9)
    ld = np.linalg.slogdet(Sig)[1]
    assert abs(est["logdet"][0, 0] - ld) <= 1e-9 * abs(ld)
    np.testing.assert_allclose(est["mu"][0, 0], np.linalg.solve(A, beta * Phi.T @ y), rtol=1e-9)


def test_pcg_with_scalar_preconditioner_equals_plain_estimates():
    """M = c I (orthogonal Phi columns of equal norm, constant alpha): the preconditioned
    E-step gives the plain E-step's s and nu for the same probes and step counts."""
    D = 16
    Q, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((D, D)))
    Phi = 0.7 * Q                                          # columns of norm 0.7
    y = np.random.default_rng(6).standard_normal(D)
    alpha = np.full((1, D), 0.4)
    kw = dict(K=5, seed=7, em_iter=0, tol=1e-13, max_iter=40)
    a = cofem.cofem_estep([Phi], [y], alpha, np.array([1.0]), 3.0, **kw)
    b = cofem.cofem_estep([Phi], [y], alpha, np.array([1.0]), 3.0, precond=True, **kw)
    np.testing.assert_allclose(b["s"], a["s"], rtol=1e-9)
    np.testing.assert_allclose(b["logdet"], a["logdet"], rtol=1e-9)
    np.testing.assert_allclose(b["mu"], a["mu"], rtol=1e-9)
    np.testing.assert_array_equal(b["steps"], a["steps"])


def test_pcg_refinement_reaches_direct_solve():
    Phi, alpha, beta, A, op = _spread_problem(D=40, N=15, seed=8, beta=1e4)
    B = np.random.default_rng(7).standard_normal((40, 2))
    minv = 1.0 / np.diag(A)
    Xs = np.linalg.solve(A, B)
    r = cofem.pcg(op, B, minv, 1e-5, 60)
    assert np.linalg.norm(r.x - Xs) > 1e-9 * np.linalg.norm(Xs)     # PCG alone is not there
    X, sweeps = cofem.refine(op, B, r.x, 1e-5, 60, 1e-12, 30, minv=minv)
    assert np.linalg.norm(X - Xs) <= 1e-9 * np.linalg.norm(Xs)
    assert sweeps.max() >= 1


# ---- warm-started mean systems -----------------------------------------------------------

def test_warm_start_from_exact_means_takes_no_step():
    Phi, y, alpha, pi, beta = _problem(T=2, C=2, D=16, N=7, seed=9)
    kw = dict(K=3, seed=1, em_iter=0, tol=1e-8, max_iter=60)
    for pc in (False, True):
        ex = cofem.exact_estep(Phi, y, alpha, pi, beta)
        w = cofem.cofem_estep(Phi, y, alpha, pi, beta, mu_init=ex["mu"], precond=pc, **kw)
        assert np.all(w["steps"][:, :, 0] == 0)
        np.testing.assert_allclose(w["mu"], ex["mu"], rtol=1e-12)


def test_warm_start_reaches_the_same_solution_with_fewer_steps():
    """From a nearby start (the exact means perturbed by 1e-3) the mean systems reach the
    same converged means in fewer steps; the probe systems are untouched."""
    Phi, y, alpha, pi, beta = _problem(T=2, C=2, D=40, N=15, seed=10, beta=1e3)
    alpha = 10.0 ** np.random.default_rng(11).uniform(-1, 2, size=alpha.shape)
    kw = dict(K=4, seed=2, em_iter=1, tol=1e-10, max_iter=200)
    ex = cofem.exact_estep(Phi, y, alpha, pi, beta)
    start = ex["mu"] * (1 + 1e-3 * np.random.default_rng(12).standard_normal(ex["mu"].shape))
    for pc in (False, True):
        cold = cofem.cofem_estep(Phi, y, alpha, pi, beta, precond=pc, **kw)
        warm = cofem.cofem_estep(Phi, y, alpha, pi, beta, mu_init=start, precond=pc, **kw)
        # both stop at ||r|| <= 1e-10 ||b0||: errors of order kappa * 1e-10 (kappa ~ 1e4 here)
        for e in (warm, cold):
            assert np.linalg.norm(e["mu"] - ex["mu"]) <= 1e-5 * np.linalg.norm(ex["mu"])
        assert np.all(warm["steps"][:, :, 0] < cold["steps"][:, :, 0])
        np.testing.assert_array_equal(warm["steps"][:, :, 1:], cold["steps"][:, :, 1:])
        # the probe systems run the same solves (the batched products' order of summation
        # may differ with the set of active columns)
        np.testing.assert_allclose(warm["s"], cold["s"], rtol=1e-10)
        np.testing.assert_allclose(warm["logdet"], cold["logdet"], rtol=1e-12)


def test_exact_em_with_warm_start_matches_cold_em():
    Phi, y, alpha, pi, beta = _problem(T=3, C=2, D=14, N=6, seed=13, beta=200.0)
    kw = dict(K=8, seed=3, tol=1e-12, max_iter=100, alpha0=alpha)
    cold = cofem.em(Phi, y, pi, beta, 4, **kw)
    warm = cofem.em(Phi, y, pi, beta, 4, warm_start=True, **kw)
    np.testing.assert_allclose(warm["alpha"], cold["alpha"], rtol=1e-8)
    np.testing.assert_allclose(warm["last"]["q"], cold["last"]["q"], atol=1e-10)
