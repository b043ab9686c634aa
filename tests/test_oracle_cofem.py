"""Pins for the oracle's covariance-free E-step: CG (Alg. 1), the Lanczos matrix (Eq. 9), the
log-det quadrature (Eqs. 10-11), the diagonal estimator (Eq. 4) and refinement.

Routes independent of the oracle: dense solves and eigendecompositions of A, Lanczos/CG
identities (Sec. 3.2), exhaustive averaging over all 2^D Rademacher probes (unbiasedness,
Sec. 3.1-3.2), the diagonal special case Phi = I, the closed-form variance of the diagonal
estimator, and agreement with exact EM as K grows."""
import itertools

import numpy as np

from oracle import cofem, philox


def _spd_problem(D=10, N=6, seed=0, beta=20.0):
    rng = np.random.default_rng(seed)
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    alpha = rng.uniform(0.5, 2.0, size=D)
    A = beta * Phi.T @ Phi + np.diag(alpha)
    op = lambda V, idx=None: cofem.apply_A(Phi, beta, alpha, V)
    return Phi, alpha, beta, A, op


def test_cg_matches_dense_solve():
    Phi, alpha, beta, A, op = _spd_problem(D=30, N=12)
    B = np.random.default_rng(1).standard_normal((30, 3))
    res = cofem.cg(op, B, 1e-13, 200)
    np.testing.assert_allclose(res.x, np.linalg.solve(A, B), rtol=1e-9, atol=1e-12)
    assert np.all(res.rel_resid <= 1e-13)


def test_cg_stops_at_tolerance_and_cap():
    Phi, alpha, beta, A, op = _spd_problem(D=40, N=20)
    b = np.random.default_rng(2).standard_normal((40, 1))
    r = cofem.cg(op, b, 1e-4, 500)
    assert r.rel_resid[0] <= 1e-4
    # the step before the last had not yet converged
    r2 = cofem.cg(op, b, 0.0, int(r.steps[0]) - 1)
    assert r2.rel_resid[0] > 1e-4
    capped = cofem.cg(op, b, 0.0, 3)
    assert capped.steps[0] == 3


def test_cg_replay_step_counts():
    Phi, alpha, beta, A, op = _spd_problem(D=20, N=8)
    B = np.random.default_rng(3).standard_normal((20, 3))
    r = cofem.cg(op, B, 0.0, 50, steps=np.array([2, 5, 9]))
    assert list(r.steps) == [2, 5, 9]


def test_lanczos_first_entry_is_rayleigh_quotient():
    """||p||^2 * G_11 = p^T A p, since the first Lanczos vector is p / ||p||."""
    Phi, alpha, beta, A, op = _spd_problem()
    p = philox.probes(0, 0, 0, 0, 1, 1, 10)[0]
    r = cofem.cg(op, p[:, None], 0.0, 6)
    G = cofem.lanczos_tridiag(r.gamma[0], r.xi[0], 6)
    assert abs(10 * G[0, 0] - p @ A @ p) <= 1e-12 * abs(p @ A @ p)


def test_lanczos_inverse_entry_is_cg_quadrature():
    """CG as Gauss quadrature: ||p||^2 (G_U^-1)_11 = p^T x_{U+1} for every U."""
    Phi, alpha, beta, A, op = _spd_problem(D=12, N=7)
    p = philox.probes(1, 0, 0, 0, 1, 1, 12)[0]
    for U in (1, 2, 4, 7):
        r = cofem.cg(op, p[:, None], 0.0, U)
        G = cofem.lanczos_tridiag(r.gamma[0], r.xi[0], U)
        lhs = 12 * np.linalg.inv(G)[0, 0]
        assert abs(lhs - p @ r.x[:, 0]) <= 1e-10 * abs(lhs)


def test_lanczos_eigenvalues_and_full_quadrature():
    """With U = D steps the Lanczos matrix is similar to A, and D sum_u S_u1^2 log lambda_u
    equals p^T log(A) p (Eq. 10)."""
    Phi, alpha, beta, A, op = _spd_problem(D=8, N=8, beta=2.0)
    p = philox.probes(2, 0, 0, 0, 1, 1, 8)[0]
    r = cofem.cg(op, p[:, None], 0.0, 8)
    assert r.steps[0] == 8
    G = cofem.lanczos_tridiag(r.gamma[0], r.xi[0], 8)
    np.testing.assert_allclose(np.linalg.eigvalsh(G), np.linalg.eigvalsh(A), rtol=1e-9)
    lam, V = np.linalg.eigh(A)
    logA = (V * np.log(lam)) @ V.T
    quad = cofem.lanczos_log_quadrature(r.gamma[0], r.xi[0], 8, 8.0)
    assert abs(quad - p @ logA @ p) <= 1e-9 * abs(p @ logA @ p)


def test_off_diagonal_sign_is_immaterial():
    """Flipping the sign of the off-diagonal of Eq. 9 leaves lambda and S_u1^2 unchanged."""
    Phi, alpha, beta, A, op = _spd_problem(D=9, N=5)
    p = philox.probes(3, 0, 0, 0, 1, 1, 9)[0]
    r = cofem.cg(op, p[:, None], 0.0, 6)
    G = cofem.lanczos_tridiag(r.gamma[0], r.xi[0], 6)
    F = np.diag([(-1) ** i for i in range(6)])
    l1, V1 = np.linalg.eigh(G)
    l2, V2 = np.linalg.eigh(F @ G @ F)
    np.testing.assert_allclose(l1, l2, rtol=1e-12)
    np.testing.assert_allclose(V1[0] ** 2, V2[0] ** 2, atol=1e-12)


def test_exhaustive_probes_give_exact_diagonal_and_logdet():
    """Averaging over all 2^D Rademacher probes, s equals diag(Sigma) exactly (Eq. 4 is
    unbiased) and with U = D steps the estimate of Eq. 11 equals log det Sigma."""
    D, N = 8, 5
    rng = np.random.default_rng(4)
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    y = rng.standard_normal(N)
    alpha = rng.uniform(0.5, 2.0, size=(1, D))
    beta = 3.0
    allp = np.array(list(itertools.product([1.0, -1.0], repeat=D)))
    est = cofem.cofem_estep([Phi], [y], alpha, np.array([1.0]), beta, len(allp), 0, 0,
                            0.0, D, probe_fn=lambda t, c: allp)
    A = beta * Phi.T @ Phi + np.diag(alpha[0])
    Sig = np.linalg.inv(A)
    np.testing.assert_allclose(est["s"][0, 0], np.diag(Sig), rtol=1e-9)
    assert abs(est["logdet"][0, 0] - np.linalg.slogdet(Sig)[1]) <= 1e-9 * abs(np.linalg.slogdet(Sig)[1])
    np.testing.assert_allclose(est["mu"][0, 0], np.linalg.solve(A, beta * Phi.T @ y), rtol=1e-9)


def test_diagonal_special_case():
    """Phi = I (N = D): A = diag(beta + alpha), so mu = beta y / (beta + alpha),
    Sigma_dd = 1 / (beta + alpha); the diagonal estimate is exact for any K and the log-det
    estimate is exact once CG has converged."""
    D = 16
    rng = np.random.default_rng(5)
    y = rng.standard_normal(D)
    alpha = rng.uniform(0.1, 4.0, size=(1, D))
    alpha[0, :4] = alpha[0, 4]                        # repeated eigenvalues
    beta = 2.5
    est = cofem.cofem_estep([np.eye(D)], [y], alpha, np.array([1.0]), beta, 3, 11, 0,
                            1e-14, 50)
    np.testing.assert_allclose(est["mu"][0, 0], beta * y / (beta + alpha[0]), rtol=1e-10)
    np.testing.assert_allclose(est["s"][0, 0], 1 / (beta + alpha[0]), rtol=1e-10)
    want = -np.sum(np.log(beta + alpha[0]))
    assert abs(est["logdet"][0, 0] - want) <= 1e-10 * abs(want)
    assert est["steps"][0, 0, 1:].max() <= D - 3      # at most #distinct eigenvalues steps


def test_diagonal_estimator_variance_closed_form():
    """Var(s_d) = (1/K) sum_{j != d} Sigma_dj^2 for Rademacher probes; the empirical error over
    many seeds matches it (z-score) and scales as K^-1/2."""
    D, N, beta = 10, 6, 4.0
    rng = np.random.default_rng(6)
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    y = rng.standard_normal(N)
    alpha = rng.uniform(0.5, 2.0, size=(1, D))
    Sig = np.linalg.inv(beta * Phi.T @ Phi + np.diag(alpha[0]))
    var1 = (np.sum(Sig ** 2, axis=1) - np.diag(Sig) ** 2)
    for K in (4, 64):
        errs = []
        for seed in range(60):
            est = cofem.cofem_estep([Phi], [y], alpha, np.array([1.0]), beta, K, seed, 0,
                                    1e-13, 60)
            errs.append(est["s"][0, 0] - np.diag(Sig))
        errs = np.array(errs)
        z = errs.mean(axis=0) / np.sqrt(var1 / K / len(errs))
        assert np.all(np.abs(z) < 4.5), z
        ratio = errs.var(axis=0) / (var1 / K)
        assert 0.5 < ratio.mean() < 1.6, ratio


def test_refinement_reaches_direct_solve():
    Phi, alpha, beta, A, op = _spd_problem(D=40, N=15, beta=1e4)
    alpha[:5] = 1e-3                                   # ill-conditioned (op sees this too)
    A = beta * Phi.T @ Phi + np.diag(alpha)
    B = np.random.default_rng(7).standard_normal((40, 2))
    r = cofem.cg(op, B, 1e-8, 25)
    assert np.abs(r.x - np.linalg.solve(A, B)).max() > 1e-6   # CG alone is not there yet
    X, sweeps = cofem.refine(op, B, r.x, 1e-8, 25, 1e-12, 30)
    np.testing.assert_allclose(X, np.linalg.solve(A, B), rtol=1e-9)
    assert sweeps.max() >= 1


def test_cofem_approaches_exact_em_as_k_grows():
    """With converged solves and many probes the CoFEM E-step agrees with the exact one."""
    rng = np.random.default_rng(8)
    T, C, D, N, beta = 3, 2, 24, 10, 100.0
    Phi = [rng.standard_normal((N, D)) / np.sqrt(N) for _ in range(T)]
    y = [rng.standard_normal(N) for _ in range(T)]
    alpha = rng.uniform(0.3, 3.0, size=(C, D))
    pi = np.array([0.5, 0.5])
    ex = cofem.exact_estep(Phi, y, alpha, pi, beta)
    errs = []
    for K in (16, 1024):
        co = cofem.cofem_estep(Phi, y, alpha, pi, beta, K, 1, 0, 1e-13, 200)
        np.testing.assert_allclose(co["mu"], ex["mu"], rtol=1e-8, atol=1e-10)
        errs.append((np.abs(co["s"] - ex["s"]).max(), np.abs(co["logdet"] - ex["logdet"]).max()))
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]
    assert errs[1][1] < 0.05 * np.abs(ex["logdet"]).max()


def test_logdet_estimate_meets_the_cited_bound_at_its_K_and_U():
    """Sec. 3.2's cited result: with K >= 24/eps^2 log(2/eta) probes and
    U >= sqrt(kappa)/4 log(O(kappa)/(eps sqrt(kappa))) CG steps, Eq. 11 is within
    eps |log det Sigma| with probability > 1 - eta.  kappa = 100, eps = eta = 0.1 (so K = 7190
    and, taking the O(kappa) constant as kappa, U = 12 < D = 30); over 20 independent probe
    sets the estimate must be within the bound at least 1 - eta of the time."""
    D, kappa, eps, eta = 30, 100.0, 0.1, 0.1
    K = int(np.ceil(24.0 / eps ** 2 * np.log(2.0 / eta)))
    U = int(np.ceil(np.sqrt(kappa) / 4.0 * np.log(kappa / (eps * np.sqrt(kappa)))))
    assert (K, U) == (7190, 12)
    rng = np.random.default_rng(14)
    Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
    lam = np.geomspace(1.0, kappa, D)
    A = (Q * lam) @ Q.T
    logdet_sigma = -float(np.sum(np.log(lam)))
    hits = 0
    for seed in range(20):
        P = np.sign(np.random.default_rng(100 + seed).standard_normal((D, K)))
        res = cofem.cg(lambda V, idx=None: A @ V, P, 0.0, U, steps=np.full(K, U))
        nu = cofem.logdet_estimate(res.gamma, res.xi, res.steps, D)
        hits += abs(nu - logdet_sigma) <= eps * abs(logdet_sigma)
    assert hits >= (1.0 - eta) * 20


def test_cofem_tracks_exact_em_iteration_by_iteration():
    """Sec. 4 (Fig. 1(d)): CoFEM's approximations leave EM's rate of convergence unchanged.
    With converged solves and many probes, the log-likelihood seen by every E-step and the
    alpha trajectory follow exact EM's, and the final assignments agree."""
    rng = np.random.default_rng(15)
    T, C, D, N, beta = 4, 2, 24, 10, 100.0
    Phi = [rng.standard_normal((N, D)) / np.sqrt(N) for _ in range(T)]
    y = [rng.standard_normal(N) for _ in range(T)]
    alpha0 = rng.uniform(0.3, 3.0, size=(C, D))
    pi = np.array([0.5, 0.5])
    n = 6
    ex = cofem.em(Phi, y, pi, beta, n, method="exact", alpha0=alpha0)
    co = cofem.em(Phi, y, pi, beta, n, K=2048, seed=4, tol=1e-12, max_iter=200, alpha0=alpha0)
    lx, lc = ex["loglik_trace"], co["loglik_trace"]
    # measured: within 1% at every iteration, per-iteration gains within 5.3% of the total
    # gain, alpha within a factor e^0.42 (the estimators' noise at D = 24, K = 2048)
    assert np.max(np.abs(lc - lx)) <= 0.02 * np.max(np.abs(lx))
    gain_x, gain_c = np.diff(lx), np.diff(lc)
    assert np.max(np.abs(gain_c - gain_x)) <= 0.1 * (lx[-1] - lx[0])
    assert lc[-1] - lc[0] >= 0.9 * (lx[-1] - lx[0])
    for ax, ac in zip(ex["alphas"], co["alphas"]):
        assert np.max(np.abs(np.log(ac) - np.log(ax))) <= 0.6
    np.testing.assert_array_equal(co["assign"], ex["assign"])
