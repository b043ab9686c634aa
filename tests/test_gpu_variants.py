"""GPU parity of the method variants against the oracle, through the C ABI: learned cluster
priors, probes shared across clusters and Jacobi-preconditioned CG (dense FP32, dense
BF16X3 tensor-core operator, Fourier operator, adjoint solve).

Tolerances as for the plain E-step: mu and s at norm-wise relative error <= 1e-4 per vector,
responsibilities at absolute error <= 1e-4 when the oracle replays the GPU's own CG
coefficients, hard assignments bit-exact, probes bit-exact."""
import numpy as np
import pytest

from oracle import cofem, philox
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import check_free_q, make_ctx, rel_err_rows, task_lists

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
Q_TOL = 1e-4


@pytest.fixture(scope="module")
def small():
    return synth.plain_small()


def _late_alpha(C, D, seed, lo=4.0, hi=6.0):
    """alpha as EM leaves it after some iterations: ~90% pruned entries with
    alpha = 10^U(lo, hi) above beta ||Phi e_d||^2, ~10% active ones with alpha = 10^U(-1, 1).
    Here the diagonal of A varies over decades, so the Jacobi preconditioner matters (plain
    CG runs to its step cap on it)."""
    rng = np.random.default_rng(seed)
    a = 10.0 ** rng.uniform(lo, hi, size=(C, D))
    act = rng.random((C, D)) < 0.1
    a[act] = 10.0 ** rng.uniform(-1.0, 1.0, size=int(act.sum()))
    return a.astype(np.float32)


_OUTS = dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, q=cmcs.OUT_Q, logdet=cmcs.OUT_LOGDET,
             ell=cmcs.OUT_ELL, steps=cmcs.OUT_STEPS, gamma=cmcs.OUT_GAMMA, xi=cmcs.OUT_XI,
             assign=cmcs.OUT_ASSIGN)


def _gpu_estep(ctx, alpha32, em_iter):
    ctx.set_alpha(alpha32, em_iter)
    ctx.estep()
    g = {k: ctx.read(v) for k, v in _OUTS.items()}
    g["summary"] = ctx.summary()
    return g


def _replay(P, Y, wl, g, o, alpha32, precond):
    """nu, ell and q the oracle forms from the GPU's CG coefficients and its refined means
    (with the preconditioner: Eq. 11 on the pcg coefficients minus sum_d log m_d)."""
    T, C = len(P), alpha32.shape[0]
    nu = np.zeros((T, C))
    ell = np.zeros((T, C))
    for t in range(T):
        b0 = cofem.rhs_mean(P[t], Y[t], wl.beta)
        for c in range(C):
            a = alpha32[c].astype(np.float64)
            nu[t, c] = cofem.logdet_estimate(g["gamma"][t, c].astype(np.float64),
                                             g["xi"][t, c].astype(np.float64),
                                             g["steps"][t, c, 1:], wl.D)
            if precond:
                nu[t, c] -= float(np.sum(np.log(cofem.jacobi_diag(P[t], wl.beta, a))))
            ell[t, c] = cofem.ell(nu[t, c], a, b0, o["mu"][t, c])
    return cofem.responsibilities(ell, wl.pi), ell, nu


def _check_pair(P, Y, wl, g, o, alpha32, precond, nu_rtol, soft=()):
    assert rel_err_rows(g["mu"], o["mu"]).max() <= REL_TOL
    assert rel_err_rows(g["s"], o["s"]).max() <= REL_TOL
    q_rep, ell_rep, nu_rep = _replay(P, Y, wl, g, o, alpha32, precond)
    assert np.max(np.abs(g["logdet"] - nu_rep) / np.abs(nu_rep)) <= nu_rtol
    assert np.max(np.abs(g["q"] - q_rep)) <= Q_TOL
    assert np.max(np.abs(g["logdet"] - o["logdet"]) / np.abs(o["logdet"])) <= 1e-4
    check_free_q(g["q"], o["q"], soft_tasks=soft)
    assert np.array_equal(g["assign"], np.argmax(o["q"], axis=1))


# ---- probes shared across clusters -------------------------------------------------------

def test_shared_probes_bit_exact_and_estep_parity(small):
    P, Y = task_lists(small)
    alpha = synth.uniform_alpha(small.C, small.D, seed=3)
    with make_ctx(small, refine_max=12, refine_tol=1e-6, probe_share=True) as ctx:
        pr = ctx.probes(2)
        g = _gpu_estep(ctx, alpha, 2)
    for t in range(small.T):
        ref = philox.probes(small.seed, 2, t, 0, small.C, small.K, small.D)
        for c in range(small.C):
            assert np.array_equal(pr[t, c].astype(np.float64), ref), (t, c)
    o = cofem.cofem_estep(P, Y, alpha.astype(np.float64), small.pi, small.beta, small.K,
                          small.seed, 2, small.cg_tol, small.cg_max_iter, refine_tol=1e-12,
                          refine_max=40, probe_share=True)
    # tasks 0 and 3: largest q 0.979 and 0.970
    _check_pair(P, Y, small, g, o, alpha, False, 1e-9, soft=(0, 3))


# ---- learned priors ----------------------------------------------------------------------

def test_learned_pi_matches_oracle_update(small):
    alpha = synth.uniform_alpha(small.C, small.D, seed=4)
    with make_ctx(small, refine_max=8, refine_tol=1e-6, learn_pi=True) as ctx:
        np.testing.assert_allclose(ctx.read(cmcs.OUT_PI), small.pi, rtol=1e-15)
        ctx.set_alpha(alpha, 0)
        ctx.em_iter(1)
        q1 = ctx.read(cmcs.OUT_Q)
        pi1 = ctx.read(cmcs.OUT_PI)
        ctx.estep()                                  # uses the learned priors
        q2, ell2 = ctx.read(cmcs.OUT_Q), ctx.read(cmcs.OUT_ELL)
    np.testing.assert_allclose(pi1, cofem.pi_update(q1), rtol=1e-13, atol=1e-300)
    assert abs(pi1.sum() - 1.0) <= 1e-14
    np.testing.assert_allclose(q2, cofem.responsibilities(ell2, pi1), atol=1e-12)


def test_fixed_pi_is_left_alone(small):
    alpha = synth.uniform_alpha(small.C, small.D, seed=4)
    with make_ctx(small, refine_max=4, refine_tol=1e-6) as ctx:
        ctx.set_alpha(alpha, 0)
        ctx.em_iter(2)
        np.testing.assert_array_equal(ctx.read(cmcs.OUT_PI), small.pi)


# ---- Jacobi-preconditioned CG ----------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_precond_estep_parity(small, precision):
    P, Y = task_lists(small)
    alpha = _late_alpha(small.C, small.D, seed=5)
    with make_ctx(small, refine_max=12, refine_tol=1e-6, precond=True,
                  precision=precision) as ctx:
        g = _gpu_estep(ctx, alpha, 1)
    with make_ctx(small, refine_max=12, refine_tol=1e-6, precision=precision) as ctx:
        plain = _gpu_estep(ctx, alpha, 1)
    o = cofem.cofem_estep(P, Y, alpha.astype(np.float64), small.pi, small.beta, small.K,
                          small.seed, 1, small.cg_tol, small.cg_max_iter, refine_tol=1e-12,
                          refine_max=40, precond=True)
    # sum_d log m_d: FP64 on both sides, the column norms rounded to FP32 once on the GPU
    _check_pair(P, Y, small, g, o, alpha, True, 1e-6)
    assert g["summary"]["refine_diverged"] == 0
    # the preconditioned first solve needs fewer steps on this alpha
    assert g["summary"]["cg_steps_mean"] < plain["summary"]["cg_steps_mean"]


def test_precond_fourier_estep_parity():
    wl = synth.fourier_small()
    P = [wl.phi_real(t) for t in range(wl.T)]
    Y = [wl.y_real(t) for t in range(wl.T)]
    alpha = _late_alpha(wl.C, wl.D, seed=6, lo=2.0)
    with cmcs.Context.from_fourier(wl, device=True, refine_max=16, refine_tol=1e-6,
                                   precond=True) as ctx:
        g = _gpu_estep(ctx, alpha, 2)
    o = cofem.cofem_estep(P, Y, alpha.astype(np.float64), wl.pi, wl.beta, wl.K, wl.seed, 2,
                          wl.cg_tol, wl.cg_max_iter, refine_tol=1e-12, refine_max=40,
                          precond=True)
    _check_pair(P, Y, wl, g, o, alpha, True, 1e-6)


def test_precond_adjoint_matches_exact():
    import torch
    wl = synth.make_workload("adjoint", 2, 2, 64, (20, 40), nnz=6, sigma=0.05, beta=100.0, K=4,
                             cg_tol=1e-7, cg_max_iter=200, seed=31)
    alpha = _late_alpha(2, 64, seed=7, lo=2.0)
    w = np.random.default_rng(8).standard_normal((2, 2, 64)).astype(np.float32)
    with cmcs.Context(torch.from_numpy(wl.Phi).cuda(), torch.from_numpy(wl.y).cuda(), wl.N,
                      C=wl.C, K=wl.K, beta=wl.beta, cg_tol=wl.cg_tol, cg_max_iter=wl.cg_max_iter,
                      refine_max=16, refine_tol=1e-7, precond=True) as ctx:
        ctx.set_alpha(alpha, 0)
        ctx.estep()
        dy, da, _ = ctx.adjoint(torch.from_numpy(w).cuda(), with_phi=False)
    dy, da = dy.cpu().numpy(), da.cpu().numpy()
    ref_dy, ref_da = [], np.zeros((2, 64))
    for t in range(wl.T):
        Pt, yt = wl.phi(t).astype(np.float64), wl.yt(t).astype(np.float64)
        dyt = np.zeros(Pt.shape[0])
        for c in range(wl.C):
            r = cofem.mean_adjoint(Pt, yt, wl.beta, alpha[c].astype(np.float64),
                                   w[t, c].astype(np.float64))
            dyt += r["dy"]
            ref_da[c] += r["dalpha"]
        ref_dy.append(dyt)
    ref_dy = np.concatenate(ref_dy)
    assert np.linalg.norm(dy - ref_dy) <= 1e-4 * np.linalg.norm(ref_dy)
    assert rel_err_rows(da, ref_da).max() <= 1e-4


def test_em_parity_with_all_variants(small):
    """Ten EM iterations with learned priors, shared probes and the Jacobi preconditioner on
    both sides, from the library's own alpha draw: alpha, pi, q, assignments and the
    reconstructions against the oracle's EM loop."""
    P, Y = task_lists(small)
    with make_ctx(small, refine_max=12, refine_tol=1e-6, learn_pi=True, probe_share=True,
                  precond=True) as ctx:
        ctx.em_iter(small.em_iters)
        a_g, pi_g = ctx.read(cmcs.OUT_ALPHA), ctx.read(cmcs.OUT_PI)
        q_g, asg = ctx.read(cmcs.OUT_Q), ctx.read(cmcs.OUT_ASSIGN)
        recon = ctx.read(cmcs.OUT_RECON)
        summ = ctx.summary()
    o = cofem.em(P, Y, small.pi, small.beta, small.em_iters, K=small.K, seed=small.seed,
                 tol=small.cg_tol, max_iter=small.cg_max_iter, C=small.C, D=small.D,
                 refine_tol=1e-12, refine_max=40, learn_pi=True, probe_share=True,
                 precond=True)
    assert summ["refine_diverged"] == 0
    assert np.array_equal(asg, o["assign"])
    err = check_free_q(q_g, o["last"]["q"])
    # pi = mean_t q: its error is at most the mean of the per-task q errors (plus rounding)
    assert np.max(np.abs(pi_g - o["pi"])) <= err.mean() + 1e-12
    # learned priors can empty a cluster (here all tasks end in one); the alpha of a cluster
    # with next to no responsibility is a ratio of sums weighted by ~1e-10, so alpha is
    # compared for the occupied clusters
    occupied = o["last"]["q"].sum(axis=0) > 0.5
    assert occupied.any()
    assert rel_err_rows(a_g[occupied], o["alpha"][occupied]).max() <= REL_TOL
    assert rel_err_rows(recon, o["recon"]).max() <= REL_TOL


def test_warm_start_em_parity(small):
    """Ten EM iterations whose mean systems start from the previous E-step's means, on both
    sides: alpha, q, assignments and reconstructions against the oracle's EM loop; the mean
    systems of the last E-step take fewer CG steps than from x_1 = 0."""
    P, Y = task_lists(small)
    steps = {}
    for warm in (False, True):
        with make_ctx(small, refine_max=12, refine_tol=1e-6, warm_start=warm) as ctx:
            ctx.em_iter(small.em_iters)
            steps[warm] = ctx.read(cmcs.OUT_STEPS)[:, :, 0]
            if warm:
                a_g, q_g = ctx.read(cmcs.OUT_ALPHA), ctx.read(cmcs.OUT_Q)
                asg, recon = ctx.read(cmcs.OUT_ASSIGN), ctx.read(cmcs.OUT_RECON)
                summ = ctx.summary()
    o = cofem.em(P, Y, small.pi, small.beta, small.em_iters, K=small.K, seed=small.seed,
                 tol=small.cg_tol, max_iter=small.cg_max_iter, C=small.C, D=small.D,
                 refine_tol=1e-12, refine_max=40, warm_start=True)
    assert summ["refine_diverged"] == 0
    assert np.array_equal(asg, o["assign"])
    check_free_q(q_g, o["last"]["q"], soft_tasks=(2,))      # task 2: q = (0.992, 0.008)
    assert rel_err_rows(a_g, o["alpha"]).max() <= REL_TOL
    assert rel_err_rows(recon, o["recon"]).max() <= REL_TOL
    assert np.all(steps[True] <= steps[False]) and np.any(steps[True] < steps[False])


@pytest.mark.parametrize("wl_name, soft", [("fourier-small", ()),
                                           # largest q 0.817, 0.703 and 0.533
                                           ("fourier-2k", (0, 1, 3))])
def test_all_variants_on_the_fourier_operator(wl_name, soft):
    """Three EM iterations with every variant on (learned priors, shared probes, Jacobi,
    warm start) on the Fourier operator, single-CTA (D = 256) and four-step (D = 2000) paths,
    against the oracle's EM loop on the dense real-stacked matrices."""
    wl = synth.WORKLOADS[wl_name]()
    n = 3
    kw = dict(learn_pi=True, probe_share=True, precond=True, warm_start=True)
    with cmcs.Context.from_fourier(wl, device=True, refine_max=16, refine_tol=1e-6, **kw) as ctx:
        ctx.em_iter(n)
        a_g, pi_g = ctx.read(cmcs.OUT_ALPHA), ctx.read(cmcs.OUT_PI)
        q_g, asg = ctx.read(cmcs.OUT_Q), ctx.read(cmcs.OUT_ASSIGN)
        summ = ctx.summary()
    P = [wl.phi_real(t) for t in range(wl.T)]
    Y = [wl.y_real(t) for t in range(wl.T)]
    o = cofem.em(P, Y, wl.pi, wl.beta, n, K=wl.K, seed=wl.seed, tol=wl.cg_tol,
                 max_iter=wl.cg_max_iter, C=wl.C, D=wl.D, refine_tol=1e-12, refine_max=40, **kw)
    assert summ["refine_diverged"] == 0
    assert np.array_equal(asg, o["assign"])
    err = check_free_q(q_g, o["last"]["q"], soft_tasks=soft)
    assert np.max(np.abs(pi_g - o["pi"])) <= err.mean() + 1e-12
    occupied = o["last"]["q"].sum(axis=0) > 0.5
    assert rel_err_rows(a_g[occupied], o["alpha"][occupied]).max() <= REL_TOL
