"""The Fourier operator of Sec. 4 through its four-step path (lengths D = 2^a 5^b that are not
powers of two, and powers of two beyond one CTA): the FP32 operator, the FP64 refinement
residual, b0 and E-steps against the oracle.

At D = 2000 the oracle uses the dense real-stacked matrix (arithmetic without any FFT); at
D = 16384 and D = 100,000 (the largest length of the paper's timings) it uses its FFT-form
operator, pinned against the dense matrix at small D.  Bounds as for the single-CTA path:
operator 1e-5, residual 2e-7 (FP32 rounding of an FP64 result), b0 1e-6, mu and s 1e-4."""
import numpy as np
import pytest

from oracle import cofem
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import rel_err_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wl2k():
    return synth.fourier_2k()


def _ctx(wl, **kw):
    return cmcs.Context.from_fourier(wl, device=True, **kw)


def _late_alpha(C, D, seed, lo=2.0, hi=6.0):
    rng = np.random.default_rng(seed)
    a = 10.0 ** rng.uniform(lo, hi, size=(C, D))
    act = rng.random((C, D)) < 0.1
    a[act] = 10.0 ** rng.uniform(-1.0, 1.0, size=int(act.sum()))
    return a.astype(np.float32)


def _check_operator(wl, dense: bool):
    R = wl.C * (wl.K + 1)
    V = np.random.default_rng(3).standard_normal((wl.T, R, wl.D)).astype(np.float32)
    with _ctx(wl) as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        b0 = ctx.read(cmcs.OUT_B0)
        Z = ctx.apply(V)
        Rz = ctx.apply(V, accurate=True, B=np.zeros_like(V))     # 0 - A V in FP64
    for t in range(wl.T):
        P = wl.phi_real(t) if dense else None
        for j in range(R):
            c = j // (wl.K + 1)
            v = V[t, j].astype(np.float64)
            ref = (cofem.apply_A(P, wl.beta, alpha[c], v) if dense
                   else cofem.apply_A_fourier(wl.mask[t], wl.beta, alpha[c], v))
            assert rel_err_rows(Z[t, j], ref) <= 1e-5, (t, j)
            assert rel_err_rows(-Rz[t, j], ref) <= 2e-7, (t, j)
        ref_b0 = cofem.rhs_mean_fourier(wl.mask[t], wl.yt(t), wl.beta)
        assert rel_err_rows(b0[t], ref_b0) <= 1e-6, t


def test_operator_residual_b0_at_2000(wl2k):
    _check_operator(wl2k, dense=True)


@pytest.mark.parametrize("D,N", [(16384, 4096), (100000, 25000)])
def test_operator_residual_b0_at_large_lengths(D, N):
    wl = synth.make_fourier("f-large", 2, 1, D, N, K=3, cg_tol=1e-5, cg_max_iter=50, seed=4)
    _check_operator(wl, dense=False)


def _replay(wl, g, o, alpha32, precond):
    nu = np.zeros((wl.T, wl.C))
    ell = np.zeros((wl.T, wl.C))
    for t in range(wl.T):
        P = wl.phi_real(t)
        b0 = cofem.rhs_mean(P, wl.y_real(t), wl.beta)
        for c in range(wl.C):
            a = alpha32[c].astype(np.float64)
            nu[t, c] = cofem.logdet_estimate(g["gamma"][t, c].astype(np.float64),
                                             g["xi"][t, c].astype(np.float64),
                                             g["steps"][t, c, 1:], wl.D)
            if precond:
                nu[t, c] -= float(np.sum(np.log(cofem.jacobi_diag(P, wl.beta, a))))
            ell[t, c] = cofem.ell(nu[t, c], a, b0, o["mu"][t, c])
    return cofem.responsibilities(ell, wl.pi), nu


@pytest.mark.parametrize("precond", [False, True])
def test_estep_parity_at_2000(wl2k, precond):
    wl = wl2k
    alpha = _late_alpha(wl.C, wl.D, seed=5) if precond else synth.uniform_alpha(wl.C, wl.D, seed=3)
    with _ctx(wl, refine_max=16, refine_tol=1e-6, precond=precond) as ctx:
        ctx.set_alpha(alpha, 2)
        ctx.estep()
        g = {k: ctx.read(v) for k, v in dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, q=cmcs.OUT_Q,
                                              logdet=cmcs.OUT_LOGDET, steps=cmcs.OUT_STEPS,
                                              gamma=cmcs.OUT_GAMMA, xi=cmcs.OUT_XI,
                                              assign=cmcs.OUT_ASSIGN).items()}
        summ = ctx.summary()
    P = [wl.phi_real(t) for t in range(wl.T)]
    Y = [wl.y_real(t) for t in range(wl.T)]
    o = cofem.cofem_estep(P, Y, alpha.astype(np.float64), wl.pi, wl.beta, wl.K, wl.seed, 2,
                          wl.cg_tol, wl.cg_max_iter, refine_tol=1e-12, refine_max=40,
                          precond=precond)
    assert summ["refine_diverged"] == 0
    assert rel_err_rows(g["mu"], o["mu"]).max() <= 1e-4
    assert rel_err_rows(g["s"], o["s"]).max() <= 1e-4
    q_rep, nu_rep = _replay(wl, g, o, alpha, precond)
    assert np.max(np.abs(g["logdet"] - nu_rep) / np.abs(nu_rep)) <= 1e-6
    assert np.max(np.abs(g["q"] - q_rep)) <= 1e-4
    assert np.array_equal(g["assign"], np.argmax(o["q"], axis=1))


@pytest.mark.parametrize("em_first,precond", [(False, False), (True, True)])
def test_estep_sampled_pair_at_100000(em_first, precond):
    """D = 100,000, N = 25,000, K = 15, U = 50 (Sec. 4's setting at the paper's largest
    length), two tasks and two clusters; one (task, cluster) pair against the oracle's
    FFT-form E-step on that pair.  The first E-step (alpha from its Uniform(0, 1) draw) runs
    plain CG; the E-step after one M-step (alpha up to its clamp 1e10) runs the Jacobi-
    preconditioned form, which its FP32 refinement needs at this length."""
    wl = synth.make_fourier("f-100k", 2, 2, 100000, 25000, K=15, cg_tol=1e-5, cg_max_iter=50,
                            seed=6)
    with _ctx(wl, refine_max=8, refine_tol=1e-5, precond=precond) as ctx:
        if em_first:
            ctx.em_iter(1)
        alpha = ctx.read(cmcs.OUT_ALPHA)
        it = ctx.summary()["em_iters_done"]
        ctx.set_alpha(alpha, it)
        ctx.estep()
        mu, s, q = ctx.read(cmcs.OUT_MU), ctx.read(cmcs.OUT_S), ctx.read(cmcs.OUT_Q)
        summ = ctx.summary()
    assert summ["refine_diverged"] == 0
    np.testing.assert_allclose(q.sum(axis=1), 1.0, atol=1e-12)
    t, c = 1, 1
    o = cofem.cofem_estep([cofem.FourierSensing(wl.mask[t])], [wl.y_real(t)],
                          alpha[c:c + 1].astype(np.float64), np.array([1.0]), wl.beta, wl.K,
                          wl.seed, it, wl.cg_tol, wl.cg_max_iter, tasks=[t], clusters=[c],
                          C_total=wl.C, refine_tol=1e-10, refine_max=20, precond=precond)
    assert rel_err_rows(mu[t, c], o["mu"][0, 0]) <= 1e-4
    assert rel_err_rows(s[t, c], o["s"][0, 0]) <= 1e-4


def test_unsupported_lengths_are_rejected():
    # 3 divides D: neither a power of two nor 2^a 5^b
    wl = synth.make_fourier("f-bad", 1, 1, 3 * 1024, 768, K=1, seed=7)
    with pytest.raises(cmcs.CmcsError) as ei:
        _ctx(wl)
    assert ei.value.status == cmcs.ERR_UNSUPPORTED


def test_fourstep_path_forced_at_a_power_of_two(monkeypatch):
    """CMCS_DFT_FOURSTEP=1 sends D = 256 (otherwise one CTA per pair) through the four-step
    path: operator, residual, b0 and the E-step match the oracle there too."""
    monkeypatch.setenv("CMCS_DFT_FOURSTEP", "1")
    wl = synth.fourier_small()
    _check_operator(wl, dense=True)
    alpha = synth.uniform_alpha(wl.C, wl.D, seed=3)
    with _ctx(wl, refine_max=16, refine_tol=1e-6) as ctx:
        ctx.set_alpha(alpha, 2)
        ctx.estep()
        mu, s = ctx.read(cmcs.OUT_MU), ctx.read(cmcs.OUT_S)
    P = [wl.phi_real(t) for t in range(wl.T)]
    Y = [wl.y_real(t) for t in range(wl.T)]
    o = cofem.cofem_estep(P, Y, alpha.astype(np.float64), wl.pi, wl.beta, wl.K, wl.seed, 2,
                          wl.cg_tol, wl.cg_max_iter, refine_tol=1e-12, refine_max=40)
    assert rel_err_rows(mu, o["mu"]).max() <= 1e-4
    assert rel_err_rows(s, o["s"]).max() <= 1e-4
