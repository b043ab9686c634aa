"""The structured sensing operator of Sec. 4 (Phi_t = Omega_t F, a subsampled unitary DFT, real
signals, complex measurements) through cmcs_create_dft, against the oracle: the FFT operator
and its FP64 residual against the dense real-stacked matrix, b0, a full E-step on a small
Fourier workload, and a sampled pair at D = 8192.

The oracle runs the same method on the real matrix [Re Phi_t; Im Phi_t] (2 N_t x D) with
y_t stacked the same way, whose normal equations are those of the reading
A = beta Re(Phi^H Phi) + diag(alpha), b0 = beta Re(Phi^H y)."""
import numpy as np
import pytest

from oracle import cofem, philox
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import rel_err_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    return synth.fourier_small()


def _ctx(wl, **kw):
    return cmcs.Context.from_fourier(wl, device=True, **kw)


def _dense(wl):
    return ([wl.phi_real(t) for t in range(wl.T)], [wl.y_real(t) for t in range(wl.T)])


def _replay_q(wl, g, o, alpha32):
    """q, nu and ell the oracle computes from the GPU's own CG coefficients (Eqs. 9-11) and
    the oracle's refined means."""
    nu = np.zeros((wl.T, wl.C))
    ell = np.zeros((wl.T, wl.C))
    for t in range(wl.T):
        b0 = cofem.rhs_mean(wl.phi_real(t), wl.y_real(t), wl.beta)
        for c in range(wl.C):
            nu[t, c] = cofem.logdet_estimate(g["gamma"][t, c].astype(np.float64),
                                             g["xi"][t, c].astype(np.float64),
                                             g["steps"][t, c, 1:], wl.D)
            ell[t, c] = cofem.ell(nu[t, c], alpha32[c].astype(np.float64), b0, o["mu"][t, c])
    return cofem.responsibilities(ell, wl.pi), nu, ell


def test_fourier_operator_and_residual_match_oracle(small):
    wl = small
    R = wl.C * (wl.K + 1)
    V = np.random.default_rng(3).standard_normal((wl.T, R, wl.D)).astype(np.float32)
    with _ctx(wl) as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        Z = ctx.apply(V)
        Rz = ctx.apply(V, accurate=True, B=np.zeros_like(V))     # 0 - A V in FP64
    for t in range(wl.T):
        P = wl.phi_real(t)
        for j in range(R):
            c = j // (wl.K + 1)
            ref = cofem.apply_A(P, wl.beta, alpha[c], V[t, j].astype(np.float64))
            assert rel_err_rows(Z[t, j], ref) <= 1e-5, (t, j)
            assert rel_err_rows(-Rz[t, j], ref) <= 2e-7, (t, j)


def test_fourier_b0_matches_oracle(small):
    wl = small
    with _ctx(wl) as ctx:
        b0 = ctx.read(cmcs.OUT_B0)
    for t in range(wl.T):
        ref = cofem.rhs_mean_fourier(wl.mask[t], wl.yt(t), wl.beta)
        assert rel_err_rows(b0[t], ref) <= 1e-6


def test_fourier_estep_parity(small):
    wl = small
    P, Y = _dense(wl)
    alpha = synth.uniform_alpha(wl.C, wl.D, seed=3)
    with _ctx(wl, refine_max=16, refine_tol=1e-6) as ctx:
        ctx.set_alpha(alpha, 2)
        ctx.estep()
        g = {k: ctx.read(v) for k, v in dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, q=cmcs.OUT_Q,
                                              logdet=cmcs.OUT_LOGDET, ell=cmcs.OUT_ELL,
                                              steps=cmcs.OUT_STEPS, gamma=cmcs.OUT_GAMMA,
                                              xi=cmcs.OUT_XI, assign=cmcs.OUT_ASSIGN).items()}
        summ = ctx.summary()
    o = cofem.cofem_estep(P, Y, alpha.astype(np.float64), wl.pi, wl.beta, wl.K, wl.seed, 2,
                          wl.cg_tol, wl.cg_max_iter, refine_tol=1e-12, refine_max=40)
    assert summ["refine_diverged"] == 0
    assert rel_err_rows(g["mu"], o["mu"]).max() <= 1e-4
    assert rel_err_rows(g["s"], o["s"]).max() <= 1e-4
    q_rep, nu_rep, ell_rep = _replay_q(wl, g, o, alpha)
    np.testing.assert_allclose(g["logdet"], nu_rep, rtol=1e-9)
    assert np.max(np.abs(g["q"] - q_rep)) <= 1e-4
    assert np.array_equal(g["assign"], np.argmax(o["q"], axis=1))
    np.testing.assert_allclose(g["logdet"], o["logdet"], rtol=1e-4)


def test_fourier_workload_sampled_pair():
    """The D = 8192 Fourier workload (T = 40, N = 2048, K = 15, U = 50): one EM iteration,
    then an E-step; a sampled (task, cluster) pair against exact solves on the dense
    real-stacked matrix."""
    wl = synth.fourier()
    with _ctx(wl, refine_max=8, refine_tol=1e-5) as ctx:
        ctx.em_iter(1)
        alpha = ctx.read(cmcs.OUT_ALPHA)
        it = ctx.summary()["em_iters_done"]
        ctx.estep()
        mu = ctx.read(cmcs.OUT_MU)
        s = ctx.read(cmcs.OUT_S)
        q = ctx.read(cmcs.OUT_Q)
    np.testing.assert_allclose(q.sum(axis=1), 1.0, atol=1e-12)
    t, c = 17, 2
    P = wl.phi_real(t)
    y = wl.y_real(t)
    pk = philox.probes(wl.seed, it, t, c, wl.C, wl.K, wl.D)
    B = np.concatenate([cofem.rhs_mean(P, y, wl.beta)[:, None], pk.T], axis=1)
    X = cofem.solve_exact(P, wl.beta, alpha[c].astype(np.float64), B)
    assert rel_err_rows(mu[t, c], X[:, 0]) <= 1e-4
    assert rel_err_rows(s[t, c], np.mean(pk.T * X[:, 1:], axis=1)) <= 1e-4


def test_fourier_context_rejects_dense_only_calls(small):
    with _ctx(small) as ctx:
        ctx.estep()
        with pytest.raises(cmcs.CmcsError):
            ctx.adjoint(np.zeros((small.T, small.C, small.D), np.float32))
