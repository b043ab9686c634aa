"""Parity at the full sizes of the precision workload (T=16, C=4, D=16384, N=4096, K=64:
R = 260 columns, two tensor-core column tiles) and of the differentiation workload (T=64,
C=4, D=2048, N=512, K=32), on outputs the oracle computes one (task, cluster) pair at a time
with the exact Cholesky solve (Eq. 3).

The GPU runs the BF16X3 tensor-core operator with compensated refinement (refine_tol 1e-5),
the configuration the benchmark uses; its solutions are compared with the exact ones, which
the refined CG of Alg. 1 converges to."""
import numpy as np
import pytest

from oracle import cofem, philox
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import make_ctx, rel_err_rows

pytestmark = pytest.mark.gpu

REFINE = dict(refine_max=8, refine_tol=1e-5)


def _pair_exact(wl, alpha, it, t, c, G=None):
    """mu and s of pair (t, c) from exact solves with the same probes (Eqs. 3, 4)."""
    P = wl.phi(t).astype(np.float64)
    y = wl.yt(t).astype(np.float64)
    if G is None:
        G = wl.beta * (P.T @ P)
    pk = philox.probes(wl.seed, it, t, c, wl.C, wl.K, wl.D)            # [K, D]
    B = np.concatenate([cofem.rhs_mean(P, y, wl.beta)[:, None], pk.T], axis=1)
    X = cofem.solve_exact(P, wl.beta, alpha[c].astype(np.float64), B, G)
    return X[:, 0], np.mean(pk.T * X[:, 1:], axis=1)


@pytest.fixture(scope="module", params=["bf16x3", "bf16_mixed"])
def precision_run(request):
    """The precision workload on the tensor-core operator: the BF16 pair throughout, or the
    mixed path (the first solve with Phi as one BF16 plane, refinement with the pair)."""
    wl = synth.precision()
    with make_ctx(wl, precision=request.param, **REFINE) as ctx:
        ctx.em_iter(1)
        alpha = ctx.read(cmcs.OUT_ALPHA)
        it = ctx.summary()["em_iters_done"]
        ctx.estep()
        g = {k: ctx.read(v) for k, v in dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, logdet=cmcs.OUT_LOGDET,
                                              ell=cmcs.OUT_ELL, steps=cmcs.OUT_STEPS,
                                              gamma=cmcs.OUT_GAMMA, xi=cmcs.OUT_XI,
                                              q=cmcs.OUT_Q).items()}
        g["summary"] = ctx.summary()
    g["precision"] = request.param
    return wl, alpha, it, g


def test_precision_workload_sampled_pair(precision_run):
    """mu and s at 1e-4 (the BF16 pair) or at the reduced-precision bar of 1e-3 (the mixed
    path) against exact solves; nu and ell in replay."""
    wl, alpha, it, g = precision_run
    tol = 1e-4 if g["precision"] == "bf16x3" else 1e-3
    assert wl.C * (wl.K + 1) > 256                     # two TMEM column tiles
    assert g["summary"]["refine_diverged"] == 0
    t, c = 3, 2
    mu, s = _pair_exact(wl, alpha, it, t, c)
    assert rel_err_rows(g["mu"][t, c], mu) <= tol
    assert rel_err_rows(g["s"][t, c], s) <= tol
    nu = cofem.logdet_estimate(g["gamma"][t, c].astype(np.float64), g["xi"][t, c].astype(np.float64),
                               g["steps"][t, c, 1:], wl.D)
    assert abs(g["logdet"][t, c] - nu) <= 1e-9 * abs(nu)
    b0 = cofem.rhs_mean(wl.phi(t).astype(np.float64), wl.yt(t).astype(np.float64), wl.beta)
    ell = cofem.ell(nu, alpha[c].astype(np.float64), b0, mu)
    assert abs(g["ell"][t, c] - ell) <= 1e-6 * abs(ell)
    np.testing.assert_allclose(g["q"].sum(axis=1), 1.0, atol=1e-12)


@pytest.fixture(scope="module")
def diff_wl():
    return synth.differentiation()


def test_differentiation_workload_adjoint(diff_wl):
    """cmcs_adjoint at full size for a random dL/dmu: dy and dPhi of two sampled tasks (sums over
    all clusters) and dalpha of one cluster (sum over all 64 tasks) against the oracle's
    closed-form adjoint on exact solves.

    dy = beta Phi_t sum_c lambda_tc.  With D = 2048 > N = 512, lambda = A^-1 g is dominated by
    its component in the null space of Phi_t, which Phi_t removes: ||Phi lambda|| is far below
    ||Phi||_2 ||lambda||.  A solve accurate to a relative eps in lambda therefore fixes dy only
    to eps beta ||Phi_t||_2 sum_c ||lambda_tc||, and that is the scale dy is graded on (the
    refinement stops at eps = 1e-5).  dalpha = -sum_t lambda * mu has no such cancellation and
    is graded norm-wise."""
    wl = diff_wl
    rng = np.random.default_rng(77)
    w = rng.standard_normal((wl.T, wl.C, wl.D)).astype(np.float32)
    with make_ctx(wl, precision="bf16x3", **REFINE) as ctx:
        ctx.estep()
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        mu_gpu = ctx.read(cmcs.OUT_MU)
        dy, da, dP = ctx.adjoint(w)
    ro = wl.row_off
    c_chk = 1
    da_ref = np.zeros(wl.D)
    for t in range(wl.T):
        P = wl.phi(t).astype(np.float64)
        y = wl.yt(t).astype(np.float64)
        G = wl.beta * (P.T @ P)
        if t in (0, 37):
            dy_t = np.zeros(wl.N[t])
            dP_t = np.zeros((wl.N[t], wl.D))
            P2 = np.linalg.norm(P, 2)
            lam_scale = phi_scale = 0.0
            for c in range(wl.C):
                a = cofem.mean_adjoint(P, y, wl.beta, alpha[c], w[t, c].astype(np.float64), G)
                assert rel_err_rows(mu_gpu[t, c], a["mu"]) <= 1e-4, (t, c)
                dy_t += a["dy"]
                dP_t += a["dPhi"]
                nl = np.linalg.norm(a["lam"])
                lam_scale += nl
                phi_scale += nl * (np.linalg.norm(y - P @ a["mu"]) + P2 * np.linalg.norm(a["mu"]))
                if c == c_chk:
                    da_ref += a["dalpha"]
            assert np.linalg.norm(dy[ro[t]:ro[t + 1]] - dy_t) <= 1e-4 * wl.beta * P2 * lam_scale, t
            # dPhi = beta sum_c [(y - Phi mu) lambda^T - (Phi lambda) mu^T]: graded on the size of
            # its two outer products, the second of which carries the same cancellation as dy
            assert np.linalg.norm(dP[ro[t]:ro[t + 1]] - dP_t) <= 1e-4 * wl.beta * phi_scale, t
        else:
            a = cofem.mean_adjoint(P, y, wl.beta, alpha[c_chk], w[t, c_chk].astype(np.float64), G)
            da_ref += a["dalpha"]
    assert rel_err_rows(da[c_chk], da_ref) <= 1e-4


def test_differentiation_workload_adam_steps(diff_wl):
    """The differentiation workload's loss sum_t ||mu_{t, a_t} - z_t||^2 through PosteriorMeans:
    the workload's 100 Adam steps on Phi at full size lower it."""
    import torch
    from paper_2310_00420_gb300.adjoint import posterior_means
    wl = diff_wl
    Phi = torch.tensor(wl.Phi, device="cuda", requires_grad=True)
    y = torch.tensor(wl.y, device="cuda")
    z = torch.tensor(wl.z, device="cuda")
    opt = torch.optim.Adam([Phi], lr=1e-4)
    losses = []
    with make_ctx(wl, precision="bf16x3", **REFINE) as ctx:
        ctx.estep()
        al = torch.tensor(ctx.read(cmcs.OUT_ALPHA), device="cuda")
        assign = torch.tensor(ctx.read(cmcs.OUT_ASSIGN).astype(np.int64), device="cuda")
        rows = torch.arange(wl.T, device="cuda")
        for _ in range(100):
            mu = posterior_means(ctx, Phi, y, al, 0)
            loss = ((mu[rows, assign] - z) ** 2).sum()
            opt.zero_grad()
            loss.backward()
            assert torch.isfinite(Phi.grad).all()
            opt.step()
            losses.append(float(loss.detach()))
    assert losses[-1] < losses[0], losses
