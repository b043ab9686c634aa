"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (floating point): mu, s and alpha at norm-wise relative error <= 1e-4 per vector
for the FP32 path, responsibilities at absolute error <= 1e-4, hard assignments bit-exact;
random draws (probes, alpha initialisation) bit-exact.  Kernel-level checks use bounds
derived from their arithmetic (stated at each test)."""
import numpy as np
import pytest

from oracle import cofem, philox
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import check_free_q, make_ctx, rel_err_rows, task_lists

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4      # mu, s, alpha (FP32 path)
Q_TOL = 1e-4        # responsibilities, absolute


@pytest.fixture(scope="module")
def small():
    return synth.plain_small()


def test_probes_bit_exact(small):
    with make_ctx(small) as ctx:
        for e in (0, 5):
            P = ctx.probes(e)
            for t in range(small.T):
                for c in range(small.C):
                    ref = philox.probes(small.seed, e, t, c, small.C, small.K, small.D)
                    assert np.array_equal(P[t, c].astype(np.float64), ref), (e, t, c)


def test_alpha_init_bit_exact(small):
    with make_ctx(small) as ctx:
        a = ctx.read(cmcs.OUT_ALPHA)
    ref = philox.alpha_init(small.seed, small.C, small.D)
    assert np.array_equal(a.astype(np.float64), ref)


def test_b0_matches_oracle(small):
    P, Y = task_lists(small)
    with make_ctx(small) as ctx:
        b0 = ctx.read(cmcs.OUT_B0)
    ref = np.stack([cofem.rhs_mean(P[t], Y[t], small.beta) for t in range(small.T)])
    # the stored value is the FP32 rounding of a compensated sum: relative 2^-24 per entry
    np.testing.assert_allclose(b0, ref, rtol=1.2e-7, atol=1e-30)


def test_operator_matches_oracle(small):
    """FP32 GEMMs over N = 64 and D = 256 terms: a normwise error of 2e-6 is ~30 ulps."""
    P, Y = task_lists(small)
    R = small.C * (small.K + 1)
    rng = np.random.default_rng(11)
    V = rng.standard_normal((small.T, R, small.D)).astype(np.float32)
    with make_ctx(small) as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        Z = ctx.apply(V)
    for t in range(small.T):
        for j in range(R):
            c = j // (small.K + 1)
            ref = cofem.apply_A(P[t], small.beta, alpha[c], V[t, j].astype(np.float64))
            assert rel_err_rows(Z[t, j], ref) < 2e-6, (t, j)


def test_residual_is_compensated(small):
    """B - A X for X = fl32(A^-1 B): the true residual is ~1e-7 of ||B||, so an FP32 residual
    would be all rounding; the compensated one must match FP64 to FP32 output rounding."""
    P, Y = task_lists(small)
    R = small.C * (small.K + 1)
    rng = np.random.default_rng(12)
    B = rng.standard_normal((small.T, R, small.D)).astype(np.float32)
    with make_ctx(small) as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        X = np.empty_like(B)
        for t in range(small.T):
            for c in range(small.C):
                A = small.beta * P[t].T @ P[t] + np.diag(alpha[c])
                js = slice(c * (small.K + 1), (c + 1) * (small.K + 1))
                X[t, js] = np.linalg.solve(A, B[t, js].astype(np.float64).T).T.astype(np.float32)
        Rg = ctx.apply(X, accurate=True, B=B)
    for t in range(small.T):
        for j in range(R):
            c = j // (small.K + 1)
            x = X[t, j].astype(np.float64)
            ref = B[t, j].astype(np.float64) - cofem.apply_A(P[t], small.beta, alpha[c], x)
            # magnitude of the summed terms: |B| + beta |Phi|^T |Phi| |x| + alpha |x|
            scale = np.linalg.norm(np.abs(B[t, j]) + cofem.apply_A(np.abs(P[t]), small.beta,
                                                                    alpha[c], np.abs(x)))
            err = np.linalg.norm(Rg[t, j] - ref)
            # compensated sums: ~2^-44 of the terms; a plain FP32 residual errs by ~1e-7 * scale
            assert err <= 2e-7 * np.linalg.norm(ref) + 1e-11 * scale, (t, j, err, scale)


def test_quadrature_matches_oracle_on_same_coefficients(small):
    """The GPU's FP64 implicit-QR eigen step vs LAPACK on the same Lanczos coefficients."""
    import torch
    P, Y = task_lists(small)
    alpha = philox.alpha_init(0, small.C, small.D)
    rows_g, rows_x, steps = [], [], []
    for t in range(2):
        for c in range(small.C):
            Pk = philox.probes(0, 0, t, c, small.C, 6, small.D)
            for U in (1, 2, 7, 40, 100):
                r = cofem.cg(lambda V, idx: cofem.apply_A(P[t], small.beta, alpha[c], V), Pk.T,
                             0.0, U)
                for k in range(6):
                    gk = np.zeros(100, np.float32)
                    xk = np.zeros(100, np.float32)
                    gk[:U] = r.gamma[k][:U]
                    xk[:U] = r.xi[k][:U]
                    rows_g.append(gk)
                    rows_x.append(xk)
                    steps.append(int(r.steps[k]))
    g = np.stack(rows_g)
    x = np.stack(rows_x)
    st = np.array(steps, dtype=np.int32)
    out, status = cmcs.lanczos_quadrature(torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda(),
                                          torch.from_numpy(st).cuda())
    assert status == 0
    out = out.cpu().numpy()
    for i in range(len(st)):
        G = cofem.lanczos_tridiag(g[i].astype(np.float64), x[i].astype(np.float64), int(st[i]))
        lam, V = np.linalg.eigh(G)
        ref = float(np.sum(V[0] ** 2 * np.log(lam)))
        scale = float(np.sum(V[0] ** 2 * np.abs(np.log(lam)))) + 1.0
        assert abs(out[i] - ref) <= 1e-9 * scale, (i, out[i], ref)


@pytest.mark.parametrize("scale", [1e-30, 1e-20, 1e20, 1e30])
def test_quadrature_at_extreme_scales(small, scale):
    """The eigen step on Lanczos matrices scaled by `scale` (the CG coefficients of scale * A:
    gamma / scale, the same xi), whose chased rotations leave single precision's range, against
    LAPACK: sum_u S_u1^2 log lambda_u shifts by exactly log(scale)."""
    import torch
    P, Y = task_lists(small)
    alpha = philox.alpha_init(0, small.C, small.D)
    Pk = philox.probes(0, 0, 0, 0, small.C, 8, small.D)
    r = cofem.cg(lambda V, idx: cofem.apply_A(P[0], small.beta, alpha[0], V), Pk.T, 0.0, 100)
    g = np.stack([(r.gamma[k] / scale).astype(np.float32) for k in range(8)])
    x = np.stack([r.xi[k].astype(np.float32) for k in range(8)])
    st = r.steps.astype(np.int32)
    out, status = cmcs.lanczos_quadrature(torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda(),
                                          torch.from_numpy(st).cuda())
    assert status == 0
    out = out.cpu().numpy()
    for i in range(8):
        G = cofem.lanczos_tridiag(g[i].astype(np.float64), x[i].astype(np.float64), int(st[i]))
        lam, V = np.linalg.eigh(G)
        ref = float(np.sum(V[0] ** 2 * np.log(lam)))
        mag = float(np.sum(V[0] ** 2 * np.abs(np.log(lam)))) + 1.0
        assert abs(out[i] - ref) <= 1e-9 * mag, (scale, i, out[i], ref)


def replay_q(wl, g, o, alpha32):
    """Responsibilities the oracle computes from the GPU's own CG coefficients (replay of the
    Lanczos coefficients, Eqs. 9-11) and the oracle's refined means: q, ell, nu."""
    T, C = wl.T, wl.C
    nu = np.zeros((T, C))
    ell = np.zeros((T, C))
    for t in range(T):
        b0 = cofem.rhs_mean(wl.phi(t).astype(np.float64), wl.yt(t).astype(np.float64), wl.beta)
        for c in range(C):
            nu[t, c] = cofem.logdet_estimate(g["gamma"][t, c].astype(np.float64),
                                             g["xi"][t, c].astype(np.float64),
                                             g["steps"][t, c, 1:], wl.D)
            ell[t, c] = cofem.ell(nu[t, c], alpha32[c].astype(np.float64), b0, o["mu"][t, c])
    return cofem.responsibilities(ell, wl.pi), ell, nu


def _estep_pair(wl, alpha32, em_iter, refine_tol_gpu=1e-6):
    P, Y = task_lists(wl)
    with make_ctx(wl, refine_max=12, refine_tol=refine_tol_gpu) as ctx:
        ctx.set_alpha(alpha32, em_iter)
        ctx.estep()
        g = {k: ctx.read(v) for k, v in dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, q=cmcs.OUT_Q,
                                              logdet=cmcs.OUT_LOGDET, ell=cmcs.OUT_ELL,
                                              steps=cmcs.OUT_STEPS, gamma=cmcs.OUT_GAMMA,
                                              xi=cmcs.OUT_XI, assign=cmcs.OUT_ASSIGN).items()}
        g["summary"] = ctx.summary()
    o = cofem.cofem_estep(P, Y, alpha32.astype(np.float64), wl.pi, wl.beta, wl.K, wl.seed, em_iter,
                          wl.cg_tol, wl.cg_max_iter, refine_tol=1e-12, refine_max=40)
    return g, o


def test_estep_parity_plain_small(small):
    alpha = synth.uniform_alpha(small.C, small.D, seed=3)
    g, o = _estep_pair(small, alpha, em_iter=2)
    assert rel_err_rows(g["mu"], o["mu"]).max() <= REL_TOL
    assert rel_err_rows(g["s"], o["s"]).max() <= REL_TOL
    # log det, ell, q: the oracle's quadrature on the GPU's own CG coefficients (replay) ...
    q_rep, ell_rep, nu_rep = replay_q(small, g, o, alpha)
    assert np.max(np.abs(g["logdet"] - nu_rep) / np.abs(nu_rep)) <= 1e-9
    assert np.max(np.abs(g["ell"] - ell_rep) / np.abs(ell_rep)) <= 1e-6
    assert np.max(np.abs(g["q"] - q_rep)) <= Q_TOL
    # ... and the free-running FP32 vs FP64 CG estimates
    assert np.max(np.abs(g["logdet"] - o["logdet"]) / np.abs(o["logdet"])) <= 1e-4
    check_free_q(g["q"], o["q"])
    assert np.array_equal(g["assign"], np.argmax(o["q"], axis=1))


def test_mstep_matches_oracle_on_gpu_estep(small):
    alpha = synth.uniform_alpha(small.C, small.D, seed=4)
    with make_ctx(small, refine_max=8, refine_tol=1e-6) as ctx:
        ctx.set_alpha(alpha, 0)
        ctx.em_iter(1)
        mu, s, q = ctx.read(cmcs.OUT_MU), ctx.read(cmcs.OUT_S), ctx.read(cmcs.OUT_Q)
        new = ctx.read(cmcs.OUT_ALPHA)
    ref = cofem.m_step(q, mu.astype(np.float64), s.astype(np.float64), alpha.astype(np.float64))
    # FP64 sums of the same FP32 inputs, one FP32 rounding of the result
    np.testing.assert_allclose(new, ref, rtol=2e-7)


def test_em_parity_plain_small(small):
    """Ten EM iterations of Alg. 2 from the library's own alpha draw on both sides."""
    P, Y = task_lists(small)
    with make_ctx(small, refine_max=12, refine_tol=1e-6) as ctx:
        ctx.em_iter(small.em_iters)
        a_g = ctx.read(cmcs.OUT_ALPHA)
        q_g = ctx.read(cmcs.OUT_Q)
        asg = ctx.read(cmcs.OUT_ASSIGN)
        recon = ctx.read(cmcs.OUT_RECON)
    o = cofem.em(P, Y, small.pi, small.beta, small.em_iters, K=small.K, seed=small.seed,
                 tol=small.cg_tol, max_iter=small.cg_max_iter, C=small.C, D=small.D,
                 refine_tol=1e-12, refine_max=40)
    assert np.array_equal(asg, o["assign"])
    check_free_q(q_g, o["last"]["q"], soft_tasks=(2,))      # task 2: q = (0.992, 0.008)
    assert rel_err_rows(a_g, o["alpha"]).max() <= REL_TOL
    assert rel_err_rows(recon, o["recon"]).max() <= REL_TOL


@pytest.mark.parametrize("shape, soft", [
    (dict(T=3, C=3, D=200, N=(37, 150), K=5), (2,)),   # task 2: q = (0.005, 0.320, 0.675)
    (dict(T=1, C=1, D=129, N=10, K=1), ()),
    (dict(T=2, C=2, D=384, N=(1, 300), K=3), ())])
def test_ragged_and_degenerate_shapes(shape, soft):
    wl = synth.make_workload("ragged", shape["T"], shape["C"], shape["D"], shape["N"], nnz=5,
                             sigma=0.01, K=shape["K"], cg_tol=1e-6, cg_max_iter=60, seed=7)
    alpha = synth.uniform_alpha(wl.C, wl.D, seed=8) + np.float32(0.05)
    g, o = _estep_pair(wl, alpha, em_iter=1)
    assert rel_err_rows(g["mu"], o["mu"]).max() <= REL_TOL
    assert rel_err_rows(g["s"], o["s"]).max() <= REL_TOL
    q_rep, _, _ = replay_q(wl, g, o, alpha)
    assert np.max(np.abs(g["q"] - q_rep)) <= Q_TOL
    check_free_q(g["q"], o["q"], soft_tasks=soft)
    with make_ctx(wl) as ctx:
        P = ctx.probes(1)
    for t in range(wl.T):
        for c in range(wl.C):
            assert np.array_equal(P[t, c].astype(np.float64),
                                  philox.probes(wl.seed, 1, t, c, wl.C, wl.K, wl.D))


def test_nan_measurement_is_reported(small):
    y = small.y.copy()
    y[3] = np.nan
    import torch
    ctx = cmcs.Context(torch.from_numpy(small.Phi).cuda(), torch.from_numpy(y).cuda(), small.N,
                       C=small.C, K=small.K, beta=small.beta)
    with pytest.raises(cmcs.CmcsError) as ei:
        ctx.estep()
    assert ei.value.status == cmcs.ERR_NUMERIC
    ctx.close()


def test_set_alpha_rejects_nonpositive(small):
    with make_ctx(small) as ctx:
        a = np.ones((small.C, small.D), np.float32)
        a[1, 3] = 0.0
        with pytest.raises(cmcs.CmcsError) as ei:
            ctx.set_alpha(a, 0)
        assert ei.value.status == cmcs.ERR_INVALID_ARG


def test_host_and_device_inputs_agree(small):
    with cmcs.Context(small.Phi, small.y, small.N, C=small.C, K=small.K, beta=small.beta,
                      cg_tol=small.cg_tol, seed=small.seed) as h, make_ctx(small) as d:
        h.estep()
        d.estep()
        assert np.array_equal(h.read(cmcs.OUT_MU), d.read(cmcs.OUT_MU))
        assert np.array_equal(h.read(cmcs.OUT_Q), d.read(cmcs.OUT_Q))


def test_estep_is_deterministic(small):
    with make_ctx(small, refine_max=2) as a, make_ctx(small, refine_max=2) as b:
        a.estep()
        b.estep()
        for w in (cmcs.OUT_MU, cmcs.OUT_S, cmcs.OUT_LOGDET, cmcs.OUT_Q):
            assert np.array_equal(a.read(w), b.read(w))
