"""Adjoint of the E-step means (cmcs_adjoint, the PosteriorMeans autograd Function) against
FP64 central finite differences of the exact means and against dense FP64 autograd.

mu_tc = (beta Phi_t^T Phi_t + diag alpha_c)^-1 beta Phi_t^T y_t (Eq. 3); the loss is linear,
L = sum w * mu, so dL/dmu = w.  The GPU solves in FP32 with compensated refinement, so its
gradients carry ~1e-6 relative error; the bound 1e-4 is normwise (or relative to the sum of
the directional terms' magnitudes for the finite-difference check)."""
import numpy as np
import pytest

from paper_2310_00420_gb300 import cmcs, synth

pytestmark = pytest.mark.gpu

BETA = 100.0


def _problem(T, C, D, N, seed):
    wl = synth.make_workload("adjoint", T, C, D, N, nnz=6, sigma=0.05, beta=BETA, K=4,
                             cg_tol=1e-7, cg_max_iter=200, seed=seed)
    rng = np.random.default_rng(seed + 1)
    alpha = rng.uniform(0.3, 2.0, size=(C, D)).astype(np.float32)
    w = rng.standard_normal((T, C, D)).astype(np.float32)
    return wl, alpha, w


def _exact_mu(Phi_list, y_list, alpha, beta):
    T, (C, D) = len(Phi_list), alpha.shape
    mu = np.zeros((T, C, D))
    for t in range(T):
        G = beta * Phi_list[t].T @ Phi_list[t]
        b = beta * Phi_list[t].T @ y_list[t]
        for c in range(C):
            mu[t, c] = np.linalg.solve(G + np.diag(alpha[c]), b)
    return mu


def _gpu_grads(wl, alpha, w):
    import torch
    with cmcs.Context(torch.from_numpy(wl.Phi).cuda(), torch.from_numpy(wl.y).cuda(), wl.N,
                      C=wl.C, K=wl.K, beta=wl.beta, cg_tol=wl.cg_tol, cg_max_iter=wl.cg_max_iter,
                      refine_max=16, refine_tol=1e-7) as ctx:
        ctx.set_alpha(alpha, 0)
        ctx.estep()
        mu = ctx.read(cmcs.OUT_MU)
        dy, da, dP = ctx.adjoint(torch.from_numpy(w).cuda())
        return mu, dy.cpu().numpy(), da.cpu().numpy(), dP.cpu().numpy()


def test_adjoint_matches_fp64_finite_differences():
    wl, alpha, w = _problem(T=2, C=2, D=64, N=(20, 40), seed=31)
    mu, dy, da, dP = _gpu_grads(wl, alpha, w)
    P = [wl.phi(t).astype(np.float64) for t in range(wl.T)]
    Y = [wl.yt(t).astype(np.float64) for t in range(wl.T)]
    A64 = alpha.astype(np.float64)
    np.testing.assert_allclose(mu, _exact_mu(P, Y, A64, BETA), rtol=1e-4, atol=1e-6)
    rng = np.random.default_rng(5)
    h = 1e-6
    W = w.astype(np.float64)
    loss = lambda P_, Y_, A_: float(np.sum(W * _exact_mu(P_, Y_, A_, BETA)))
    for _ in range(16):
        vP = [rng.standard_normal(p.shape) for p in P]
        vY = [rng.standard_normal(v.shape) for v in Y]
        vA = rng.standard_normal(A64.shape)
        plus = loss([p + h * v for p, v in zip(P, vP)], [y + h * v for y, v in zip(Y, vY)], A64 + h * vA)
        minus = loss([p - h * v for p, v in zip(P, vP)], [y - h * v for y, v in zip(Y, vY)], A64 - h * vA)
        fd = (plus - minus) / (2 * h)
        terms = [np.sum(dP[wl.row_off[t]:wl.row_off[t + 1]] * vP[t]) for t in range(wl.T)]
        terms += [np.sum(dy[wl.row_off[t]:wl.row_off[t + 1]] * vY[t]) for t in range(wl.T)]
        terms += [np.sum(da * vA)]
        ad = float(np.sum(terms))
        scale = float(np.sum(np.abs(terms)))
        assert abs(ad - fd) <= 1e-4 * scale, (ad, fd, scale)


def test_adjoint_matches_dense_autograd_d128():
    torch = pytest.importorskip("torch")
    wl, alpha, w = _problem(T=2, C=2, D=128, N=48, seed=41)
    mu, dy, da, dP = _gpu_grads(wl, alpha, w)
    Phi = torch.tensor(wl.Phi, dtype=torch.float64, requires_grad=True)
    y = torch.tensor(wl.y, dtype=torch.float64, requires_grad=True)
    al = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    L = 0.0
    for t in range(wl.T):
        Pt = Phi[wl.row_off[t]:wl.row_off[t + 1]]
        yt = y[wl.row_off[t]:wl.row_off[t + 1]]
        for c in range(wl.C):
            A = BETA * Pt.T @ Pt + torch.diag(al[c])
            m = torch.linalg.solve(A, BETA * Pt.T @ yt)
            L = L + (torch.tensor(w[t, c], dtype=torch.float64) * m).sum()
    L.backward()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(dP, Phi.grad.numpy()) <= 1e-4
    assert rel(dy, y.grad.numpy()) <= 1e-4
    assert rel(da, al.grad.numpy()) <= 1e-4


def test_autograd_function_descends():
    """A few Adam steps on Phi through PosteriorMeans reduce sum_t ||mu_{t,c(t)} - z_t||^2."""
    import torch
    from paper_2310_00420_gb300.adjoint import posterior_means
    wl, alpha, _ = _problem(T=3, C=2, D=96, N=40, seed=51)
    Phi = torch.tensor(wl.Phi, device="cuda", requires_grad=True)
    y = torch.tensor(wl.y, device="cuda")
    al = torch.tensor(alpha, device="cuda", requires_grad=True)
    z = torch.tensor(wl.z, device="cuda")
    opt = torch.optim.Adam([Phi], lr=1e-3)
    losses = []
    with cmcs.Context(Phi.detach(), y, wl.N, C=wl.C, K=wl.K, beta=wl.beta, cg_tol=1e-7,
                      cg_max_iter=200, refine_max=16, refine_tol=1e-7) as ctx:
        for it in range(8):
            mu = posterior_means(ctx, Phi, y, al, 0)
            loss = ((mu[:, 0] - z) ** 2).sum()
            opt.zero_grad()
            loss.backward()
            assert Phi.grad is not None and al.grad is not None
            opt.step()
            losses.append(float(loss))
    assert losses[-1] < losses[0]
