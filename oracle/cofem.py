"""Plain FP64 reference for exact EM and covariance-free EM (CoFEM) on the clustered
multi-task compressive sensing model (Lin & Ba, "An efficient algorithm for clustered
multi-task compressive sensing").

TEST INFRASTRUCTURE ONLY: this is the slow, obviously-correct CPU oracle the CUDA path is
checked against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import it; the library itself never does, and nothing here is shared with the CUDA code.

Everything is float64 numpy.  Library primitives used as single steps: matrix products,
Cholesky (numpy.linalg.cholesky), triangular solves (scipy.linalg.solve_triangular) and the
symmetric eigensolver (numpy.linalg.eigh).  Inputs Phi_t and y_t arrive as the FP32 values
the GPU sees and are promoted to float64 exactly.

Conventions: T tasks, C clusters, D signal dimension, N_t rows of Phi_t, K probes per
(t, c).  The paper also uses K for the number of clusters in Eq. 1 and Sec. 4; here C is
always the cluster count and K the probe count.

Readings where the paper leaves a choice (each applied identically on the GPU):
* CG stopping (Alg. 1 runs "until convergence"): system i stops after the first step u with
  ||r_{u+1}||_2 <= tol * ||b||_2, or after max_iter steps, or when r'r == 0 or d'Ad <= 0.
  U_i is the number of completed steps; the Lanczos matrix of Eq. 9 uses gamma_1..gamma_U
  and xi_1..xi_{U-1}.
* Probes are fresh for every (EM iteration, t, c, k) (Alg. 2 samples them inside the loop).
* M-step (Eq. 5 with diag Sigma replaced by s): the per-task term max(mu^2 + s, 0), then
  alpha = clamp(num / den, alpha_min, alpha_max); den <= num / alpha_max gives alpha_max; a
  cluster whose total responsibility is below 1e-300 keeps its previous alpha.
* The returned responsibilities and means are those of the last E-step (Alg. 2 returns
  mu_{t, a_t} after the loop); ties in argmax go to the lowest cluster index.
* Variants, off by default: learned priors (``pi_update``, floored at 1e-300 so that log pi
  stays finite), probes shared across clusters, and Jacobi-preconditioned CG (``pcg``, whose
  stopping test is Alg. 1's on the symmetrically scaled system); see ``cofem_estep``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.linalg import solve_triangular

from . import philox

LOG_2PI = float(np.log(2.0 * np.pi))


# --------------------------------------------------------------------------------------
# model pieces (Eqs. 1, 3, 5)
# --------------------------------------------------------------------------------------

def rhs_mean(Phi_t: np.ndarray, y_t: np.ndarray, beta: float) -> np.ndarray:
    """b0 = beta * Phi_t^T y_t, the right-hand side of the posterior-mean system (Eq. 7)."""
    return beta * (Phi_t.T @ y_t)


def apply_A(Phi_t: np.ndarray, beta: float, alpha_c: np.ndarray, V: np.ndarray) -> np.ndarray:
    """A V with A = beta Phi_t^T Phi_t + diag(alpha_c) (Eq. 7), V of shape [D] or [D, m]."""
    if V.ndim == 1:
        return beta * (Phi_t.T @ (Phi_t @ V)) + alpha_c * V
    return beta * (Phi_t.T @ (Phi_t @ V)) + alpha_c[:, None] * V


def apply_A_fourier(mask_t: np.ndarray, beta: float, alpha_c: np.ndarray,
                    V: np.ndarray) -> np.ndarray:
    """A V for the structured sensing matrix Phi_t = Omega_t F of Sec. 4 (F the unitary DFT,
    Omega_t the rows selected by the 0/1 mask_t) with real z: A = beta Re(Phi^H Phi) +
    diag(alpha_c), and Phi^H Phi = F^H diag(mask) F, applied with FFTs (Sec. 3.3: CG needs
    only products with A).  V is [D] or [D, m]."""
    V = np.asarray(V, dtype=np.float64)
    m = np.asarray(mask_t, dtype=np.float64)
    ax = 0
    spec = np.fft.fft(V, axis=ax)
    shape = (-1,) + (1,) * (V.ndim - 1)
    out = np.fft.ifft(m.reshape(shape) * spec, axis=ax).real
    return beta * out + np.asarray(alpha_c, dtype=np.float64).reshape(shape) * V


def rhs_mean_fourier(mask_t: np.ndarray, y_t: np.ndarray, beta: float) -> np.ndarray:
    """b0 = beta Re(Phi_t^H y_t) for Phi_t = Omega_t F: the measured coefficients y_t (in
    ascending frequency order) placed at their frequencies, then F^H = sqrt(D) ifft."""
    m = np.asarray(mask_t)
    D = m.shape[0]
    Y = np.zeros(D, dtype=np.complex128)
    Y[np.nonzero(m)[0]] = np.asarray(y_t, dtype=np.complex128)
    return beta * (np.sqrt(D) * np.fft.ifft(Y)).real


class FourierSensing:
    """Phi_t = Omega_t F of Sec. 4 held as its 0/1 frequency mask, for E-steps at sizes where
    the dense real-stacked matrix does not fit.  Same reading as ``apply_A_fourier``: unitary
    F, real z, the complex measurements taken as [Re y_t; Im y_t] (ascending frequency)."""

    def __init__(self, mask_t: np.ndarray):
        self.mask = np.asarray(mask_t)

    def apply(self, beta: float, alpha_c: np.ndarray, V: np.ndarray) -> np.ndarray:
        return apply_A_fourier(self.mask, beta, alpha_c, V)

    def rhs(self, y_real: np.ndarray, beta: float) -> np.ndarray:
        n = y_real.shape[0] // 2
        return rhs_mean_fourier(self.mask, y_real[:n] + 1j * y_real[n:], beta)

    def diag(self, beta: float, alpha_c: np.ndarray) -> np.ndarray:
        """The diagonal of A: every column of Omega_t F has squared norm N_t / D."""
        m = self.mask
        return beta * float(np.count_nonzero(m)) / m.shape[0] + np.asarray(alpha_c, np.float64)


def task_const(y_t: np.ndarray, beta: float) -> float:
    """The c-independent part of log p(y_t | alpha_c):  log p = ell/2 - task_const, with
    task_const = (N log 2pi - N log beta + beta ||y||^2) / 2 (from Eqs. 1 and 3)."""
    N = y_t.shape[0]
    return 0.5 * (N * LOG_2PI - N * np.log(beta) + beta * float(y_t @ y_t))


def ell(logdet_sigma: float, alpha_c: np.ndarray, b0: np.ndarray, mu: np.ndarray) -> float:
    """ell_{t,c} = log det Sigma + sum_d log alpha_cd + beta y^T Phi mu  (Eq. 3), where
    beta y^T Phi mu is written as b0^T mu."""
    return float(logdet_sigma) + float(np.sum(np.log(alpha_c))) + float(b0 @ mu)


def responsibilities(ell_tc: np.ndarray, pi: np.ndarray) -> np.ndarray:
    """q_t = softmax_c(ell_tc / 2 + log pi_c)  (Eq. 3), max-shifted log-sum-exp, [T, C]."""
    z = 0.5 * ell_tc + np.log(pi)[None, :]
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def log_likelihood(ell_tc: np.ndarray, pi: np.ndarray, consts: np.ndarray) -> float:
    """L(theta) = (1/T) sum_t log sum_c pi_c p(y_t | alpha_c)  (Sec. 2), using
    log p(y_t | alpha_c) = ell_tc / 2 - consts[t]."""
    z = 0.5 * ell_tc + np.log(pi)[None, :]
    m = z.max(axis=1)
    lse = m + np.log(np.exp(z - m[:, None]).sum(axis=1))
    return float(np.mean(lse - consts))


def pi_update(q: np.ndarray, pi_floor: float = 1e-300) -> np.ndarray:
    """Cluster priors learned by EM (Sec. 2 notes that pi may be learned): the maximiser of
    sum_t sum_c q_tc log pi_c over the simplex, pi_c = (1/T) sum_t q_tc.  Reading: a cluster
    whose share underflows is floored at pi_floor and the priors are renormalised, so that
    log pi stays finite (the cluster then stays empty, as it would in exact arithmetic)."""
    pi = np.maximum(np.asarray(q, dtype=np.float64).mean(axis=0), pi_floor)
    return pi / pi.sum()


def jacobi_diag(Phi_t: np.ndarray, beta: float, alpha_c: np.ndarray) -> np.ndarray:
    """The diagonal m of A = beta Phi_t^T Phi_t + diag(alpha_c) (Eq. 7):
    m_d = beta sum_n Phi_nd^2 + alpha_d, the Jacobi preconditioner M = diag(m)."""
    P = np.asarray(Phi_t, dtype=np.float64)
    return beta * np.einsum("nd,nd->d", P, P) + np.asarray(alpha_c, dtype=np.float64)


def m_step(q: np.ndarray, mu: np.ndarray, s: np.ndarray, alpha_prev: np.ndarray,
           alpha_min: float = 1e-10, alpha_max: float = 1e10) -> np.ndarray:
    """Eq. 5: alpha_cd = sum_t q_tc / sum_t q_tc (mu_tcd^2 + s_tcd), with the clamps above.
    q [T, C], mu and s [T, C, D], alpha_prev [C, D]."""
    num = q.sum(axis=0)                                                   # [C]
    den = np.einsum("tc,tcd->cd", q, np.maximum(mu * mu + s, 0.0))        # [C, D]
    out = np.empty_like(alpha_prev)
    for c in range(q.shape[1]):
        if num[c] < 1e-300:
            out[c] = alpha_prev[c]
            continue
        with np.errstate(divide="ignore"):
            a = num[c] / den[c]
        a = np.where(den[c] <= num[c] / alpha_max, alpha_max, a)
        out[c] = np.clip(a, alpha_min, alpha_max)
    return out


# --------------------------------------------------------------------------------------
# Alg. 1: conjugate gradient, run side by side over the columns of B
# --------------------------------------------------------------------------------------

@dataclass
class CGResult:
    x: np.ndarray        # [D, m]
    gamma: np.ndarray    # [m, max_iter]  step sizes gamma_u
    xi: np.ndarray       # [m, max_iter]  direction coefficients xi_u
    steps: np.ndarray    # [m] completed steps U_i
    rel_resid: np.ndarray  # [m] ||r_{U+1}|| / ||b|| of the recursive residual


def cg(apply, B: np.ndarray, tol: float, max_iter: int, steps: np.ndarray = None,
       ref: np.ndarray = None) -> CGResult:
    """Alg. 1 with x_1 = 0, r_1 = d_1 = b, for every column of B (independent systems).

    apply(V) returns A V for the columns given.  If ``steps`` is given, column i runs exactly
    steps[i] steps (replay of a step count measured elsewhere) instead of the tol test.  ref
    (squared norms per column, default ||b||^2) is what the tol test compares against; a column
    already within tol of it takes no step."""
    D, m = B.shape
    X = np.zeros((D, m))
    R = B.astype(np.float64).copy()
    Dd = R.copy()
    rr = np.einsum("ij,ij->j", R, R)
    bb = rr.copy() if ref is None else np.asarray(ref, dtype=np.float64).copy()
    gam = np.zeros((m, max_iter))
    xi = np.zeros((m, max_iter))
    U = np.zeros(m, dtype=np.int64)
    if steps is None:
        active = (rr > 0.0) & ((ref is None) | (rr > (tol * tol) * bb))
    else:
        active = (np.asarray(steps) > 0) & (rr > 0.0)
    for u in range(max_iter):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        Dd_a = Dd[:, idx]
        AD = apply(Dd_a, idx)
        dAd = np.einsum("ij,ij->j", Dd_a, AD)
        ok = dAd > 0.0
        if not ok.all():
            active[idx[~ok]] = False
            idx, Dd_a, AD, dAd = idx[ok], Dd_a[:, ok], AD[:, ok], dAd[ok]
            if idx.size == 0:
                break
        g = rr[idx] / dAd                                   # gamma_u
        X[:, idx] += g * Dd_a                               # x_{u+1}
        R_a = R[:, idx] - g * AD                            # r_{u+1}
        rr_new = np.einsum("ij,ij->j", R_a, R_a)
        x_u = rr_new / rr[idx]                              # xi_u
        R[:, idx] = R_a
        Dd[:, idx] = R_a + x_u * Dd_a                       # d_{u+1}
        gam[idx, u] = g
        xi[idx, u] = x_u
        U[idx] += 1
        rr[idx] = rr_new
        if steps is None:
            done = (rr_new <= (tol * tol) * bb[idx]) | (rr_new == 0.0)
        else:
            done = U[idx] >= np.asarray(steps)[idx]
        active[idx[done]] = False
    rel = np.sqrt(rr / np.where(bb > 0, bb, 1.0))
    return CGResult(X, gam, xi, U, rel)


def pcg(apply, B: np.ndarray, minv: np.ndarray, tol: float, max_iter: int,
        steps: np.ndarray = None, ref: np.ndarray = None) -> CGResult:
    """Alg. 1 with a diagonal (Jacobi) preconditioner M = diag(m), minv = 1/m of shape [D]:
    x_1 = 0, r_1 = b, z_1 = M^-1 r_1, d_1 = z_1 and, per step,
        gamma_u = r_u^T z_u / d_u^T A d_u,   x_{u+1} = x_u + gamma_u d_u,
        r_{u+1} = r_u - gamma_u A d_u,       z_{u+1} = M^-1 r_{u+1},
        xi_u = r_{u+1}^T z_{u+1} / r_u^T z_u, d_{u+1} = z_{u+1} + xi_u d_u.
    Substituting x = M^-1/2 xh, r = M^1/2 rh, d = M^-1/2 dh turns these into Alg. 1 on
    Ah = M^-1/2 A M^-1/2 with right-hand side bh = M^-1/2 b and the same gamma_u and xi_u, so
    the matrix of Eq. 9 built from them is the Lanczos matrix of Ah started at bh / ||bh||.
    Reading of the stopping test: the one of Alg. 1 on that system, r^T z <= tol^2 b^T M^-1 b
    (||rh|| <= tol ||bh||); the other stops, ``steps`` and ``ref`` (here in the M^-1 norm) are
    as in ``cg``."""
    D, m = B.shape
    mi = np.asarray(minv, dtype=np.float64).reshape(D, 1)
    X = np.zeros((D, m))
    R = B.astype(np.float64).copy()
    Z = mi * R
    Dd = Z.copy()
    rz = np.einsum("ij,ij->j", R, Z)
    bz = rz.copy() if ref is None else np.asarray(ref, dtype=np.float64).copy()
    gam = np.zeros((m, max_iter))
    xi = np.zeros((m, max_iter))
    U = np.zeros(m, dtype=np.int64)
    if steps is None:
        active = (rz > 0.0) & ((ref is None) | (rz > (tol * tol) * bz))
    else:
        active = (np.asarray(steps) > 0) & (rz > 0.0)
    for u in range(max_iter):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        Dd_a = Dd[:, idx]
        AD = apply(Dd_a, idx)
        dAd = np.einsum("ij,ij->j", Dd_a, AD)
        ok = dAd > 0.0
        if not ok.all():
            active[idx[~ok]] = False
            idx, Dd_a, AD, dAd = idx[ok], Dd_a[:, ok], AD[:, ok], dAd[ok]
            if idx.size == 0:
                break
        g = rz[idx] / dAd                                   # gamma_u
        X[:, idx] += g * Dd_a
        R_a = R[:, idx] - g * AD                            # r_{u+1}
        Z_a = mi * R_a                                      # z_{u+1}
        rz_new = np.einsum("ij,ij->j", R_a, Z_a)
        x_u = rz_new / rz[idx]                              # xi_u
        R[:, idx] = R_a
        Dd[:, idx] = Z_a + x_u * Dd_a                       # d_{u+1}
        gam[idx, u] = g
        xi[idx, u] = x_u
        U[idx] += 1
        rz[idx] = rz_new
        if steps is None:
            done = (rz_new <= (tol * tol) * bz[idx]) | (rz_new == 0.0)
        else:
            done = U[idx] >= np.asarray(steps)[idx]
        active[idx[done]] = False
    rel = np.sqrt(rz / np.where(bz > 0, bz, 1.0))
    return CGResult(X, gam, xi, U, rel)


def refine(apply, B: np.ndarray, X: np.ndarray, tol: float, max_iter: int, refine_tol: float,
           refine_max: int, minv: np.ndarray = None):
    """Iterative refinement of the CG solutions X of A X = B: each sweep forms the residual
    B - A X, solves A delta = residual by Alg. 1 (x_1 = 0, same tol and step cap; ``pcg``
    with the same preconditioner when minv is given) and adds delta; column i stops once
    ||delta_i|| <= refine_tol * ||x_i||.  Returns (X, sweeps [m])."""
    X = X.copy()
    m = B.shape[1]
    sweeps = np.zeros(m, dtype=np.int64)
    active = np.ones(m, dtype=bool)
    for _ in range(refine_max):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        Rres = B[:, idx] - apply(X[:, idx], idx)
        sub_apply = lambda V, sub: apply(V, idx[sub])
        if minv is None:
            res = cg(sub_apply, Rres, tol, max_iter)
        else:
            res = pcg(sub_apply, Rres, minv, tol, max_iter)
        X[:, idx] += res.x
        sweeps[idx] += 1
        dn = np.linalg.norm(res.x, axis=0)
        xn = np.linalg.norm(X[:, idx], axis=0)
        active[idx[dn <= refine_tol * xn]] = False
    return X, sweeps


# --------------------------------------------------------------------------------------
# Eqs. 9-11: Lanczos quadrature of p^T log(A) p from the CG coefficients
# --------------------------------------------------------------------------------------

def lanczos_tridiag(gamma: np.ndarray, xi: np.ndarray, U: int) -> np.ndarray:
    """The U x U matrix of Eq. 9: G_11 = 1/gamma_1, G_uu = 1/gamma_u + xi_{u-1}/gamma_{u-1},
    G_{u,u-1} = G_{u-1,u} = sqrt(xi_{u-1}) / gamma_{u-1} (1-based indices as in the paper)."""
    G = np.zeros((U, U))
    G[0, 0] = 1.0 / gamma[0]
    for u in range(1, U):
        G[u, u] = 1.0 / gamma[u] + xi[u - 1] / gamma[u - 1]
        G[u, u - 1] = G[u - 1, u] = np.sqrt(xi[u - 1]) / gamma[u - 1]
    return G


def lanczos_log_quadrature(gamma: np.ndarray, xi: np.ndarray, U: int, pnorm2: float) -> float:
    """Eq. 10 restricted to the U x U Lanczos matrix (the inner sum of Eq. 11):
    ||p||^2 * sum_u S_{u,1}^2 log lambda_u, with the eigenpairs of G = S^T diag(lambda) S."""
    if U <= 0:
        return 0.0
    G = lanczos_tridiag(gamma, xi, U)
    lam, V = np.linalg.eigh(G)              # columns of V are eigenvectors: S = V^T
    first = V[0, :]                         # S_{u,1} for u = 1..U
    return float(pnorm2 * np.sum(first * first * np.log(lam)))


def logdet_estimate(gamma: np.ndarray, xi: np.ndarray, steps: np.ndarray, D: int) -> float:
    """Eq. 11: nu = -(1/K) sum_k sum_u D * (S^{(k)}_{u,1})^2 log lambda^{(k)}_u, where D is
    ||p_k||^2 for a Rademacher probe.  gamma, xi: [K, max_iter]; steps: [K]."""
    K = gamma.shape[0]
    tot = 0.0
    for k in range(K):
        tot += lanczos_log_quadrature(gamma[k], xi[k], int(steps[k]), float(D))
    return -tot / K


# --------------------------------------------------------------------------------------
# E-steps
# --------------------------------------------------------------------------------------

def _task_arrays(Phi_list, y_list):
    P = [p if isinstance(p, FourierSensing) else np.asarray(p, dtype=np.float64) for p in Phi_list]
    Y = [np.asarray(v, dtype=np.float64) for v in y_list]
    return P, Y


def exact_estep(Phi_list, y_list, alpha: np.ndarray, pi: np.ndarray, beta: float) -> dict:
    """Eq. 3 evaluated exactly: Sigma_tc = (beta Phi^T Phi + diag alpha_c)^-1 by Cholesky
    A = L L^T, mu = Sigma b0, diag Sigma from the columns of L^-1, log det Sigma = -2 sum log L_ii."""
    P, Y = _task_arrays(Phi_list, y_list)
    T, (C, D) = len(P), alpha.shape
    mu = np.zeros((T, C, D))
    sdiag = np.zeros((T, C, D))
    logdet = np.zeros((T, C))
    ell_tc = np.zeros((T, C))
    consts = np.array([task_const(Y[t], beta) for t in range(T)])
    for t in range(T):
        G = beta * (P[t].T @ P[t])
        b0 = rhs_mean(P[t], Y[t], beta)
        for c in range(C):
            A = G + np.diag(alpha[c])
            L = np.linalg.cholesky(A)
            Linv = solve_triangular(L, np.eye(D), lower=True)          # Sigma = Linv^T Linv
            w = solve_triangular(L, b0, lower=True)
            mu[t, c] = solve_triangular(L.T, w, lower=False)
            sdiag[t, c] = np.einsum("ij,ij->j", Linv, Linv)
            logdet[t, c] = -2.0 * np.sum(np.log(np.diag(L)))
            ell_tc[t, c] = ell(logdet[t, c], alpha[c], b0, mu[t, c])
    q = responsibilities(ell_tc, pi)
    return dict(mu=mu, s=sdiag, logdet=logdet, ell=ell_tc, q=q,
                loglik=log_likelihood(ell_tc, pi, consts))


def solve_exact(Phi_t: np.ndarray, beta: float, alpha_c: np.ndarray, B: np.ndarray,
                G: np.ndarray = None) -> np.ndarray:
    """Sigma B with Sigma = (beta Phi_t^T Phi_t + diag alpha_c)^-1 (Eq. 3), by Cholesky: the
    exact solutions of the systems A mu = b0 and A x_k = p_k (Eq. 7) that Alg. 1 and its
    refinement approximate.  B is [D] or [D, m]; G = beta Phi_t^T Phi_t may be passed in to
    share it across clusters."""
    P = np.asarray(Phi_t, dtype=np.float64)
    if G is None:
        G = beta * (P.T @ P)
    A = G + np.diag(np.asarray(alpha_c, dtype=np.float64))
    L = np.linalg.cholesky(A)
    w = solve_triangular(L, np.asarray(B, dtype=np.float64), lower=True)
    return solve_triangular(L.T, w, lower=False)


def mean_adjoint(Phi_t: np.ndarray, y_t: np.ndarray, beta: float, alpha_c: np.ndarray,
                 g: np.ndarray, G: np.ndarray = None) -> dict:
    """Reverse-mode derivative of the posterior mean mu = Sigma beta Phi_t^T y_t (Eq. 3) for a
    loss L with dL/dmu = g.  With A = Sigma^-1 = beta Phi^T Phi + diag alpha and
    b = beta Phi^T y, differentiating A mu = b gives d mu = Sigma (db - dA mu), so
    dL = lam^T (db - dA mu) with lam = Sigma g (Sigma is symmetric).  Expanding db and dA:
        dL/dy     = beta Phi lam
        dL/dalpha = -lam * mu
        dL/dPhi   = beta (y lam^T - (Phi mu) lam^T - (Phi lam) mu^T)."""
    P = np.asarray(Phi_t, dtype=np.float64)
    y = np.asarray(y_t, dtype=np.float64)
    if G is None:
        G = beta * (P.T @ P)
    mu = solve_exact(P, beta, alpha_c, rhs_mean(P, y, beta), G)
    lam = solve_exact(P, beta, alpha_c, np.asarray(g, dtype=np.float64), G)
    Pmu, Plam = P @ mu, P @ lam
    return dict(mu=mu, lam=lam, dy=beta * Plam, dalpha=-lam * mu,
                dPhi=beta * (np.outer(y, lam) - np.outer(Pmu, lam) - np.outer(Plam, mu)))


def cofem_estep(Phi_list, y_list, alpha: np.ndarray, pi: np.ndarray, beta: float, K: int,
                seed: int, em_iter: int, tol: float, max_iter: int, probe_fn=None,
                steps: np.ndarray = None, tasks=None, refine_tol: float = None,
                refine_max: int = 8, clusters=None, C_total: int = None,
                probe_share: bool = False, precond: bool = False, mu_init=None) -> dict:
    """Alg. 2, inner loop (one E-step): for every (t, c) solve A mu = b0 and A x_k = p_k by CG
    (Eq. 7, Alg. 1), s = (1/K) sum_k p_k * x_k (Eq. 4), the log-det estimate of Eq. 11 from the
    CG coefficients of the probe systems, ell (Eq. 3) and the responsibilities (Eq. 3).

    probe_fn(t, c) -> [K, D] overrides the Philox probes; steps [T, C, K+1] replays given CG
    step counts; tasks gives the global task index of each entry of Phi_list (for the probe
    counter) when the list is a subset; likewise clusters gives the global index of each row
    of alpha and C_total the full cluster count (bounded samples).  With refine_tol set, mu and every x_k are refined
    (``refine``) after the first CG solve, which alone supplies the Lanczos coefficients.

    An entry of Phi_list may be a ``FourierSensing`` (Sec. 4's Phi_t = Omega_t F); its y_list
    entry is then [Re y_t; Im y_t].

    Variants (off by default):
    * probe_share: every cluster of task t uses the probes of cluster 0, p_{t,c,k} = p_{t,0,k}
      (common random numbers across c, so the estimation noise of ell_tc - ell_tc' shrinks).
    * precond: Jacobi-preconditioned CG (``pcg``) with M = diag(m), m = ``jacobi_diag``.  The
      probe systems become A x_k = w * p_k with w = sqrt(m), so that the scaled system
      Ah xh = M^-1/2 (w * p_k) = p_k starts its Lanczos process at a Rademacher vector; then
      diag(A^-1) = M^-1/2 diag(Ah^-1) M^-1/2 gives s = (1/K) sum_k p_k * x_k / w, and
      log det A = log det Ah + sum_d log m_d gives nu = (Eq. 11 on the pcg coefficients)
      - sum_d log m_d.
    * mu_init [T, C, D]: the mean system starts from x_1 = mu_init (the previous E-step's
      means).  It is Alg. 1 on A delta = b0 - A mu_init from delta = 0, stopped at the cold
      start's absolute target ||r|| <= tol ||b0|| (||b0|| in the M^-1 norm with precond), and
      mu = mu_init + delta.  The probe systems keep x_1 = 0, which their Lanczos reading
      needs."""
    P, Y = _task_arrays(Phi_list, y_list)
    T, (C, D) = len(P), alpha.shape
    tasks = list(range(T)) if tasks is None else list(tasks)
    clusters = list(range(C)) if clusters is None else list(clusters)
    C_total = C if C_total is None else int(C_total)
    mu = np.zeros((T, C, D))
    s = np.zeros((T, C, D))
    nu = np.zeros((T, C))
    ell_tc = np.zeros((T, C))
    U = np.zeros((T, C, K + 1), dtype=np.int64)
    gam = np.zeros((T, C, K + 1, max_iter))
    xis = np.zeros((T, C, K + 1, max_iter))
    rel = np.zeros((T, C, K + 1))
    consts = np.array([task_const(Y[t], beta) for t in range(T)])
    for t in range(T):
        fs = isinstance(P[t], FourierSensing)
        b0 = P[t].rhs(Y[t], beta) if fs else rhs_mean(P[t], Y[t], beta)
        for c in range(C):
            if probe_fn is None:
                pc = 0 if probe_share else clusters[c]
                Pk = philox.probes(seed, em_iter, tasks[t], pc, C_total, K, D)
            else:
                Pk = np.asarray(probe_fn(t, c), dtype=np.float64)
            if fs:
                op = lambda V, idx, t=t, c=c: P[t].apply(beta, alpha[c], V)
            else:
                op = lambda V, idx, t=t, c=c: apply_A(P[t], beta, alpha[c], V)
            st = None if steps is None else steps[t, c]
            if precond:
                m_d = P[t].diag(beta, alpha[c]) if fs else jacobi_diag(P[t], beta, alpha[c])
                w = np.sqrt(m_d)
                B = np.concatenate([b0[:, None], w[:, None] * Pk.T], axis=1)
            else:
                B = np.concatenate([b0[:, None], Pk.T], axis=1)          # [D, K+1]
            Bs, ref, x0 = B, None, None
            if mu_init is not None:
                x0 = np.asarray(mu_init[t, c], dtype=np.float64)
                Bs = B.copy()
                Bs[:, 0] = B[:, 0] - op(x0[:, None], None)[:, 0]
                # the tol test's reference: the cold start's ||b||^2 (b^T M^-1 b with precond)
                ref = np.einsum("ij,ij->j", B, B / m_d[:, None] if precond else B)
            if precond:
                res = pcg(op, Bs, 1.0 / m_d, tol, max_iter, st, ref=ref)
            else:
                res = cg(op, Bs, tol, max_iter, st, ref=ref)
            X = res.x
            if x0 is not None:
                X = X.copy()
                X[:, 0] += x0
            if refine_tol is not None:
                X, _ = refine(op, B, X, tol, max_iter, refine_tol, refine_max,
                              minv=(1.0 / m_d) if precond else None)
            mu[t, c] = X[:, 0]
            s[t, c] = np.mean(Pk.T * X[:, 1:], axis=1)
            nu[t, c] = logdet_estimate(res.gamma[1:], res.xi[1:], res.steps[1:], D)
            if precond:
                s[t, c] /= w
                nu[t, c] -= float(np.sum(np.log(m_d)))
            ell_tc[t, c] = ell(nu[t, c], alpha[c], b0, mu[t, c])
            U[t, c] = res.steps
            gam[t, c] = res.gamma
            xis[t, c] = res.xi
            rel[t, c] = res.rel_resid
    q = responsibilities(ell_tc, pi)
    return dict(mu=mu, s=s, logdet=nu, ell=ell_tc, q=q, steps=U, gamma=gam, xi=xis,
                rel_resid=rel, loglik=log_likelihood(ell_tc, pi, consts))


# --------------------------------------------------------------------------------------
# Alg. 2: the EM loop (exact or covariance-free E-step)
# --------------------------------------------------------------------------------------

def em(Phi_list, y_list, pi: np.ndarray, beta: float, n_iter: int, *, method: str = "cofem",
       K: int = 16, seed: int = 0, tol: float = 1e-5, max_iter: int = 100,
       alpha0: np.ndarray = None, em_iter_offset: int = 0, alpha_min: float = 1e-10,
       alpha_max: float = 1e10, D: int = None, C: int = None, refine_tol: float = None,
       refine_max: int = 8, learn_pi: bool = False, probe_share: bool = False,
       precond: bool = False, warm_start: bool = False) -> dict:
    """n_iter EM iterations from alpha0 (default: the Alg. 2 Uniform(0,1) draw).  Returns the
    last E-step's outputs, the final alpha (and pi), the hard assignments argmax_c q_tc and
    the reconstructions mu_{t, a_t}, plus the log-likelihood seen by every E-step.  With
    learn_pi each M-step also sets pi = ``pi_update(q)``; probe_share, precond and warm_start
    (each E-step's mean systems start from the previous E-step's means) select the E-step
    variants of ``cofem_estep``."""
    if alpha0 is None:
        alpha = philox.alpha_init(seed, C, D)
    else:
        alpha = np.asarray(alpha0, dtype=np.float64).copy()
    pi = np.asarray(pi, dtype=np.float64).copy()
    trace = []
    alphas = [alpha.copy()]
    est = None
    for it in range(n_iter):
        if method == "exact":
            est = exact_estep(Phi_list, y_list, alpha, pi, beta)
        else:
            mu0 = est["mu"] if (warm_start and est is not None) else None
            est = cofem_estep(Phi_list, y_list, alpha, pi, beta, K, seed, em_iter_offset + it,
                              tol, max_iter, refine_tol=refine_tol, refine_max=refine_max,
                              probe_share=probe_share, precond=precond, mu_init=mu0)
        trace.append(est["loglik"])
        alpha = m_step(est["q"], est["mu"], est["s"], alpha, alpha_min, alpha_max)
        if learn_pi:
            pi = pi_update(est["q"])
        alphas.append(alpha.copy())
    assign = np.argmax(est["q"], axis=1)
    recon = est["mu"][np.arange(len(assign)), assign]
    return dict(last=est, alpha=alpha, pi=pi, alphas=alphas, assign=assign, recon=recon,
                loglik_trace=np.array(trace))
