"""Seeded synthetic workloads for clustered multi-task compressive sensing.

This module only *generates inputs*: sensing matrices Phi_t, measurements y_t, the
ground-truth sparse signals z_t and their ground-truth cluster labels.  It holds none of
the inference method's arithmetic and is the one module that both the CUDA path and the
FP64 oracle use.

Two sensing setups.  ``make_fourier`` follows Sec. 4 itself (Phi_t = Omega_t F, a subsampled
unitary DFT; see FourierWorkload).  ``make_workload`` follows the model of Eq. 1 with the
simulation protocol of Sec. 4, except that Phi_t is a dense Gaussian matrix:

* Phi_t has i.i.d. entries N(0, 1/N_t), stored row-major (N_t x D), FP32.
* Ground-truth clusters partition the tasks (contiguous blocks of equal size, or
  Dirichlet(1) proportions with at least one task each).
* Each ground-truth cluster draws a support of round(sparsity * D) indices; a task keeps
  its cluster's support except for a fraction ``perturb`` of it, which is replaced by
  indices drawn outside the support.
* z_t is N(0, 1) on its support and zero elsewhere; y_t = Phi_t z_t + N(0, sigma_t^2).

All arrays are rounded to FP32 once, so both sides of any comparison see the same problem.
The random streams come from numpy's counter-based Philox bit generator keyed by
(seed, stream tag); the same seed gives the same workload within one numpy version.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# stream tags: each random quantity has a stream of its own
_TAG_PHI, _TAG_SUPPORT, _TAG_VALUES, _TAG_NOISE, _TAG_SIZES, _TAG_ALPHA = 1, 2, 3, 4, 5, 6


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), tag]))


@dataclass
class Workload:
    """One synthetic problem instance plus the solver settings it is run with."""

    name: str
    T: int
    C: int
    D: int
    N: np.ndarray                 # int64 [T]
    Phi: np.ndarray               # float32 [sum N_t, D], tasks packed row-wise
    row_off: np.ndarray           # int64 [T+1]; task t owns rows row_off[t]:row_off[t+1]
    y: np.ndarray                 # float32 [sum N_t], packed like Phi's rows
    z: np.ndarray                 # float32 [T, D] ground truth
    labels: np.ndarray            # int64 [T] ground-truth cluster of each task
    sigma: np.ndarray             # float64 [T] noise std used for each task
    beta: float = 1.0e4
    pi: np.ndarray = None         # float64 [C]
    K: int = 16
    cg_tol: float = 1e-5
    cg_max_iter: int = 100
    em_iters: int = 10
    seed: int = 0
    extra: dict = field(default_factory=dict)

    def phi(self, t: int) -> np.ndarray:
        return self.Phi[self.row_off[t]:self.row_off[t + 1]]

    def yt(self, t: int) -> np.ndarray:
        return self.y[self.row_off[t]:self.row_off[t + 1]]

    def subset(self, tasks) -> "Workload":
        """The same problem restricted to the given tasks (used to bound oracle work)."""
        tasks = list(tasks)
        Phi = np.concatenate([self.phi(t) for t in tasks], axis=0)
        y = np.concatenate([self.yt(t) for t in tasks])
        N = np.array([self.N[t] for t in tasks], dtype=np.int64)
        off = np.zeros(len(tasks) + 1, dtype=np.int64)
        off[1:] = np.cumsum(N)
        return Workload(self.name + f"[{len(tasks)} tasks]", len(tasks), self.C, self.D, N, Phi,
                        off, y, self.z[tasks].copy(), self.labels[tasks].copy(),
                        self.sigma[tasks].copy(), self.beta, self.pi.copy(), self.K, self.cg_tol,
                        self.cg_max_iter, self.em_iters, self.seed, dict(self.extra))

    @property
    def bytes_phi(self) -> int:
        return int(self.Phi.nbytes)


def _group_sizes(T: int, C: int, proportions: str, rng: np.random.Generator) -> np.ndarray:
    if proportions == "equal":
        base = np.full(C, T // C, dtype=np.int64)
        base[: T % C] += 1
        return base
    # Dirichlet(1) proportions, at least one task per group, sizes summing to T
    p = rng.dirichlet(np.ones(C))
    sizes = np.ones(C, dtype=np.int64)
    rest = T - C
    extra = np.floor(p * rest).astype(np.int64)
    sizes += extra
    short = T - sizes.sum()
    order = np.argsort(-(p * rest - extra))
    sizes[order[:short]] += 1
    return sizes


def make_workload(name: str, T: int, C: int, D: int, N, *, sparsity: float = None,
                  nnz: int = None, perturb: float = 0.0, sigma=0.01, beta: float = 1e4,
                  gt_clusters: int = None, proportions: str = "equal", K: int = 16,
                  cg_tol: float = 1e-5, cg_max_iter: int = 100, em_iters: int = 10,
                  seed: int = 0) -> Workload:
    """Generate a workload.  ``N`` is an int (all tasks) or a (lo, hi) pair for N_t ~ U[lo, hi];
    ``sigma`` is a float or a (lo, hi) pair for sigma_t ~ U[lo, hi]."""
    G = gt_clusters if gt_clusters is not None else C
    r_size = _rng(seed, _TAG_SIZES)
    if isinstance(N, (tuple, list)):
        Ns = r_size.integers(int(N[0]), int(N[1]) + 1, size=T).astype(np.int64)
    else:
        Ns = np.full(T, int(N), dtype=np.int64)
    if isinstance(sigma, (tuple, list)):
        sig = r_size.uniform(float(sigma[0]), float(sigma[1]), size=T)
    else:
        sig = np.full(T, float(sigma))
    sizes = _group_sizes(T, G, proportions, r_size)
    labels = np.repeat(np.arange(G, dtype=np.int64), sizes)

    if nnz is None:
        nnz = max(1, int(round(sparsity * D)))
    r_sup = _rng(seed, _TAG_SUPPORT)
    cluster_support = [np.sort(r_sup.choice(D, size=nnz, replace=False)) for _ in range(G)]
    n_swap = int(round(perturb * nnz))
    r_val = _rng(seed, _TAG_VALUES)
    z = np.zeros((T, D), dtype=np.float32)
    for t in range(T):
        sup = cluster_support[labels[t]].copy()
        if n_swap > 0:
            drop = r_sup.choice(nnz, size=n_swap, replace=False)
            outside = np.setdiff1d(np.arange(D), sup, assume_unique=True)
            sup[drop] = r_sup.choice(outside, size=n_swap, replace=False)
        z[t, sup] = r_val.standard_normal(nnz).astype(np.float32)

    off = np.zeros(T + 1, dtype=np.int64)
    off[1:] = np.cumsum(Ns)
    r_phi = _rng(seed, _TAG_PHI)
    Phi = np.empty((int(off[-1]), D), dtype=np.float32)
    chunk = max(1, (1 << 26) // D)
    for r0 in range(0, int(off[-1]), chunk):
        r1 = min(int(off[-1]), r0 + chunk)
        Phi[r0:r1] = r_phi.standard_normal((r1 - r0, D), dtype=np.float32)
    for t in range(T):
        Phi[off[t]:off[t + 1]] *= np.float32(1.0 / np.sqrt(float(Ns[t])))

    r_noise = _rng(seed, _TAG_NOISE)
    y = np.empty(int(off[-1]), dtype=np.float32)
    for t in range(T):
        Pt = Phi[off[t]:off[t + 1]].astype(np.float64)
        clean = Pt @ z[t].astype(np.float64)
        y[off[t]:off[t + 1]] = (clean + sig[t] * r_noise.standard_normal(int(Ns[t]))).astype(np.float32)

    pi = np.full(C, 1.0 / C)
    return Workload(name, T, C, D, Ns, Phi, off, y, z, labels, sig, beta, pi, K, cg_tol,
                    cg_max_iter, em_iters, seed)


@dataclass
class FourierWorkload:
    """The paper's own sensing setup (Sec. 4): Phi_t = Omega_t F with F the unitary D x D DFT
    and Omega_t a random row subset (N_t frequencies) of the identity; z_t real and sparse;
    y_t = Phi_t z_t + eps_t with complex noise whose real and imaginary parts are each
    N(0, sigma^2).  Stored as a 0/1 frequency mask per task and the measured coefficients in
    ascending frequency order."""

    name: str
    T: int
    C: int
    D: int
    N: np.ndarray                 # int64 [T], frequencies sampled per task
    mask: np.ndarray              # uint8 [T, D]
    y: np.ndarray                 # complex64 [sum N_t], task t's in ascending frequency order
    row_off: np.ndarray           # int64 [T+1] into y
    z: np.ndarray                 # float32 [T, D]
    labels: np.ndarray            # int64 [T]
    sigma: float
    beta: float
    pi: np.ndarray
    K: int
    cg_tol: float
    cg_max_iter: int
    em_iters: int
    seed: int

    def freqs(self, t: int) -> np.ndarray:
        return np.nonzero(self.mask[t])[0]

    def yt(self, t: int) -> np.ndarray:
        return self.y[self.row_off[t]:self.row_off[t + 1]]

    def phi_real(self, t: int) -> np.ndarray:
        """The real [Re Phi_t; Im Phi_t] (2 N_t x D, FP64) whose normal equations are those of
        the complex model with real z: A = beta Re(Phi^H Phi) + diag(alpha)."""
        k = self.freqs(t).astype(np.float64)
        d = np.arange(self.D, dtype=np.float64)
        ang = -2.0 * np.pi * np.outer(k, d) / self.D
        s = 1.0 / np.sqrt(self.D)
        return np.concatenate([np.cos(ang) * s, np.sin(ang) * s], axis=0)

    def y_real(self, t: int) -> np.ndarray:
        yt = self.yt(t)
        return np.concatenate([yt.real.astype(np.float64), yt.imag.astype(np.float64)])

    def subset(self, tasks) -> "FourierWorkload":
        """The workload restricted to the given tasks (same masks, measurements and labels)."""
        tasks = np.asarray(list(tasks), dtype=np.int64)
        N = self.N[tasks]
        off = np.concatenate([[0], np.cumsum(N)]).astype(np.int64)
        y = np.concatenate([self.yt(int(t)) for t in tasks]) if len(tasks) else self.y[:0]
        return FourierWorkload(f"{self.name}[{len(tasks)}]", len(tasks), self.C, self.D, N,
                               self.mask[tasks].copy(), y, off, self.z[tasks].copy(),
                               self.labels[tasks].copy(), self.sigma, self.beta, self.pi.copy(),
                               self.K, self.cg_tol, self.cg_max_iter, self.em_iters, self.seed)


def make_fourier(name: str, T: int, C: int, D: int, N: int, *, sparsity: float = 0.05,
                 perturb: float = 0.0, sigma: float = 0.05, gt_clusters: int = None,
                 K: int = 15, cg_tol: float = 1e-5, cg_max_iter: int = 50, em_iters: int = 50,
                 seed: int = 0) -> FourierWorkload:
    """Generate a Fourier workload (supports and values as in ``make_workload``)."""
    G = gt_clusters if gt_clusters is not None else C
    sizes = _group_sizes(T, G, "equal", _rng(seed, _TAG_SIZES))
    labels = np.repeat(np.arange(G, dtype=np.int64), sizes)
    nnz = max(1, int(round(sparsity * D)))
    r_sup = _rng(seed, _TAG_SUPPORT)
    cluster_support = [np.sort(r_sup.choice(D, size=nnz, replace=False)) for _ in range(G)]
    n_swap = int(round(perturb * nnz))
    r_val = _rng(seed, _TAG_VALUES)
    z = np.zeros((T, D), dtype=np.float32)
    for t in range(T):
        sup = cluster_support[labels[t]].copy()
        if n_swap > 0:
            drop = r_sup.choice(nnz, size=n_swap, replace=False)
            outside = np.setdiff1d(np.arange(D), sup, assume_unique=True)
            sup[drop] = r_sup.choice(outside, size=n_swap, replace=False)
        z[t, sup] = r_val.standard_normal(nnz).astype(np.float32)
    r_mask = _rng(seed, _TAG_PHI)
    mask = np.zeros((T, D), dtype=np.uint8)
    for t in range(T):
        mask[t, r_mask.choice(D, size=N, replace=False)] = 1
    r_noise = _rng(seed, _TAG_NOISE)
    off = np.arange(T + 1, dtype=np.int64) * N
    y = np.empty(T * N, dtype=np.complex64)
    for t in range(T):
        spec = np.fft.fft(z[t].astype(np.float64)) / np.sqrt(D)
        k = np.nonzero(mask[t])[0]
        noise = sigma * (r_noise.standard_normal(N) + 1j * r_noise.standard_normal(N))
        y[off[t]:off[t + 1]] = (spec[k] + noise).astype(np.complex64)
    return FourierWorkload(name, T, C, D, np.full(T, N, dtype=np.int64), mask, y, off, z, labels,
                           sigma, 1.0 / sigma ** 2, np.full(C, 1.0 / C), K, cg_tol, cg_max_iter,
                           em_iters, seed)


def fourier_small(seed: int = 0) -> FourierWorkload:
    """T=4, C=2, D=256, N=64 (D/4); 5% sparsity in 2 clusters of 2 tasks; sigma 0.05; K=15;
    CG tol 1e-8 (max 100)."""
    return make_fourier("fourier-small", 4, 2, 256, 64, K=15, cg_tol=1e-8, cg_max_iter=100,
                        em_iters=10, seed=seed)


def fourier(seed: int = 0) -> FourierWorkload:
    """The paper's Fourier setting at D=8192: T=40 tasks in 4 clusters, N = D/4, 5% sparsity,
    10% per-task support perturbation, sigma 0.05, K=15 probes, U=50 CG steps (tol 1e-5)."""
    return make_fourier("fourier", 40, 4, 8192, 2048, perturb=0.10, K=15, cg_tol=1e-5,
                        cg_max_iter=50, em_iters=50, seed=seed)


def fourier_2k(seed: int = 0) -> FourierWorkload:
    """A length that is not a power of two (D = 2000 = 2^4 5^3): T=4, C=2, N=500 (D/4); 5%
    sparsity; sigma 0.05; K=15; CG tol 1e-8 (max 100)."""
    return make_fourier("fourier-2k", 4, 2, 2000, 500, K=15, cg_tol=1e-8, cg_max_iter=100,
                        em_iters=10, seed=seed)


def fourier_16k(seed: int = 0) -> FourierWorkload:
    """The Sec. 4 setting of ``fourier`` at D = 16384 (N = 4096)."""
    return make_fourier("fourier-16k", 40, 4, 16384, 4096, perturb=0.10, K=15, cg_tol=1e-5,
                        cg_max_iter=50, em_iters=50, seed=seed)


def fourier_100k(seed: int = 0) -> FourierWorkload:
    """The Sec. 4 setting of ``fourier`` at the largest length of the paper's timings,
    D = 100,000 = 2^5 5^5 (N = 25,000)."""
    return make_fourier("fourier-100k", 40, 4, 100000, 25000, perturb=0.10, K=15, cg_tol=1e-5,
                        cg_max_iter=50, em_iters=50, seed=seed)


def uniform_alpha(C: int, D: int, seed: int, tag: int = _TAG_ALPHA) -> np.ndarray:
    """A seeded Uniform(0,1) state for alpha (FP32 values), for tests that start from a
    given alpha instead of the library's own initial draw."""
    a = _rng(seed, tag).uniform(0.0, 1.0, size=(C, D)).astype(np.float32)
    return np.maximum(a, np.float32(1e-6))


# The five workload shapes the implementation is exercised on.
def plain_small(seed: int = 0) -> Workload:
    """T=4, C=2, D=256, N=64; 10 nonzeros shared within 2 clusters of 2 tasks; sigma 0.01;
    K=20 probes, CG tol 1e-8 (max 100), 10 EM iterations."""
    return make_workload("plain-small", 4, 2, 256, 64, nnz=10, sigma=0.01, K=20, cg_tol=1e-8,
                         cg_max_iter=100, em_iters=10, seed=seed)


def plain_scale(seed: int = 0) -> Workload:
    """T=32, C=4, D=8192, N=2048; 2% sparsity, supports per cluster of 8 tasks with 10% per-task
    perturbation; sigma 0.01; K=32, CG tol 1e-5, 50 EM iterations."""
    return make_workload("plain-scale", 32, 4, 8192, 2048, sparsity=0.02, perturb=0.10,
                         sigma=0.01, K=32, cg_tol=1e-5, cg_max_iter=100, em_iters=50, seed=seed)


def batching(seed: int = 0) -> Workload:
    """T=256, N_t ~ U[256, 2048], D=4096, C=8; Dirichlet(1) cluster sizes; 1% sparsity;
    sigma_t ~ U[0.005, 0.05]; K=16."""
    return make_workload("batching", 256, 8, 4096, (256, 2048), sparsity=0.01, perturb=0.0,
                         sigma=(0.005, 0.05), proportions="dirichlet", K=16, cg_tol=1e-5,
                         cg_max_iter=100, em_iters=10, seed=seed)


def precision(seed: int = 0) -> Workload:
    """T=16, C=4, D=16384, N=4096; 0.5% sparsity; sigma 0.01; K=64; 30 EM iterations."""
    return make_workload("precision", 16, 4, 16384, 4096, sparsity=0.005, perturb=0.0,
                         sigma=0.01, K=64, cg_tol=1e-5, cg_max_iter=100, em_iters=30, seed=seed)


def differentiation(seed: int = 0) -> Workload:
    """T=64, C=4, D=2048, N=512; K=32."""
    return make_workload("differentiation", 64, 4, 2048, 512, sparsity=0.02, perturb=0.0,
                         sigma=0.01, K=32, cg_tol=1e-5, cg_max_iter=100, em_iters=10, seed=seed)


WORKLOADS = {
    "plain-small": plain_small,
    "plain-scale": plain_scale,
    "batching": batching,
    "precision": precision,
    "differentiation": differentiation,
    "fourier-small": fourier_small,
    "fourier": fourier,
    "fourier-2k": fourier_2k,
    "fourier-16k": fourier_16k,
    "fourier-100k": fourier_100k,
}
