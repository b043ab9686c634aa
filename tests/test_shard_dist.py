"""EM with the tasks split across ranks (paper_2310_00420_gb300.shard, Sec. 3.3), on CPU
processes joined by gloo.  Each rank drives a stand-in context whose E-step is the FP64
oracle's on its own task range (probes keyed by the global task index) and whose M-step sums
the gathered per-task rows in task order, as cmcs_mstep_apply does.  Two ranks must reach the
one-rank alpha, priors and responsibilities bit for bit, and both must follow the oracle's own
unsplit EM loop."""
import os
import socket
import tempfile

import numpy as np
import pytest

from oracle import cofem
from paper_2310_00420_gb300 import shard, synth

N_ITERS = 3


class OracleShard:
    """CPU stand-in for a cmcs context holding tasks [t0, t1) of a workload: estep() runs the
    oracle's E-step (Alg. 2 inner loop) for those tasks, mstep_terms() returns the rows of
    cmcs_mstep_terms (q_tc, q_tc max(mu^2 + s, 0), the task's log-likelihood term) and
    mstep_apply() is cmcs_mstep_apply's M-step (Eq. 5, learned priors) with ordered sums."""

    def __init__(self, wl, t0, t1, learn_pi=False):
        self.wl, self.t0, self.t1 = wl, t0, t1
        self.P = [wl.phi(t).astype(np.float64) for t in range(t0, t1)]
        self.Y = [wl.yt(t).astype(np.float64) for t in range(t0, t1)]
        from oracle import philox
        self.alpha = philox.alpha_init(wl.seed, wl.C, wl.D)
        self.pi = np.asarray(wl.pi, dtype=np.float64).copy()
        self.learn_pi = learn_pi
        self.it = 0
        self.est = None
        self.loglik = None

    def estep(self):
        wl = self.wl
        self.est = cofem.cofem_estep(self.P, self.Y, self.alpha, self.pi, wl.beta, wl.K, wl.seed,
                                     self.it, wl.cg_tol, wl.cg_max_iter,
                                     tasks=range(self.t0, self.t1), C_total=wl.C,
                                     refine_tol=1e-10, refine_max=20)

    def mstep_terms(self, device=False):
        wl, e = self.wl, self.est
        C, D = wl.C, wl.D
        W = C * (D + 1) + 1
        rows = np.zeros((self.t1 - self.t0, W))
        z = 0.5 * e["ell"] + np.log(self.pi)[None, :]
        for i in range(self.t1 - self.t0):
            for c in range(C):
                q = e["q"][i, c]
                rows[i, c * (D + 1)] = q
                rows[i, c * (D + 1) + 1: (c + 1) * (D + 1)] = q * np.maximum(
                    e["mu"][i, c] ** 2 + e["s"][i, c], 0.0)
            m = z[i].max()
            rows[i, C * (D + 1)] = m + np.log(np.exp(z[i] - m).sum()) - cofem.task_const(self.Y[i],
                                                                                       wl.beta)
        return rows

    def mstep_apply(self, terms):
        wl = self.wl
        C, D = wl.C, wl.D
        assert terms.shape == (wl.T, C * (D + 1) + 1)
        new = self.alpha.copy()
        for c in range(C):
            num, den = 0.0, np.zeros(D)
            for t in range(wl.T):               # in task order, as the library sums
                num += terms[t, c * (D + 1)]
                den += terms[t, c * (D + 1) + 1: (c + 1) * (D + 1)]
            if num < 1e-300:
                continue
            with np.errstate(divide="ignore"):
                a = num / den
            a = np.where(den <= num / 1e10, 1e10, a)
            new[c] = np.clip(a, 1e-10, 1e10)
        ll = 0.0
        for t in range(wl.T):
            ll += terms[t, C * (D + 1)]
        self.loglik = ll / wl.T
        if self.learn_pi:
            pi = np.array([max(sum(terms[t, c * (D + 1)] for t in range(wl.T)) / wl.T, 1e-300)
                           for c in range(C)])
            self.pi = pi / pi.sum()
        self.alpha = new
        self.it += 1


def _workload():
    return synth.make_workload("shard", 5, 2, 128, (24, 64), nnz=6, sigma=0.01, K=6,
                               cg_tol=1e-6, cg_max_iter=40, seed=3)


def _run(rank, world, learn_pi, out_dir):
    wl = _workload()
    ranges = shard.partition(wl.N, world)
    t0, t1 = ranges[rank]
    ctx = OracleShard(wl, t0, t1, learn_pi=learn_pi)
    em = shard.ShardedEM(ctx, ranges, rank, device=False)
    em.em_iter(N_ITERS)
    np.savez(os.path.join(out_dir, f"r{world}_{rank}.npz"), alpha=ctx.alpha, pi=ctx.pi,
             q=ctx.est["q"], loglik=ctx.loglik, t0=t0, t1=t1)


def _worker(rank, world, port, learn_pi, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _run(rank, world, learn_pi, out_dir)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_is_contiguous_and_balanced():
    N = np.array([256, 2048, 300, 1800, 512, 512, 1024, 700])
    for world in (1, 2, 3, 4, 8):
        r = shard.partition(N, world)
        assert r[0][0] == 0 and r[-1][1] == len(N)
        assert all(a < b for a, b in r) and all(r[i][1] == r[i + 1][0] for i in range(world - 1))
        if world == 2:
            loads = [N[a:b].sum() for a, b in r]
            assert max(loads) - min(loads) <= N.max()
    with pytest.raises(ValueError):
        shard.partition(N, 9)


@pytest.mark.parametrize("learn_pi", [False, True])
def test_two_ranks_match_one_rank_bit_for_bit(learn_pi):
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        _worker(0, 1, _free_port(), learn_pi, d)
        mp.spawn(_worker, args=(2, _free_port(), learn_pi, d), nprocs=2, join=True)
        one = np.load(os.path.join(d, "r1_0.npz"))
        two = [np.load(os.path.join(d, f"r2_{r}.npz")) for r in range(2)]
        for part in two:
            assert np.array_equal(part["alpha"], one["alpha"])
            assert np.array_equal(part["pi"], one["pi"])
            assert float(part["loglik"]) == float(one["loglik"])
        q2 = np.concatenate([p["q"] for p in two], axis=0)
        assert int(two[0]["t1"]) == int(two[1]["t0"]) and 0 < int(two[0]["t1"]) < 5
        assert np.array_equal(q2, one["q"])
        # and the split EM follows the oracle's own EM loop over all tasks
        wl = _workload()
        P = [wl.phi(t).astype(np.float64) for t in range(wl.T)]
        Y = [wl.yt(t).astype(np.float64) for t in range(wl.T)]
        o = cofem.em(P, Y, wl.pi, wl.beta, N_ITERS, K=wl.K, seed=wl.seed, tol=wl.cg_tol,
                     max_iter=wl.cg_max_iter, C=wl.C, D=wl.D, refine_tol=1e-10, refine_max=20,
                     learn_pi=learn_pi)
        np.testing.assert_allclose(one["alpha"], o["alpha"], rtol=1e-10)
        np.testing.assert_allclose(one["q"], o["last"]["q"], atol=1e-12)
