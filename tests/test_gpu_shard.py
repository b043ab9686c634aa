"""EM with the tasks split across contexts (Sec. 3.3) on the GPU: contexts holding disjoint
task ranges (task_offset, T_total), whose per-task M-step rows (cmcs_mstep_terms) are stacked
in task order and applied by each (cmcs_mstep_apply), reach the alpha, responsibilities,
assignments and means of one context holding every task bit for bit.  The contexts share one
GPU and run one after another (no kernel waits on another context); the exchange between
GPUs is the all-gather of shard.ShardedEM, tested on CPU ranks in test_shard_dist.py."""
import numpy as np
import pytest

from paper_2310_00420_gb300 import cmcs, shard, synth

pytestmark = pytest.mark.gpu


def _ctx_range(wl, t0, t1, **kw):
    import torch
    sub = wl.subset(range(t0, t1))
    return cmcs.Context(torch.from_numpy(sub.Phi).cuda(), torch.from_numpy(sub.y).cuda(), sub.N,
                        C=wl.C, K=wl.K, beta=wl.beta, pi=wl.pi, cg_max_iter=wl.cg_max_iter,
                        cg_tol=wl.cg_tol, seed=wl.seed, task_offset=t0, T_total=wl.T, **kw)


@pytest.mark.parametrize("precision, learn_pi", [("fp32", False), ("bf16x3", True)])
def test_split_contexts_match_one_context(precision, learn_pi):
    import torch
    wl = synth.make_workload("shard", 6, 3, 384, (48, 300), nnz=8, sigma=0.01, K=7,
                             cg_tol=1e-6, cg_max_iter=60, seed=5)
    kw = dict(precision=precision, refine_max=8, refine_tol=1e-6, learn_pi=learn_pi)
    n = 3
    with cmcs.Context.from_workload(wl, device=True, **kw) as whole:
        whole.em_iter(n)
        ref = {w: whole.read(w) for w in (cmcs.OUT_ALPHA, cmcs.OUT_Q, cmcs.OUT_ASSIGN,
                                          cmcs.OUT_MU, cmcs.OUT_S, cmcs.OUT_PI)}
        ref_ll = whole.summary()["loglik"]
    ranges = shard.partition(wl.N, 2)
    parts = [_ctx_range(wl, a, b, **kw) for a, b in ranges]
    try:
        with pytest.raises(cmcs.CmcsError):
            parts[0].em_iter(1)                     # a context with part of the tasks refuses
        for _ in range(n):
            rows = []
            for p in parts:
                p.estep()
                rows.append(p.mstep_terms(device=True))
            full = torch.cat(rows, dim=0).contiguous()
            for p in parts:
                p.mstep_apply(full)
        for w in (cmcs.OUT_ALPHA, cmcs.OUT_PI):
            for p in parts:
                assert np.array_equal(p.read(w), ref[w]), w
        for w in (cmcs.OUT_Q, cmcs.OUT_ASSIGN, cmcs.OUT_MU, cmcs.OUT_S):
            got = np.concatenate([p.read(w) for p in parts], axis=0)
            assert np.array_equal(got, ref[w]), w
        for p in parts:
            assert p.summary()["loglik"] == ref_ll
            assert p.summary()["em_iters_done"] == n
    finally:
        for p in parts:
            p.close()


def test_probes_follow_the_global_task_index():
    wl = synth.plain_small()
    with cmcs.Context.from_workload(wl, device=True) as whole, _ctx_range(wl, 2, 4) as part:
        assert np.array_equal(part.probes(3), whole.probes(3)[2:4])
