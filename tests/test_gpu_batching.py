"""Batching: every task (uneven N_t) and every cluster and probe in one persistent launch per
operator pass, CG chunks replayed from CUDA graphs, the autotuned operator variant -- all
against the per-task launch loop and against the FP64 oracle.

The schedule, the graphs and the tuned variant change which CTA computes a tile and how the
launches are issued, not the order of any sum, so their results must be bit-identical."""
import numpy as np
import pytest

from oracle import cofem
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import make_ctx, rel_err_rows

pytestmark = pytest.mark.gpu

OUTS = dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, q=cmcs.OUT_Q, logdet=cmcs.OUT_LOGDET,
            steps=cmcs.OUT_STEPS, alpha=cmcs.OUT_ALPHA)


@pytest.fixture(scope="module")
def ragged():
    return synth.make_workload("ragged-batch", 5, 3, 520, (100, 700), nnz=12, sigma=0.01, K=6,
                               cg_tol=1e-6, cg_max_iter=60, proportions="dirichlet", seed=13)


def _run(wl, **kw):
    with make_ctx(wl, refine_max=6, refine_tol=1e-6, **kw) as ctx:
        ctx.em_iter(2)
        out = {k: ctx.read(v) for k, v in OUTS.items()}
        out["summary"] = ctx.summary()
    return out


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_graphs_schedule_and_tuning_are_bit_identical(ragged, precision):
    base = _run(ragged, precision=precision, graphs=False)
    for kw in (dict(graphs=True), dict(schedule="per_task", graphs=False),
               dict(schedule="per_task", graphs=True), dict(autotune=True)):
        other = _run(ragged, precision=precision, **kw)
        for k in OUTS:
            assert np.array_equal(base[k], other[k]), (precision, kw, k)
    assert base["summary"]["operator_variant"] > 0


@pytest.fixture(scope="module")
def batching():
    return synth.batching()


def test_batching_workload_sampled_parity(batching):
    """T=256 tasks with N_t ~ U[256, 2048], D=4096, C=8, K=16, one launch per pass over all
    tasks (tensor-core operator, refinement as in the benchmark); sampled pairs vs the oracle."""
    wl = batching
    assert wl.N.min() < 512 and wl.N.max() > 1800
    with make_ctx(wl, precision="bf16x3", refine_max=8, refine_tol=1e-5) as ctx:
        ctx.estep()
        alpha = ctx.read(cmcs.OUT_ALPHA)
        g = {k: ctx.read(v) for k, v in dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, logdet=cmcs.OUT_LOGDET,
                                              steps=cmcs.OUT_STEPS, gamma=cmcs.OUT_GAMMA,
                                              xi=cmcs.OUT_XI, q=cmcs.OUT_Q).items()}
    np.testing.assert_allclose(g["q"].sum(axis=1), 1.0, atol=1e-12)
    t_short = int(np.argmin(wl.N))
    t_long = int(np.argmax(wl.N))
    for t, c in [(t_short, 1), (t_long, 6)]:
        o = cofem.cofem_estep([wl.phi(t).astype(np.float64)], [wl.yt(t).astype(np.float64)],
                              alpha[c:c + 1].astype(np.float64), np.array([1.0]), wl.beta, wl.K,
                              wl.seed, 0, wl.cg_tol, wl.cg_max_iter, tasks=[t], clusters=[c],
                              C_total=wl.C, refine_tol=1e-12, refine_max=40)
        assert rel_err_rows(g["mu"][t, c], o["mu"][0, 0]) <= 1e-4, (t, c)
        assert rel_err_rows(g["s"][t, c], o["s"][0, 0]) <= 1e-4, (t, c)
        nu = cofem.logdet_estimate(g["gamma"][t, c].astype(np.float64),
                                   g["xi"][t, c].astype(np.float64), g["steps"][t, c, 1:], wl.D)
        assert abs(g["logdet"][t, c] - nu) <= 1e-9 * abs(nu)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_profiling_with_graphs(ragged, precision):
    """Operator timing with captured graphs: events become graph nodes; results unchanged."""
    base = _run(ragged, precision=precision, graphs=False)
    with make_ctx(ragged, refine_max=6, refine_tol=1e-6, precision=precision, graphs=True) as ctx:
        ctx.profile(True)
        ctx.em_iter(2)
        prof = ctx.profile_read()
        mu = ctx.read(cmcs.OUT_MU)
    assert np.array_equal(mu, base["mu"])
    assert prof["operator_calls"] > 0 and prof["operator_ms"] > 0
    assert prof["operator_flops"] > 0 and prof["kernel_launches"] > prof["operator_calls"]
