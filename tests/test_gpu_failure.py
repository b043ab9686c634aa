"""Failure detection without a GPU fault: a device-side wait that can never complete gives up
after its wall-time limit, the kernel takes its abort path and frees its tensor memory, the
call returns CMCS_ERR_TIMEOUT, and the same context then runs normally again."""
import numpy as np
import pytest

from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import make_ctx

pytestmark = pytest.mark.gpu


def test_stuck_wait_times_out_and_context_recovers():
    wl = synth.make_workload("stall", 2, 2, 256, 128, nnz=8, sigma=0.01, K=4, cg_tol=1e-5,
                             cg_max_iter=20, seed=3)
    with make_ctx(wl, precision="bf16x3", refine_max=2, graphs=True) as ctx:
        ctx.estep()
        mu_ok = ctx.read(cmcs.OUT_MU)
        ctx.test_stall(True)
        with pytest.raises(cmcs.CmcsError) as ei:
            ctx.estep()
        assert ei.value.status == cmcs.ERR_TIMEOUT
        ctx.test_stall(False)
        ctx.estep()
        assert np.array_equal(ctx.read(cmcs.OUT_MU), mu_ok)


def test_stall_hook_needs_the_tensor_core_path():
    wl = synth.make_workload("stall", 1, 1, 128, 64, nnz=4, sigma=0.01, K=2, seed=3)
    with make_ctx(wl, precision="fp32") as ctx:
        with pytest.raises(cmcs.CmcsError) as ei:
            ctx.test_stall(True)
        assert ei.value.status == cmcs.ERR_UNSUPPORTED
