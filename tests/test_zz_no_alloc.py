"""The allocation-free operator entry point (cmcs_apply_noalloc), for callers that cannot call
cudaMalloc while running, against the library's regular operator (cmcs_apply) on the same
inputs, on two calls in a row (the fixed scratch array is reused between calls)."""
import numpy as np
import pytest

from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import make_ctx, rel_err_rows

pytestmark = pytest.mark.gpu


def test_noalloc_operator_matches_apply_on_two_calls():
    import torch
    wl = synth.plain_small()
    R = wl.C * (wl.K + 1)
    with make_ctx(wl) as ctx:
        alpha = torch.from_numpy(ctx.read(cmcs.OUT_ALPHA)).cuda()
        phis = [torch.from_numpy(np.ascontiguousarray(wl.phi(t))).cuda() for t in range(wl.T)]
        for call in range(2):
            rng = np.random.default_rng(100 + call)
            V = torch.from_numpy(rng.standard_normal((wl.T, R, wl.D)).astype(np.float32)).cuda()
            Z_ref = ctx.apply(V).cpu().numpy()
            for t in range(wl.T):
                for c in range(wl.C):
                    js = slice(c * (wl.K + 1), (c + 1) * (wl.K + 1))
                    Vtc = V[t, js].contiguous()
                    Z = cmcs.apply_noalloc(phis[t], alpha[c].contiguous(), wl.beta, Vtc)
                    err = rel_err_rows(Z.cpu().numpy(), Z_ref[t, js])
                    # same bound as the operator-vs-oracle test: both are FP32 GEMMs
                    assert err.max() < 2e-6, (call, t, c, err.max())


def test_noalloc_rejects_oversized_request():
    import torch
    N, D = 4096, 8
    Phi = torch.zeros((N, D), device="cuda")
    alpha = torch.ones(D, device="cuda")
    V = torch.zeros((1025, D), device="cuda")            # 1025 * 4096 > 4,194,304
    with pytest.raises(cmcs.CmcsError) as ei:
        cmcs.apply_noalloc(Phi, alpha, 1.0, V)
    assert ei.value.status == cmcs.ERR_INVALID_ARG
    assert b"exceeds" in cmcs.lib().cmcs_last_error(None)
