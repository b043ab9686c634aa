"""The allocation-free operator entry point (cmcs_apply_noalloc), for callers that cannot call
cudaMalloc while running (their device memory belongs to their own pool allocator, or they
cannot afford cudaMalloc's implicit synchronisation).  Its output is checked against the FP64
oracle's operator (Eq. 7) and against the library's regular operator (cmcs_apply) on the same
inputs, on two calls in a row (the fixed scratch array is reused between calls)."""
import numpy as np
import pytest

from oracle import cofem
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import make_ctx, rel_err_rows, task_lists

pytestmark = pytest.mark.gpu


def test_noalloc_operator_matches_oracle_and_apply_on_two_calls():
    import torch
    wl = synth.plain_small()
    P, _ = task_lists(wl)
    R = wl.C * (wl.K + 1)
    with make_ctx(wl) as ctx:
        alpha32 = ctx.read(cmcs.OUT_ALPHA)
        alpha = torch.from_numpy(alpha32).cuda()
        phis = [torch.from_numpy(np.ascontiguousarray(wl.phi(t))).cuda() for t in range(wl.T)]
        for call in range(2):
            rng = np.random.default_rng(100 + call)
            V32 = rng.standard_normal((wl.T, R, wl.D)).astype(np.float32)
            V = torch.from_numpy(V32).cuda()
            Z_ref = ctx.apply(V).cpu().numpy()
            for t in range(wl.T):
                for c in range(wl.C):
                    js = slice(c * (wl.K + 1), (c + 1) * (wl.K + 1))
                    Z = cmcs.apply_noalloc(phis[t], alpha[c].contiguous(), wl.beta,
                                           V[t, js].contiguous()).cpu().numpy()
                    ref = cofem.apply_A(P[t], wl.beta, alpha32[c].astype(np.float64),
                                        V32[t, js].astype(np.float64).T).T
                    # FP32 GEMMs over N = 64 and D = 256 terms: 2e-6 normwise is ~30 ulps
                    err = rel_err_rows(Z, ref)
                    assert err.max() < 2e-6, (call, t, c, err.max())
                    # the regular operator's FP32 path, same bound
                    assert rel_err_rows(Z, Z_ref[t, js]).max() < 2e-6, (call, t, c)


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


def test_noalloc_rejects_host_pointers():
    """A host pointer handed to the C entry point directly is refused before any launch."""
    import ctypes
    import torch
    N, D, m = 16, 8, 2
    Phi = torch.zeros((N, D), device="cuda")
    alpha = torch.ones(D, device="cuda")
    V = torch.zeros((m, D), device="cuda")
    Zh = np.zeros((m, D), np.float32)
    st = cmcs.lib().cmcs_apply_noalloc(ctypes.c_void_p(Phi.data_ptr()), N, D,
                                       ctypes.c_void_p(alpha.data_ptr()), 1.0,
                                       ctypes.c_void_p(V.data_ptr()), m,
                                       ctypes.c_void_p(Zh.ctypes.data), None)
    assert st == cmcs.ERR_INVALID_ARG
    assert b"not device memory" in cmcs.lib().cmcs_last_error(None)
