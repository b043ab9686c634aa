"""Host-side checks of the C ABI that need no GPU: the library loads, exports every function
include/cmcs.h declares, the binding's struct layouts match the header (checked by compiling
a C probe against it), and argument validation fails cleanly before touching CUDA."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2310_00420_gb300 import cmcs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cmcs.h")


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(cmcs.LIB_PATH):
        from paper_2310_00420_gb300 import build
        build.build()
    return cmcs.lib()


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:cmcs_status|void|const char \*)\s*(cmcs_\w+)\(", txt, re.M)))


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(cmcs.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", cmcs.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    syms = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in _declared():
        assert name in syms, name
        assert hasattr(L, name)


def test_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "cmcs.h"
#define O(s, f) printf(#s "." #f " %zu\n", offsetof(s, f))
int main(void) {
  printf("cmcs_config %zu\ncmcs_summary %zu\ncmcs_profile_data %zu\n", sizeof(cmcs_config),
         sizeof(cmcs_summary), sizeof(cmcs_profile_data));
  O(cmcs_profile_data, operator_ms); O(cmcs_profile_data, operator_bytes);
  O(cmcs_profile_data, residual_ms); O(cmcs_profile_data, kernel_launches);
  O(cmcs_profile_data, operator_calls_bf16); O(cmcs_profile_data, operator_ms_bf16);
  O(cmcs_config, N); O(cmcs_config, beta); O(cmcs_config, pi); O(cmcs_config, cg_max_iter);
  O(cmcs_config, cg_tol); O(cmcs_config, seed); O(cmcs_config, precision);
  O(cmcs_config, refine_max); O(cmcs_config, refine_tol); O(cmcs_config, alpha_min);
  O(cmcs_config, alpha_max); O(cmcs_config, schedule); O(cmcs_config, graphs);
  O(cmcs_config, autotune); O(cmcs_config, learn_pi); O(cmcs_config, probe_share);
  O(cmcs_config, precond); O(cmcs_config, warm_start); O(cmcs_config, task_offset);
  O(cmcs_config, T_total); O(cmcs_config, refine_steps);
  O(cmcs_summary, loglik); O(cmcs_summary, cg_steps_max); O(cmcs_summary, cg_steps_mean);
  O(cmcs_summary, cg_capped); O(cmcs_summary, refine_sweeps_max);
  O(cmcs_summary, refine_rel_max); O(cmcs_summary, min_margin);
  O(cmcs_summary, operator_applies); O(cmcs_summary, resid_rel_max);
  O(cmcs_summary, refine_diverged); O(cmcs_summary, operator_variant);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.rsplit(" ", 1) for l in lines if l.strip())
    assert int(got["cmcs_config"]) == ctypes.sizeof(cmcs.Config)
    assert int(got["cmcs_summary"]) == ctypes.sizeof(cmcs.Summary)
    assert int(got["cmcs_profile_data"]) == ctypes.sizeof(cmcs.ProfileData)
    for key, val in got.items():
        if "." in key:
            s, f = key.split(".")
            cls = {"cmcs_config": cmcs.Config, "cmcs_summary": cmcs.Summary,
                   "cmcs_profile_data": cmcs.ProfileData}[s]
            assert getattr(cls, f).offset == int(val), key


def _cfg(**kw):
    N = np.array([64, 64], dtype=np.int64)
    pi = np.array([0.5, 0.5])
    base = dict(T=2, C=2, D=32, K=4, beta=1e4, cg_max_iter=50, cg_tol=1e-5, seed=0, precision=0,
                refine_max=0, refine_tol=1e-6, alpha_min=1e-10, alpha_max=1e10)
    base.update(kw)
    cfg = cmcs.Config(base["T"], base["C"], base["D"], base["K"],
                      N.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), base["beta"],
                      pi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), base["cg_max_iter"],
                      base["cg_tol"], base["seed"], base["precision"], base["refine_max"],
                      base["refine_tol"], base["alpha_min"], base["alpha_max"], 0, 0, 0)
    cfg.task_offset = base.get("task_offset", 0)
    cfg.T_total = base.get("T_total", 0)
    cfg.refine_steps = base.get("refine_steps", 0)
    return cfg, (N, pi)


@pytest.mark.parametrize("bad", [dict(T=0), dict(C=0), dict(D=0), dict(K=0), dict(beta=0.0),
                                 dict(beta=-1.0), dict(cg_max_iter=0), dict(cg_max_iter=513),
                                 dict(cg_tol=-1.0), dict(precision=7), dict(precision=-1), dict(refine_max=-1),
                                 dict(refine_max=65), dict(alpha_min=0.0),
                                 dict(alpha_min=2.0, alpha_max=1.0), dict(task_offset=-1),
                                 dict(T_total=-1), dict(task_offset=1, T_total=2),
                                 dict(task_offset=3), dict(refine_steps=-1),
                                 dict(refine_steps=51)])
def test_create_rejects_invalid_config_without_cuda(L, bad):
    cfg, keep = _cfg(**bad)
    phi = np.zeros((128, 32), np.float32)
    y = np.zeros(128, np.float32)
    h = ctypes.c_void_p()
    st = L.cmcs_create(ctypes.byref(cfg), phi.ctypes.data, y.ctypes.data, 0, None, ctypes.byref(h))
    assert st == cmcs.ERR_INVALID_ARG
    assert not h.value
    assert L.cmcs_last_error(None)


@pytest.mark.parametrize("flag", ["learn_pi", "probe_share", "precond", "warm_start",
                                  "schedule", "graphs", "autotune"])
def test_create_rejects_bad_switches_without_cuda(L, flag):
    """Every 0/1 switch of cmcs_config accepts only 0 and 1."""
    Phi = np.zeros((128, 32), np.float32)
    y = np.zeros(128, np.float32)
    h = ctypes.c_void_p()
    for v in (2, -1):
        cfg, keep = _cfg()
        setattr(cfg, flag, v)
        assert L.cmcs_create(ctypes.byref(cfg), Phi.ctypes.data, y.ctypes.data, 0, None,
                             ctypes.byref(h)) == cmcs.ERR_INVALID_ARG, (flag, v)
        assert not h.value


def test_create_rejects_null_inputs_and_bad_pi(L):
    cfg, keep = _cfg()
    h = ctypes.c_void_p()
    assert L.cmcs_create(ctypes.byref(cfg), None, None, 0, None, ctypes.byref(h)) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_create(None, None, None, 0, None, ctypes.byref(h)) == cmcs.ERR_INVALID_ARG
    N, pi = keep
    pi[:] = [0.7, 0.7]
    phi = np.zeros((128, 32), np.float32)
    y = np.zeros(128, np.float32)
    assert L.cmcs_create(ctypes.byref(cfg), phi.ctypes.data, y.ctypes.data, 0, None,
                         ctypes.byref(h)) == cmcs.ERR_INVALID_ARG


def test_create_dft_validates_without_cuda(L):
    """The Fourier constructor rejects a null mask, a D that is neither a power of two in
    [128, 8192] nor 2^a 5^b with 16 | D up to 2^20, and any precision but FP32, before
    touching the GPU."""
    h = ctypes.c_void_p()
    y = np.zeros((8, 2), np.float32)
    cfg, keep = _cfg(D=256)
    assert L.cmcs_create_dft(ctypes.byref(cfg), None, y.ctypes.data, 0, None,
                             ctypes.byref(h)) == cmcs.ERR_INVALID_ARG
    for bad in (dict(D=200), dict(D=64), dict(D=3072), dict(D=1 << 21), dict(D=256, precision=2),
                dict(D=100000, precision=2)):
        cfg, keep = _cfg(**bad)
        mask = np.zeros((2, cfg.D), np.uint8)
        assert L.cmcs_create_dft(ctypes.byref(cfg), mask.ctypes.data, y.ctypes.data, 0, None,
                                 ctypes.byref(h)) == cmcs.ERR_UNSUPPORTED, bad
        assert not h.value


def test_calls_on_null_context_are_rejected(L):
    assert L.cmcs_estep(None) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_em_iter(None, 1) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_read(None, 0, None, 0) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_result(None, None) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_apply(None, None, None, 0, 0) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_set_alpha(None, None, 0, 0) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_probes(None, 0, None, 0) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_lanczos_quadrature(None, None, None, 1, 1, None, None, None) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_mstep_terms(None, None, 0) == cmcs.ERR_INVALID_ARG
    assert L.cmcs_mstep_apply(None, None, 0) == cmcs.ERR_INVALID_ARG
    L.cmcs_destroy(None)


def test_apply_noalloc_binding_validates_before_calling():
    """The binding of cmcs_apply_noalloc rejects tensors whose dtype, layout, shape or device
    would make the kernels read or write out of bounds, before anything reaches the library
    (these CPU tensors never get past the checks)."""
    import torch
    from paper_2310_00420_gb300 import cmcs
    N, D, m = 6, 5, 3
    Phi = torch.zeros((N, D))
    alpha = torch.ones(D)
    V = torch.zeros((m, D))
    bad = [
        dict(Phi=Phi.double()),                       # dtype
        dict(V=torch.zeros((D, m)).t()),              # non-contiguous
        dict(Phi=torch.zeros(N * D)),                 # not 2-D
        dict(V=torch.zeros((m, D + 1))),              # columns != D
        dict(alpha=torch.ones(D - 1)),                # short alpha
        dict(Z=torch.zeros((m + 1, D))),              # Z shape
        dict(),                                       # all valid but on the host
    ]
    for over in bad:
        args = dict(Phi=Phi, alpha=alpha, V=V, Z=None)
        args.update(over)
        with pytest.raises(ValueError):
            cmcs.apply_noalloc(args["Phi"], args["alpha"], 1.0, args["V"], Z=args["Z"])
