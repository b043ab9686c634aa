"""ctypes binding of libcmcs.so (include/cmcs.h): argument marshalling only.

Every step of the E-step and M-step runs inside the library's CUDA kernels.  Host arrays are
numpy; device arrays are torch CUDA tensors (PyTorch supplies device memory and streams).
The library must be built (``paper_2310_00420_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcmcs.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NUMERIC, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NUMERIC", 5: "TIMEOUT",
                6: "UNSUPPORTED"}
FP32, BF16_REFINE, BF16X3, BF16_MIXED = 0, 1, 2, 3
PRECISIONS = {"fp32": FP32, "bf16": BF16_REFINE, "bf16_refine": BF16_REFINE, "bf16x3": BF16X3,
              "bf16_mixed": BF16_MIXED}

(OUT_MU, OUT_S, OUT_Q, OUT_LOGDET, OUT_ELL, OUT_ALPHA, OUT_ASSIGN, OUT_RECON, OUT_STEPS,
 OUT_GAMMA, OUT_XI, OUT_B0, OUT_SWEEPS, OUT_RESID, OUT_PI) = range(15)

# exported symbols, in the order include/cmcs.h declares them
EXPORTS = ("cmcs_create", "cmcs_create_dft", "cmcs_set_alpha", "cmcs_estep", "cmcs_em_iter", "cmcs_read",
           "cmcs_result", "cmcs_apply", "cmcs_probes", "cmcs_lanczos_quadrature",
           "cmcs_profile", "cmcs_profile_read", "cmcs_apply_noalloc", "cmcs_set_data",
           "cmcs_adjoint", "cmcs_test_stall", "cmcs_mstep_terms", "cmcs_mstep_apply",
           "cmcs_last_error", "cmcs_destroy")


class Config(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("C", ctypes.c_int), ("D", ctypes.c_int), ("K", ctypes.c_int),
                ("N", ctypes.POINTER(ctypes.c_int64)), ("beta", ctypes.c_double),
                ("pi", ctypes.POINTER(ctypes.c_double)), ("cg_max_iter", ctypes.c_int),
                ("cg_tol", ctypes.c_double), ("seed", ctypes.c_uint64), ("precision", ctypes.c_int),
                ("refine_max", ctypes.c_int), ("refine_tol", ctypes.c_double),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("schedule", ctypes.c_int), ("graphs", ctypes.c_int), ("autotune", ctypes.c_int),
                ("learn_pi", ctypes.c_int), ("probe_share", ctypes.c_int),
                ("precond", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("task_offset", ctypes.c_int), ("T_total", ctypes.c_int),
                ("refine_steps", ctypes.c_int)]


class Summary(ctypes.Structure):
    _fields_ = [("em_iters_done", ctypes.c_int64), ("loglik", ctypes.c_double),
                ("cg_steps_max", ctypes.c_int), ("cg_steps_mean", ctypes.c_double),
                ("cg_capped", ctypes.c_int64), ("refine_sweeps_max", ctypes.c_int),
                ("refine_rel_max", ctypes.c_double), ("min_margin", ctypes.c_double),
                ("operator_applies", ctypes.c_int64), ("resid_rel_max", ctypes.c_double),
                ("refine_diverged", ctypes.c_int64), ("operator_variant", ctypes.c_int)]


class ProfileData(ctypes.Structure):
    _fields_ = [("operator_calls", ctypes.c_int64), ("operator_ms", ctypes.c_double),
                ("operator_flops", ctypes.c_double), ("operator_bytes", ctypes.c_double),
                ("residual_calls", ctypes.c_int64), ("residual_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("operator_calls_bf16", ctypes.c_int64),
                ("operator_ms_bf16", ctypes.c_double)]


class CmcsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cmcs {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libcmcs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2310_00420_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, i64, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int
    L.cmcs_create.argtypes = [ctypes.POINTER(Config), vp, vp, i, vp, ctypes.POINTER(vp)]
    L.cmcs_create_dft.argtypes = [ctypes.POINTER(Config), vp, vp, i, vp, ctypes.POINTER(vp)]
    L.cmcs_set_alpha.argtypes = [vp, vp, i, i64]
    L.cmcs_estep.argtypes = [vp]
    L.cmcs_em_iter.argtypes = [vp, i]
    L.cmcs_read.argtypes = [vp, i, vp, i]
    L.cmcs_result.argtypes = [vp, ctypes.POINTER(Summary)]
    L.cmcs_apply.argtypes = [vp, vp, vp, i, i]
    L.cmcs_probes.argtypes = [vp, i64, vp, i]
    L.cmcs_lanczos_quadrature.argtypes = [vp, vp, vp, i, i, vp, vp, vp]
    L.cmcs_profile.argtypes = [vp, i]
    L.cmcs_profile_read.argtypes = [vp, ctypes.POINTER(ProfileData)]
    L.cmcs_apply_noalloc.argtypes = [vp, i, i, vp, ctypes.c_double, vp, i, vp, vp]
    L.cmcs_set_data.argtypes = [vp, vp, vp, i]
    L.cmcs_adjoint.argtypes = [vp, vp, vp, vp, vp, i]
    L.cmcs_test_stall.argtypes = [vp, i]
    L.cmcs_mstep_terms.argtypes = [vp, vp, i]
    L.cmcs_mstep_apply.argtypes = [vp, vp, i]
    L.cmcs_last_error.argtypes = [vp]
    L.cmcs_last_error.restype = ctypes.c_char_p
    L.cmcs_destroy.argtypes = [vp]
    L.cmcs_destroy.restype = None
    for name in EXPORTS:
        if name not in ("cmcs_last_error", "cmcs_destroy"):
            getattr(L, name).restype = st
    _lib = L
    return L


def _check(status: int, handle=None):
    if status != OK:
        msg = lib().cmcs_last_error(handle).decode(errors="replace")
        raise CmcsError(status, msg)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, on_device) of a contiguous numpy array or torch tensor."""
    if _is_torch(a):
        assert a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0)
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data), 0


def _stream_handle(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return ctypes.c_void_p(0)


_OUT_META = {  # what: (dtype, shape function of (T, C, D, K, U))
    OUT_MU: (np.float32, lambda T, C, D, K, U: (T, C, D)),
    OUT_S: (np.float32, lambda T, C, D, K, U: (T, C, D)),
    OUT_Q: (np.float64, lambda T, C, D, K, U: (T, C)),
    OUT_LOGDET: (np.float64, lambda T, C, D, K, U: (T, C)),
    OUT_ELL: (np.float64, lambda T, C, D, K, U: (T, C)),
    OUT_ALPHA: (np.float32, lambda T, C, D, K, U: (C, D)),
    OUT_ASSIGN: (np.int32, lambda T, C, D, K, U: (T,)),
    OUT_RECON: (np.float32, lambda T, C, D, K, U: (T, D)),
    OUT_STEPS: (np.int32, lambda T, C, D, K, U: (T, C, K + 1)),
    OUT_GAMMA: (np.float32, lambda T, C, D, K, U: (T, C, K, U)),
    OUT_XI: (np.float32, lambda T, C, D, K, U: (T, C, K, U)),
    OUT_B0: (np.float32, lambda T, C, D, K, U: (T, D)),
    OUT_SWEEPS: (np.int32, lambda T, C, D, K, U: (T, C, K + 1)),
    OUT_RESID: (np.float32, lambda T, C, D, K, U: (T, C, K + 1)),
    OUT_PI: (np.float64, lambda T, C, D, K, U: (C,)),
}


class Context:
    """One CoFEM problem resident on the GPU (cmcs_create ... cmcs_destroy)."""

    def __init__(self, Phi, y, N, *, C: int, K: int, beta: float, pi=None, cg_max_iter: int = 100,
                 cg_tol: float = 1e-5, seed: int = 0, precision="fp32", refine_max: int = 0,
                 refine_tol: float = 1e-6, alpha_min: float = 1e-10, alpha_max: float = 1e10,
                 schedule: str = "batched", graphs: bool = True, autotune: bool = False,
                 learn_pi: bool = False, probe_share: bool = False, precond: bool = False,
                 warm_start: bool = False, task_offset: int = 0, T_total: int = 0,
                 refine_steps: int = 0, mask=None, stream=None):
        """Dense Phi [sum N_t][D] with y [sum N_t]; or, with Phi None and mask given, the
        Fourier operator of cmcs_create_dft: mask uint8 [T][D], y float32 [sum N_t][2].
        learn_pi, probe_share, precond and warm_start switch on the method variants of
        cmcs_config; task_offset and T_total place the context's tasks in a problem whose tasks
        are split across contexts (see shard.py)."""
        N = np.ascontiguousarray(np.asarray(N, dtype=np.int64))
        D = int(mask.shape[1]) if mask is not None else int(Phi.shape[1])
        self.T, self.C, self.D, self.K = int(len(N)), int(C), D, int(K)
        self.task_offset = int(task_offset)
        self.T_total = int(T_total) if T_total else self.T
        self.U = int(cg_max_iter)
        pi = np.full(C, 1.0 / C) if pi is None else np.ascontiguousarray(np.asarray(pi, np.float64))
        self._N, self._pi = N, pi                     # keep alive during create
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg = Config(self.T, self.C, self.D, self.K,
                     N.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(beta),
                     pi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(cg_max_iter),
                     float(cg_tol), int(seed) & (2**64 - 1), prec, int(refine_max),
                     float(refine_tol), float(alpha_min), float(alpha_max),
                     {"batched": 0, "per_task": 1}[schedule], 1 if graphs else 0,
                     1 if autotune else 0, 1 if learn_pi else 0, 1 if probe_share else 0,
                     1 if precond else 0, 1 if warm_start else 0, int(task_offset), int(T_total),
                     int(refine_steps))
        self.cfg = cfg
        self.fourier = mask is not None
        p_phi, dev1 = _ptr(mask if self.fourier else Phi)
        p_y, dev2 = _ptr(y)
        if dev1 != dev2:
            raise ValueError("Phi (or mask) and y must both be host arrays or both device tensors")
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        create = lib().cmcs_create_dft if self.fourier else lib().cmcs_create
        _check(create(ctypes.byref(cfg), p_phi, p_y, dev1, self._stream, ctypes.byref(h)))
        self.h = h

    @classmethod
    def from_workload(cls, wl, device: bool = True, **kw):
        args = dict(C=wl.C, K=wl.K, beta=wl.beta, pi=wl.pi, cg_max_iter=wl.cg_max_iter,
                    cg_tol=wl.cg_tol, seed=wl.seed)
        args.update(kw)
        Phi, y = wl.Phi, wl.y
        if device:
            import torch
            Phi = torch.from_numpy(Phi).cuda()
            y = torch.from_numpy(y).cuda()
        return cls(Phi, y, wl.N, **args)

    @classmethod
    def from_fourier(cls, wl, device: bool = True, **kw):
        """A context for a synth.FourierWorkload (Phi_t = Omega_t F, cmcs_create_dft)."""
        args = dict(C=wl.C, K=wl.K, beta=wl.beta, pi=wl.pi, cg_max_iter=wl.cg_max_iter,
                    cg_tol=wl.cg_tol, seed=wl.seed)
        args.update(kw)
        mask = np.ascontiguousarray(wl.mask.astype(np.uint8))
        y = np.ascontiguousarray(np.stack([wl.y.real, wl.y.imag], axis=-1).astype(np.float32))
        if device:
            import torch
            mask = torch.from_numpy(mask).cuda()
            y = torch.from_numpy(y).cuda()
        return cls(None, y, wl.N, mask=mask, **args)

    # ---- lifecycle ----
    def close(self):
        if getattr(self, "h", None):
            lib().cmcs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- calls ----
    def estep(self):
        _check(lib().cmcs_estep(self.h), self.h)

    def em_iter(self, n: int = 1):
        _check(lib().cmcs_em_iter(self.h, int(n)), self.h)

    def set_alpha(self, alpha, em_iter: int = 0):
        if not _is_torch(alpha):
            alpha = np.ascontiguousarray(np.asarray(alpha, dtype=np.float32))
        p, dev = _ptr(alpha)
        _check(lib().cmcs_set_alpha(self.h, p, dev, int(em_iter)), self.h)

    def read(self, what: int, out=None, device: bool = False):
        dt, shp = _OUT_META[what]
        shape = shp(self.T, self.C, self.D, self.K, self.U)
        if out is None:
            if device:
                import torch
                tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dt]
                out = torch.empty(shape, dtype=tdt, device="cuda")
            else:
                out = np.empty(shape, dtype=dt)
        p, dev = _ptr(out)
        _check(lib().cmcs_read(self.h, int(what), p, dev), self.h)
        return out

    def summary(self) -> dict:
        s = Summary()
        _check(lib().cmcs_result(self.h, ctypes.byref(s)), self.h)
        return {f: getattr(s, f) for f, _ in Summary._fields_}

    def set_data(self, Phi, y):
        p_phi, dev1 = _ptr(Phi)
        p_y, dev2 = _ptr(y)
        if dev1 != dev2:
            raise ValueError("Phi and y must both be host arrays or both device tensors")
        _check(lib().cmcs_set_data(self.h, p_phi, p_y, dev1), self.h)

    def adjoint(self, g, with_phi: bool = True):
        """(dy, dalpha, dPhi) for g = dL/dmu [T][C][D] (float32; numpy or CUDA tensor)."""
        n_rows = int(self._N.sum())
        if _is_torch(g):
            import torch
            dev = g.device
            dy = torch.empty(n_rows, dtype=torch.float32, device=dev)
            da = torch.empty((self.C, self.D), dtype=torch.float32, device=dev)
            dP = torch.empty((n_rows, self.D), dtype=torch.float32, device=dev) if with_phi else None
        else:
            g = np.ascontiguousarray(g, dtype=np.float32)
            dy = np.empty(n_rows, np.float32)
            da = np.empty((self.C, self.D), np.float32)
            dP = np.empty((n_rows, self.D), np.float32) if with_phi else None
        pg, dev = _ptr(g)
        _check(lib().cmcs_adjoint(self.h, pg, _ptr(dy)[0], _ptr(da)[0],
                                  _ptr(dP)[0] if dP is not None else None, dev), self.h)
        return dy, da, dP

    @property
    def mterm_width(self) -> int:
        """Doubles per task row of the M-step terms, C (D + 1) + 1."""
        return self.C * (self.D + 1) + 1

    def mstep_terms(self, out=None, device: bool = False):
        """This context's rows of the M-step terms [T][C (D + 1) + 1] (cmcs_mstep_terms)."""
        shape = (self.T, self.mterm_width)
        if out is None:
            if device:
                import torch
                out = torch.empty(shape, dtype=torch.float64, device="cuda")
            else:
                out = np.empty(shape, dtype=np.float64)
        p, dev = _ptr(out)
        _check(lib().cmcs_mstep_terms(self.h, p, dev), self.h)
        return out

    def mstep_apply(self, terms):
        """The M-step from every task's terms [T_total][C (D + 1) + 1] in global task order
        (cmcs_mstep_apply)."""
        if _is_torch(terms):
            if tuple(terms.shape) != (self.T_total, self.mterm_width) or not terms.is_contiguous():
                raise ValueError("terms must be a contiguous [T_total][C (D + 1) + 1] tensor")
        else:
            terms = np.ascontiguousarray(terms, dtype=np.float64)
            if terms.shape != (self.T_total, self.mterm_width):
                raise ValueError("terms must be [T_total][C (D + 1) + 1]")
        p, dev = _ptr(terms)
        _check(lib().cmcs_mstep_apply(self.h, p, dev), self.h)

    def test_stall(self, enable: bool):
        _check(lib().cmcs_test_stall(self.h, 1 if enable else 0), self.h)

    def profile(self, enable: bool = True):
        _check(lib().cmcs_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self) -> dict:
        p = ProfileData()
        _check(lib().cmcs_profile_read(self.h, ctypes.byref(p)), self.h)
        return {f: getattr(p, f) for f, _ in ProfileData._fields_}

    def apply(self, V, accurate: bool = False, B=None):
        """A V (accurate=False) or B - A V with compensated arithmetic (accurate=True);
        V (and B) are [T][C*(K+1)][D] float32, host numpy or device torch."""
        if _is_torch(V):
            import torch
            Z = B.clone() if (accurate and B is not None) else torch.zeros_like(V)
        else:
            V = np.ascontiguousarray(V, dtype=np.float32)
            Z = np.array(B, dtype=np.float32, copy=True) if (accurate and B is not None) else np.zeros_like(V)
        pv, dev = _ptr(V)
        pz, _ = _ptr(Z)
        _check(lib().cmcs_apply(self.h, pv, pz, dev, 1 if accurate else 0), self.h)
        return Z

    def probes(self, em_iter: int, device: bool = False):
        shape = (self.T, self.C, self.K, self.D)
        if device:
            import torch
            out = torch.empty(shape, dtype=torch.float32, device="cuda")
        else:
            out = np.empty(shape, dtype=np.float32)
        p, dev = _ptr(out)
        _check(lib().cmcs_probes(self.h, int(em_iter), p, dev), self.h)
        return out


def _check_noalloc_args(Phi, alpha, V, Z):
    """Shapes, dtypes, contiguity and device of apply_noalloc's tensors, checked before the
    library is called (a wrong one would make its kernels read or write out of bounds)."""
    import torch
    named = [("Phi", Phi), ("alpha", alpha), ("V", V)] + ([("Z", Z)] if Z is not None else [])
    for name, x in named:
        if not isinstance(x, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if x.dtype != torch.float32:
            raise ValueError(f"{name} must be float32, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if Phi.dim() != 2 or V.dim() != 2:
        raise ValueError("Phi must be [N][D] and V [m][D]")
    N, D = Phi.shape
    if N < 1 or D < 1 or V.shape[0] < 1:
        raise ValueError("Phi and V must not be empty")
    if V.shape[1] != D:
        raise ValueError(f"V has {V.shape[1]} columns, Phi has D = {D}")
    if alpha.numel() != D:
        raise ValueError(f"alpha has {alpha.numel()} entries, expected D = {D}")
    if Z is not None and tuple(Z.shape) != tuple(V.shape):
        raise ValueError(f"Z must have V's shape {tuple(V.shape)}, got {tuple(Z.shape)}")
    for name, x in named:
        if not x.is_cuda:
            raise ValueError(f"{name} must be on a CUDA device")
    dev = torch.cuda.current_device()
    for name, x in named:
        if x.device.index != dev:
            raise ValueError(f"{name} is on cuda:{x.device.index}, the current device is cuda:{dev}")


def apply_noalloc(Phi, alpha, beta: float, V, Z=None, stream=None):
    """Z = beta Phi^T (Phi V) + alpha * V for one task without any device allocation inside
    the library (Phi [N][D], alpha [D], V [m][D]: contiguous float32 tensors on the current
    CUDA device; ValueError otherwise)."""
    import torch
    _check_noalloc_args(Phi, alpha, V, Z)
    N, D = Phi.shape
    m = V.shape[0]
    if Z is None:
        Z = torch.empty_like(V)
    _check(lib().cmcs_apply_noalloc(ctypes.c_void_p(Phi.data_ptr()), int(N), int(D),
                                    ctypes.c_void_p(alpha.data_ptr()), float(beta),
                                    ctypes.c_void_p(V.data_ptr()), int(m),
                                    ctypes.c_void_p(Z.data_ptr()), _stream_handle(stream)))
    return Z


def lanczos_quadrature(gamma, xi, steps, stream=None):
    """sum_u S_u1^2 log lambda_u of each U_i x U_i Lanczos matrix (Eqs. 9-10); gamma and xi are
    [nsys][ld] float32 and steps [nsys] int32 CUDA tensors.  Returns (out float64, status int)."""
    import torch
    nsys, ld = gamma.shape
    out = torch.empty(nsys, dtype=torch.float64, device=gamma.device)
    status = torch.zeros(1, dtype=torch.int32, device=gamma.device)
    _check(lib().cmcs_lanczos_quadrature(ctypes.c_void_p(gamma.data_ptr()),
                                         ctypes.c_void_p(xi.data_ptr()),
                                         ctypes.c_void_p(steps.data_ptr()), int(nsys), int(ld),
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(status.data_ptr()),
                                         _stream_handle(stream)))
    return out, int(status.item())
