"""Shared helpers of the GPU parity tests (comparison metrics and context construction)."""
import numpy as np


def rel_err_rows(got: np.ndarray, ref: np.ndarray, axis=-1) -> np.ndarray:
    """Norm-wise relative error ||got - ref|| / ||ref|| along ``axis`` (per vector)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.linalg.norm(got - ref, axis=axis)
    den = np.linalg.norm(ref, axis=axis)
    return num / np.where(den > 0, den, 1.0)


def task_lists(wl):
    return ([wl.phi(t).astype(np.float64) for t in range(wl.T)],
            [wl.yt(t).astype(np.float64) for t in range(wl.T)])


def make_ctx(wl, **kw):
    from paper_2310_00420_gb300 import cmcs
    return cmcs.Context.from_workload(wl, device=True, **kw)
