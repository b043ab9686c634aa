"""The refinement residual on the tensor cores (digit planes of Phi, error-free splitting) against
the FP64 definition r = B - A X (Eq. 7).

The residual exists so that refinement converges to the solution of the exact system (Sec. 3.1:
the E-step needs the solutions of Eq. 7).  Its pass 2, Phi^T W, is formed without rounding; W's
digits keep 24 bits below each system's largest |W|, an error that enters r as beta Phi^T dW.
So the error e = r_gpu - r must lie in the range of beta Phi_t^T up to ~2^-40 of the summed
terms, with a dW of the size of FP32 rounding of pass 1's terms; a rounded Phi^T W would leave
errors of ~1e-7 of the terms outside that range.  Digit sums at the exactness limit (odd sums
above 2^23 in one tensor-memory accumulator) are checked on a constant Phi whose operands have
exact digit expansions."""
import numpy as np
import pytest

from oracle import cofem
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import make_ctx, task_lists

pytestmark = pytest.mark.gpu


def _workloads():
    # plain-small (one chunk per tile, R = 42 in two system tiles) and a ragged shape with
    # several chunks along D in pass 1 and uneven N_t < D
    yield "plain-small", synth.plain_small()
    yield "ragged", synth.make_workload("oz-ragged", 3, 3, 2500, (100, 700), nnz=12, sigma=0.01,
                                        K=12, cg_tol=1e-6, cg_max_iter=60, seed=5)


def _reference(P, alpha_c, beta, x, b):
    return b - cofem.apply_A(P, beta, alpha_c, x)


@pytest.mark.parametrize("name", ["plain-small", "ragged"])
@pytest.mark.parametrize("chunk", ["8", "16"])
def test_tc_residual_error_is_a_perturbation_of_w(name, chunk, monkeypatch):
    monkeypatch.setenv("CMCS_OZ_CHUNK", chunk)
    wl = dict(_workloads())[name]
    P, Y = task_lists(wl)
    R = wl.C * (wl.K + 1)
    rng = np.random.default_rng(31)
    B = rng.standard_normal((wl.T, R, wl.D)).astype(np.float32)
    with make_ctx(wl, precision="bf16x3") as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        # X = fl32(A^-1 B): the true residual is ~1e-7 of ||B||, all of it cancellation
        X = np.empty_like(B)
        for t in range(wl.T):
            for c in range(wl.C):
                A = wl.beta * P[t].T @ P[t] + np.diag(alpha[c])
                js = slice(c * (wl.K + 1), (c + 1) * (wl.K + 1))
                X[t, js] = np.linalg.solve(A, B[t, js].astype(np.float64).T).T.astype(np.float32)
        Rg = ctx.apply(X, accurate=True, B=B)
        Rg2 = ctx.apply(X, accurate=True, B=B)
        R0 = ctx.apply(np.zeros_like(X), accurate=True, B=B)
    assert np.array_equal(Rg, Rg2)                     # deterministic
    assert np.array_equal(R0, B)                       # X = 0: r = B exactly
    worst_out, worst_dw = 0.0, 0.0
    for t in range(wl.T):
        Pt = P[t]
        assert Pt.shape[0] < wl.D                      # the decomposition below needs N_t < D
        for j in range(R):
            c = j // (wl.K + 1)
            x = X[t, j].astype(np.float64)
            ref = _reference(Pt, alpha[c], wl.beta, x, B[t, j].astype(np.float64))
            scale = np.linalg.norm(np.abs(B[t, j]) + cofem.apply_A(np.abs(Pt), wl.beta, alpha[c],
                                                                   np.abs(x)))
            e = Rg[t, j].astype(np.float64) - ref
            # e = -beta Phi^T dW + (pass-2 and output rounding)
            dw, *_ = np.linalg.lstsq(wl.beta * Pt.T, -e, rcond=None)
            out = np.linalg.norm(e + wl.beta * Pt.T @ dw)
            assert out <= 2e-7 * np.linalg.norm(ref) + 1e-11 * scale, (t, j, out, scale)
            # dW: the digits of x' (24 bits below max |x'|) and of W, an error of the size of
            # FP32 rounding of pass 1's terms |Phi| |x| (x itself is much larger than W here:
            # A^-1 B lies mostly in the null space of Phi_t)
            rel_dw = np.linalg.norm(dw) / np.linalg.norm(np.abs(Pt) @ np.abs(x))
            assert rel_dw <= 2.0 ** -20, (t, j, rel_dw)
            worst_out = max(worst_out, out / scale)
            worst_dw = max(worst_dw, rel_dw)
    print(f"{name} chunk {chunk}: out-of-range error {worst_out:.2e} of the terms, "
          f"dW {worst_dw:.2e} of |Phi| |x|")


@pytest.mark.parametrize("chunk", ["8", "16"])
def test_tc_residual_digit_sums_at_the_exactness_limit(chunk, monkeypatch):
    """Phi_t = 127/128 except its first row (zero), X = 2^-11: then W = 127/128 on every other
    row, and every column of Phi^T W sums 1023 products of digits 127 x 127 over the 1024 rows of
    a task, 16,499,967 in one tensor-memory accumulator (with chunks of 1024): above 2^23 and
    odd, so the accumulation must keep all 24 bits.  A lost bit there is an error of 2^-14 in z,
    beta 2^-14 in r, far above the bound below."""
    monkeypatch.setenv("CMCS_OZ_CHUNK", chunk)
    wl = synth.make_workload("oz-exact", 2, 1, 2048, 1024, nnz=4, sigma=0.01, K=3, cg_tol=1e-6,
                             cg_max_iter=20, seed=2)
    wl.Phi[:] = np.float32(127.0 / 128.0)
    for t in range(wl.T):
        wl.Phi[wl.row_off[t]] = 0.0
    R = wl.C * (wl.K + 1)
    X = np.full((wl.T, R, wl.D), 2.0 ** -11, dtype=np.float32)
    rng = np.random.default_rng(3)
    B = rng.standard_normal((wl.T, R, wl.D)).astype(np.float32)
    with make_ctx(wl, precision="bf16x3") as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        Rg = ctx.apply(X, accurate=True, B=B)
    P, _ = task_lists(wl)
    for t in range(wl.T):
        for j in range(R):
            x = X[t, j].astype(np.float64)
            ref = _reference(P[t], alpha[0], wl.beta, x, B[t, j].astype(np.float64))
            scale = np.linalg.norm(np.abs(B[t, j]) + cofem.apply_A(np.abs(P[t]), wl.beta, alpha[0], x))
            err = np.linalg.norm(Rg[t, j] - ref)
            assert err <= 2e-7 * np.linalg.norm(ref) + 1e-11 * scale, (t, j, err, scale)


def test_tc_residual_refinement_matches_double_single(monkeypatch):
    """The E-step refined with the tensor-core residual and with the double-single SIMT one
    (CMCS_OZ=0) reach the same means and variances (both against exact solves: 1e-4)."""
    wl = synth.plain_small()
    out = {}
    for oz in ("1", "0"):
        monkeypatch.setenv("CMCS_OZ", oz)
        with make_ctx(wl, precision="bf16x3", refine_tol=1e-6, refine_max=8) as ctx:
            ctx.estep()
            out[oz] = (ctx.read(cmcs.OUT_MU).astype(np.float64), ctx.read(cmcs.OUT_S).astype(np.float64))
    for a, b in zip(out["1"], out["0"]):
        rel = np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)
        assert rel.max() <= 1e-5, rel.max()
