"""The operator for narrow right-hand-side blocks (R = C(K+1) <= 8 systems per task, two GEMVs
that stream Phi once per pass) against the FP64 definition A V = beta Phi_t^T Phi_t V +
alpha_c V (Eq. 7), and the E-step run on it against the oracle (Alg. 2).

Shapes: D = 700 (D_pad = 768, so the second 512-coordinate block of pass 2 is half empty) and
N_t uneven in [90, 300] (W staged in chunks of 256 rows).  Bounds as for the FP32 GEMM tiles:
FP32 sums over at most 768 and 384 terms, 5e-6 normwise is a few tens of ulps."""
import numpy as np
import pytest

from oracle import cofem
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import make_ctx, rel_err_rows, task_lists
from test_gpu_parity import _estep_pair, replay_q

pytestmark = pytest.mark.gpu


def _wl(C, K, seed=4):
    return synth.make_workload("gemv", 3, C, 700, (90, 300), nnz=6, sigma=0.01, K=K, cg_tol=1e-7,
                               cg_max_iter=80, seed=seed)


@pytest.mark.parametrize("C,K", [(1, 1), (2, 1), (2, 3), (1, 7)])
def test_gemv_operator_matches_oracle(C, K):
    wl = _wl(C, K)
    P, _ = task_lists(wl)
    R = C * (K + 1)
    rng = np.random.default_rng(13)
    V = rng.standard_normal((wl.T, R, wl.D)).astype(np.float32)
    with make_ctx(wl) as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        Z = ctx.apply(V)
        Z2 = ctx.apply(V)
    assert np.array_equal(Z, Z2)                       # fixed summation order
    for t in range(wl.T):
        for j in range(R):
            ref = cofem.apply_A(P[t], wl.beta, alpha[j // (K + 1)], V[t, j].astype(np.float64))
            assert rel_err_rows(Z[t, j], ref) < 5e-6, (t, j)


def test_gemv_estep_matches_oracle():
    """E-step with R = 4 (C = 2, K = 1) on the GEMV operator: means and variances against the
    oracle's refined FP64 solves, log-det and responsibilities in coefficient replay."""
    wl = _wl(2, 1, seed=6)
    alpha = synth.uniform_alpha(wl.C, wl.D, seed=7)
    g, o = _estep_pair(wl, alpha, em_iter=1)
    assert rel_err_rows(g["mu"], o["mu"]).max() <= 1e-4
    assert rel_err_rows(g["s"], o["s"]).max() <= 1e-4
    q_rep, ell_rep, nu_rep = replay_q(wl, g, o, alpha)
    assert np.max(np.abs(g["logdet"] - nu_rep) / np.abs(nu_rep)) <= 1e-9
    assert np.max(np.abs(g["q"] - q_rep)) <= 1e-4
