"""Tensor-core operator (tcgen05) parity: the BF16-split operator against the FP64 oracle, and
the E-step on it (with refinement) against the oracle.

Bounds: BF16X3 keeps ~16 significant bits per product (Phi and the vectors each split into two
BF16 parts, the lo*lo term dropped), so a normwise operator error of 1e-4 is ~6 units of 2^-16;
BF16_REFINE rounds Phi itself to 8 bits (2^-9 relative per entry), bound 1e-2.  After
refinement the E-step meets the path's tolerances: 1e-4 (BF16X3, the FP32 bar) and 1e-3 (BF16
with refinement), responsibilities 1e-4 in coefficient replay."""
import numpy as np
import pytest

from oracle import cofem
from paper_2310_00420_gb300 import cmcs, synth

from gpu_helpers import make_ctx, rel_err_rows, task_lists
from test_gpu_parity import replay_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    return synth.plain_small()


@pytest.mark.parametrize("precision,bound", [("bf16x3", 1e-4), ("bf16", 1e-2)])
def test_tc_operator_matches_oracle(small, precision, bound):
    P, Y = task_lists(small)
    R = small.C * (small.K + 1)
    rng = np.random.default_rng(21)
    V = rng.standard_normal((small.T, R, small.D)).astype(np.float32)
    with make_ctx(small, precision=precision) as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        Z = ctx.apply(V)
        Z2 = ctx.apply(V)
    assert np.array_equal(Z, Z2)                       # deterministic
    errs = []
    for t in range(small.T):
        for j in range(R):
            c = j // (small.K + 1)
            ref = cofem.apply_A(P[t], small.beta, alpha[c], V[t, j].astype(np.float64))
            errs.append(rel_err_rows(Z[t, j], ref))
    assert max(errs) < bound, max(errs)


@pytest.mark.parametrize("shape", [dict(T=3, C=3, D=200, N=(37, 150), K=5),
                                   dict(T=2, C=4, D=384, N=(1, 300), K=70)])
def test_tc_operator_ragged(shape):
    """Uneven N_t, D not a multiple of 128, and R = C(K+1) = 284 > 256 (two TMEM column blocks)."""
    wl = synth.make_workload("ragged", shape["T"], shape["C"], shape["D"], shape["N"], nnz=5,
                             sigma=0.01, K=shape["K"], seed=9)
    P, Y = task_lists(wl)
    R = wl.C * (wl.K + 1)
    V = np.random.default_rng(22).standard_normal((wl.T, R, wl.D)).astype(np.float32)
    with make_ctx(wl, precision="bf16x3") as ctx:
        alpha = ctx.read(cmcs.OUT_ALPHA).astype(np.float64)
        Z = ctx.apply(V)
    for t in range(wl.T):
        for j in range(R):
            c = j // (wl.K + 1)
            ref = cofem.apply_A(P[t], wl.beta, alpha[c], V[t, j].astype(np.float64))
            assert rel_err_rows(Z[t, j], ref) < 1e-4, (t, j)


def test_bf16_phi_refinement_divergence_is_detected(small):
    """Rounding Phi itself to BF16 moves the small eigenvalues of A by about
    beta ||Phi - bf16(Phi)||^2 ~ 1 here, more than the smallest alpha, so refinement from
    BF16-Phi inner solves does not contract.  The library must notice, undo the growing
    corrections and report the systems, not return a blown-up solution silently."""
    alpha = synth.uniform_alpha(small.C, small.D, seed=3)
    with make_ctx(small, precision="bf16", refine_max=16, refine_tol=1e-6) as ctx:
        ctx.set_alpha(alpha, 2)
        ctx.estep()
        summ = ctx.summary()
        mu = ctx.read(cmcs.OUT_MU)
    assert summ["refine_diverged"] > 0
    assert np.all(np.isfinite(mu))


@pytest.mark.parametrize("precision,tol", [("bf16x3", 1e-4), ("bf16_mixed", 1e-4)])
def test_tc_estep_parity(small, precision, tol):
    """E-step on the tensor-core operator against the oracle's refined FP64 solves.  The mixed
    path runs its first solve (the Lanczos coefficients) with Phi as one BF16 plane and refines
    with the BF16 pair, so its solutions meet the same bound; nu is graded in replay."""
    P, Y = task_lists(small)
    alpha = synth.uniform_alpha(small.C, small.D, seed=3)
    with make_ctx(small, precision=precision, refine_max=16, refine_tol=1e-6) as ctx:
        ctx.set_alpha(alpha, 2)
        ctx.estep()
        g = {k: ctx.read(v) for k, v in dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, q=cmcs.OUT_Q,
                                              logdet=cmcs.OUT_LOGDET, ell=cmcs.OUT_ELL,
                                              steps=cmcs.OUT_STEPS, gamma=cmcs.OUT_GAMMA,
                                              xi=cmcs.OUT_XI, assign=cmcs.OUT_ASSIGN).items()}
    o = cofem.cofem_estep(P, Y, alpha.astype(np.float64), small.pi, small.beta, small.K,
                          small.seed, 2, small.cg_tol, small.cg_max_iter, refine_tol=1e-12,
                          refine_max=40)
    assert rel_err_rows(g["mu"], o["mu"]).max() <= tol
    assert rel_err_rows(g["s"], o["s"]).max() <= tol
    q_rep, _, _ = replay_q(small, g, o, alpha)
    assert np.max(np.abs(g["q"] - q_rep)) <= 1e-4
    assert np.array_equal(g["assign"], np.argmax(o["q"], axis=1))


@pytest.mark.parametrize("precision", ["bf16x3", "bf16"])
def test_operator_schedules_agree(precision, monkeypatch):
    """The fused launch (pass 1 and pass 2 of every task in one persistent kernel, pass 2 reading
    Phi MN-major), the two-launch MN-major schedule (pass 2 launched programmatically, its tiles
    waiting on per-task counts of finished pass-1 tiles, or launched after pass 1) and the
    two-launch schedule over a transposed copy of Phi accumulate the same products in the same
    k order."""
    wl = synth.make_workload("ragged", 3, 3, 200, (37, 300), nnz=5, sigma=0.01, K=70, seed=9)
    R = wl.C * (wl.K + 1)
    V = np.random.default_rng(23).standard_normal((wl.T, R, wl.D)).astype(np.float32)
    Z = {}
    for mode, early in (("0", "1"), ("3", "1"), ("3", "0"), ("2", "0")):
        monkeypatch.setenv("CMCS_TC_MODE", mode)
        monkeypatch.setenv("CMCS_TC_EARLY", early)
        with make_ctx(wl, precision=precision) as ctx:
            Z[mode + early] = ctx.apply(V)
            Z[mode + early + "again"] = ctx.apply(V)
    Z["0"], Z["2"] = Z["01"], Z["20"]
    assert np.array_equal(Z["01"], Z["01again"])
    assert np.array_equal(Z["31"], Z["31again"])
    assert np.array_equal(Z["0"], Z["31"])
    assert np.array_equal(Z["31"], Z["30"])          # pass 2 launched early or after pass 1
    np.testing.assert_allclose(Z["2"], Z["0"], rtol=1e-5, atol=1e-5 * np.abs(Z["0"]).max())


def test_mixed_precision_em_parity(small):
    """Ten EM iterations of the mixed path (first solves with Phi as one BF16 plane, BF16-pair
    refinement) against the oracle's EM loop: the reduced-precision bar of 1e-3 for alpha and
    the reconstructions, bit-exact assignments, responsibilities at 1e-4 except the named soft
    task.  The profile counts the one-plane applications (the first solves)."""
    from gpu_helpers import check_free_q
    P, Y = task_lists(small)
    with make_ctx(small, precision="bf16_mixed", refine_max=12, refine_tol=1e-6) as ctx:
        ctx.profile(True)
        ctx.em_iter(small.em_iters)
        prof = ctx.profile_read()
        a_g, q_g = ctx.read(cmcs.OUT_ALPHA), ctx.read(cmcs.OUT_Q)
        asg, recon = ctx.read(cmcs.OUT_ASSIGN), ctx.read(cmcs.OUT_RECON)
        summ = ctx.summary()
    o = cofem.em(P, Y, small.pi, small.beta, small.em_iters, K=small.K, seed=small.seed,
                 tol=small.cg_tol, max_iter=small.cg_max_iter, C=small.C, D=small.D,
                 refine_tol=1e-12, refine_max=40)
    assert summ["refine_diverged"] == 0
    assert np.array_equal(asg, o["assign"])
    check_free_q(q_g, o["last"]["q"], soft_tasks=(2,))      # task 2: q = (0.992, 0.008)
    assert rel_err_rows(a_g, o["alpha"]).max() <= 1e-3
    assert rel_err_rows(recon, o["recon"]).max() <= 1e-3
    assert 0 < prof["operator_calls_bf16"] < prof["operator_calls"]


@pytest.mark.parametrize("splitk", ["4", "2", "3", "default"])
def test_one_read_schedule_matches_oracle(splitk, monkeypatch):
    """The one-read schedule (CMCS_TC_MODE=4: pass-1 row tiles split along K, reduced in split
    order by the last unit, each task's pass-2 tiles following its pass-1 units in one launch)
    against the oracle's operator, uneven N_t, and its E-step against the refined FP64 solves.
    It is an evaluation switch, slower than the default two launches (Phi is not held in L2
    long enough), kept under test."""
    if splitk != "default":                               # "default": the two-launch schedule
        monkeypatch.setenv("CMCS_TC_MODE", "4")
        monkeypatch.setenv("CMCS_TC_SPLITK", splitk)
    # N_t well below D, as in the paper's workloads (the BF16-pair refinement contracts)
    wl = synth.make_workload("ragged", 4, 3, 640, (60, 300), nnz=8, sigma=0.01, K=9, seed=19)
    P, Y = task_lists(wl)
    R = wl.C * (wl.K + 1)
    V = np.random.default_rng(24).standard_normal((wl.T, R, wl.D)).astype(np.float32)
    a32 = synth.uniform_alpha(wl.C, wl.D, seed=8) + np.float32(0.05)
    alpha = a32.astype(np.float64)
    with make_ctx(wl, precision="bf16x3", refine_max=12, refine_tol=1e-6) as ctx:
        ctx.set_alpha(a32, 0)
        Z = ctx.apply(V)
        assert np.array_equal(Z, ctx.apply(V))           # fixed summation order
        ctx.estep()
        mu, s_ = ctx.read(cmcs.OUT_MU), ctx.read(cmcs.OUT_S)
    for t in range(wl.T):
        for j in range(R):
            c = j // (wl.K + 1)
            ref = cofem.apply_A(P[t], wl.beta, alpha[c], V[t, j].astype(np.float64))
            assert rel_err_rows(Z[t, j], ref) < 1e-4, (t, j)
    o = cofem.cofem_estep(P, Y, alpha, wl.pi, wl.beta, wl.K, wl.seed, 0, wl.cg_tol,
                          wl.cg_max_iter, refine_tol=1e-12, refine_max=40)
    assert rel_err_rows(mu, o["mu"]).max() <= 1e-4
    assert rel_err_rows(s_, o["s"]).max() <= 1e-4
