#!/usr/bin/env python3
"""CoFEM benchmark: EM iterations per second of covariance-free EM on one GB300.

A step is one EM iteration of Alg. 2 (E-step over every task and cluster: batched CG on the
posterior-mean system and K probe systems, refinement of the solutions, diagonal and
log-det estimates, responsibilities; then the M-step) on the plain-scale workload
(T=32, C=4, D=8192, N=2048, K=32 probes, CG tol 1e-5, at most 100 steps), synthetic seeded
inputs, solutions refined to the accuracy the parity tests check.  The default path keeps Phi
as a BF16 pair on the tcgen05 tensor cores (FP32-class products, FP32 accumulation); the
plain FP32 SIMT form is timed beside it on the same workload ("fp32_form").

Beside the headline the default run times, in the same JSON line, the precision workload
(T=16, D=16384, K=64: BF16X3 and FP32 forms, error against exact FP64 solves) and the
batching workload (T=256 uneven tasks: one launch per pass against a per-task launch loop),
each on a short stated sample.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload instead.  Multi-GPU (torchrun): the tasks of the one problem are
split over the ranks (Sec. 3.3; every E-step needs only its own tasks, the M-step's sums are
exchanged in one all-gather per EM iteration), and value is that problem's EM iterations/s
(strong scaling); --replicas runs an independent problem per rank instead (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "CoFEM EM iterations/s (plain-scale workload, one replica per GPU)"


def _metric(workload: str, sharded: bool = False) -> str:
    """The metric's name for the workload timed (the default is plain-scale)."""
    m = METRIC if workload == "plain-scale" else METRIC.replace("plain-scale", workload)
    return m.replace("one replica per GPU", "tasks split over the GPUs") if sharded else m
UNIT = "EM iters/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain-scale")
    ap.add_argument("--tasks", type=int, default=0,
                    help="keep only the first TASKS tasks of the workload (profiling slices)")
    ap.add_argument("--precision", default="bf16x3",
                    help="bf16x3 (tensor cores, Phi as a BF16 pair) or fp32 (SIMT FP32)")
    ap.add_argument("--no-fp32-form", action="store_true",
                    help="skip timing the plain FP32 form beside the tensor-core path")
    ap.add_argument("--schedule", default="batched", choices=["batched", "per_task"])
    ap.add_argument("--compare-schedule", action="store_true",
                    help="also time the per-task launch loop on the same workload")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--refine-max", type=int, default=8)
    ap.add_argument("--refine-tol", type=float, default=1e-5)
    ap.add_argument("--refine-steps", type=int, default=50,
                    help="step cap of the refinement sweeps' CG solves (0: the first solve's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="keep the error against FP64 but skip timing the CPU oracle")
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs, run independent replicas instead of splitting "
                         "the tasks of one problem over them")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the precision and batching workload legs of the default run")
    ap.add_argument("--precond", action="store_true",
                    help="Jacobi-preconditioned CG (method variant)")
    ap.add_argument("--learn-pi", action="store_true", help="learn the cluster priors")
    ap.add_argument("--probe-share", action="store_true",
                    help="probes shared across the clusters of a task")
    ap.add_argument("--warm-start", action="store_true",
                    help="mean systems start from the previous E-step's means")
    ap.add_argument("--compare-precond", action="store_true",
                    help="also time the Jacobi-preconditioned form on the same workload")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm), "sm_min_mhz": min(sm) if sm else None,
                "power_w_median": statistics.median(pw) if pw else None,
                "power_w_max": max(pw) if pw else None}


def aggregate(ms_local: float, steps: int, world: int, device: str = "cuda", units=None):
    """Whole-job throughput over ranks: the slowest rank's time and the units all ranks
    processed (default: every rank's steps, i.e. independent replicas; one problem split over
    the ranks passes units = steps).  Returns (value in units/s, max ms over ranks)."""
    ms_max = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    total = world * steps if units is None else units
    return total / (ms_max / 1e3), ms_max


# DRAM bytes (read + write) of one operator application of the tensor-core operator (k_tc<1> +
# k_tc<3>) on plain-scale with BF16X3, from one ncu capture on the 8-task slice scaled by
# 32 / 8 tasks, keyed to the SHA-256 prefix of the kernel source it was taken on: once that
# source changes the figure no longer describes the kernel and traffic is reported as null.
_TRAFFIC = {"kernels_tc.cu+tc_ptx.cuh": "cd8ab4ddca22cb16",
            "plain-scale/bf16x3": 4 * ((571.588096 + 0.462336) + (548.529408 + 25.012480)) * 1e6}


def _source_sha(*names: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2310_00420_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _operator_traffic(wl, precision: str):
    if wl.name == "plain-scale" and wl.T == 32 and precision == "bf16x3":
        if _source_sha("kernels_tc.cu", "tc_ptx.cuh") == _TRAFFIC["kernels_tc.cu+tc_ptx.cuh"]:
            return _TRAFFIC["plain-scale/bf16x3"]
    return None


def _fp32_sgemm_peak():
    """FP32 throughput measured the way the BF16 peak is: cuBLAS SGEMM (TF32 off) at
    8192^3, best of 10 with CUDA events; TFLOP/s."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        c = a @ b
        best = None
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b, c
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def _single_cta_fft(D: int) -> bool:
    """Whether the Fourier operator at length D runs one CTA per pair (fused CG step)."""
    return 128 <= D <= 8192 and (D & (D - 1)) == 0 and os.environ.get("CMCS_DFT_FOURSTEP") != "1"


def _workload(name: str, seed: int, tasks: int = 0):
    from paper_2310_00420_gb300 import synth
    wl = synth.WORKLOADS[name](seed=seed)
    if tasks and tasks < wl.T:
        wl = wl.subset(range(tasks))
    return wl


def _oracle_pair(wl, alpha, em_iter, t, c, refine_tol, refine_max, precond=False,
                 probe_share=False):
    """The FP64 oracle's E-step for one (task, cluster) pair: K + 1 CG solves + refinement."""
    from oracle import cofem
    if hasattr(wl, "phi_real"):          # Fourier workload: FFT-form operator of the oracle
        P, Y = [cofem.FourierSensing(wl.mask[t])], [wl.y_real(t)]
    else:
        P = [wl.phi(t).astype(np.float64)]
        Y = [wl.yt(t).astype(np.float64)]
    t0 = time.perf_counter()
    o = cofem.cofem_estep(P, Y, np.asarray(alpha[c:c + 1], np.float64), np.array([1.0]), wl.beta,
                          wl.K, wl.seed, em_iter, wl.cg_tol, wl.cg_max_iter, tasks=[t],
                          clusters=[c], C_total=wl.C, refine_tol=refine_tol, refine_max=refine_max,
                          precond=precond, probe_share=probe_share)
    return o, time.perf_counter() - t0


def _cpu_cores():
    n = os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


# (task, cluster) pairs the CPU oracle times, spread over tasks and clusters
N_CPU_PAIRS = 8


def _cpu_pairs(wl):
    return [((7 * i) % wl.T, i % wl.C) for i in range(min(N_CPU_PAIRS, wl.T * wl.C))]


def _cpu_sample(wl, pairs, times, refine_tol, refine_max):
    """The cpu_baseline object for oracle E-step times of the given pairs (seconds each)."""
    per_iter = statistics.mean(times) * wl.T * wl.C            # extrapolated EM iteration
    return {"value": 1.0 / per_iter, "unit": UNIT, "cores": _cpu_cores(), "kind": "oracle",
            "extrapolated": True, "pairs_timed": len(times), "seconds_timed": float(sum(times)),
            "pair_seconds": {"mean": statistics.mean(times), "min": min(times),
                             "max": max(times)},
            "alpha_state": "initial draw of Alg. 2 (EM iteration 0)",
            "sample": f"{len(times)} (task, cluster) pairs of the E-step spread over tasks and "
                      f"clusters {pairs}, each {wl.K + 1} FP64 CG solves + refinement "
                      f"(refine_tol {refine_tol}, at most {refine_max} sweeps) at the initial "
                      f"alpha; EM iteration extrapolated x{wl.T * wl.C} pairs from the mean"}


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import philox
    wl = _workload(a.workload, 0, a.tasks)
    alpha = philox.alpha_init(wl.seed, wl.C, wl.D)
    pairs = _cpu_pairs(wl)
    for i in range(a.warmup):
        t, c = pairs[i % len(pairs)]
        _oracle_pair(wl, alpha, 0, t, c, a.refine_tol, a.refine_max)
    times, used = [], []
    for i in range(a.steps):
        t, c = pairs[i % len(pairs)]
        _, dt = _oracle_pair(wl, alpha, 0, t, c, a.refine_tol, a.refine_max)
        times.append(dt)
        used.append((t, c))
    cpu = _cpu_sample(wl, sorted(set(used)), times, a.refine_tol, a.refine_max)
    value = cpu["value"]
    line = {"impl": "reference", "metric": _metric(a.workload), "value": value, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 / value, "extrapolated": True,
            "ms_per_sample": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{wl.name} T={wl.T} C={wl.C} D={wl.D} N={int(wl.N[0])} "
                                   f"K={wl.K} tol={wl.cg_tol} max_iter={wl.cg_max_iter}",
                       "refine_tol": a.refine_tol, "refine_max": a.refine_max,
                       "step": "one (task, cluster) pair of the E-step per timed step; "
                               "ms_per_step is the EM iteration extrapolated from their mean"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time_ctx(ctx, warmup: int, steps: int) -> dict:
    """EM iterations/s of a context (CUDA events around `steps` iterations after `warmup`),
    with its operator profile and CG statistics."""
    import torch
    for _ in range(warmup):
        ctx.em_iter(1)
    ctx.profile(True)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(steps):
        ctx.em_iter(1)
    f1.record()
    torch.cuda.synchronize()
    ms = f0.elapsed_time(f1)
    pr = ctx.profile_read()
    sm = ctx.summary()
    ctx.profile(False)
    calls = max(1, pr["operator_calls"])
    return {"value": steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "warmup": warmup, "steps": steps,
            "cg_steps_mean": sm["cg_steps_mean"], "cg_capped": sm["cg_capped"],
            "operator_applies": sm["operator_applies"],
            "operator_ms_per_application": pr["operator_ms"] / calls,
            "operator_gbs": pr["operator_bytes"] / (pr["operator_ms"] * 1e-3) / 1e9
            if pr["operator_ms"] else None,
            "operator_tflops": pr["operator_flops"] / (pr["operator_ms"] * 1e-3) / 1e12
            if pr["operator_ms"] else None,
            "residual_ms_per_step": pr["residual_ms"] / steps,
            "resid_rel_max": sm["resid_rel_max"], "refine_diverged": sm["refine_diverged"],
            "operator_applies_bf16_plane": pr["operator_calls_bf16"],
            "bf16_plane_ms_per_application": (pr["operator_ms_bf16"] / pr["operator_calls_bf16"]
                                              if pr["operator_calls_bf16"] else None)}


def precision_leg(a, peaks) -> dict:
    """The precision workload (T=16, C=4, D=16384, N=4096, K=64; R = 260 in two tensor-core
    column tiles): EM iterations/s of the BF16X3 tensor-core path and of the plain FP32 form,
    the operator's HBM fraction, and the error of mu and s on a sampled pair against the
    oracle's exact FP64 solves (Cholesky, Eq. 3), with the M-step's alpha against the oracle's
    M-step on the same E-step outputs."""
    import torch
    from oracle import cofem, philox
    from paper_2310_00420_gb300 import cmcs
    wl = _workload("precision", 0)
    kw = dict(C=wl.C, K=wl.K, beta=wl.beta, pi=wl.pi, cg_max_iter=wl.cg_max_iter,
              cg_tol=wl.cg_tol, seed=wl.seed, refine_max=a.refine_max, refine_tol=a.refine_tol,
              refine_steps=0)
    Phi_d = torch.from_numpy(wl.Phi).cuda()
    y_d = torch.from_numpy(wl.y).cuda()
    out = {"workload": f"{wl.name} T={wl.T} C={wl.C} D={wl.D} N={int(wl.N[0])} K={wl.K} "
                       f"tol={wl.cg_tol} max_iter={wl.cg_max_iter}"}
    ctx = cmcs.Context(Phi_d, y_d, wl.N, precision="bf16x3", **kw)
    tc = _time_ctx(ctx, 1, 2)
    tc["hbm_frac"] = tc["operator_gbs"] / peaks["hbm_gbs"] if tc["operator_gbs"] else None
    # sampled pair against exact FP64 solves with the same probes
    alpha = ctx.read(cmcs.OUT_ALPHA)
    it = ctx.summary()["em_iters_done"]
    ctx.set_alpha(alpha, it)
    ctx.em_iter(1)
    mu_g, s_g, q_g = ctx.read(cmcs.OUT_MU), ctx.read(cmcs.OUT_S), ctx.read(cmcs.OUT_Q)
    alpha_next = ctx.read(cmcs.OUT_ALPHA)
    ctx.close()
    t, c = 3, 2
    P = wl.phi(t).astype(np.float64)
    yv = wl.yt(t).astype(np.float64)
    pk = philox.probes(wl.seed, it, t, c, wl.C, wl.K, wl.D)
    B = np.concatenate([cofem.rhs_mean(P, yv, wl.beta)[:, None], pk.T], axis=1)
    t0 = time.perf_counter()
    X = cofem.solve_exact(P, wl.beta, alpha[c].astype(np.float64), B)
    dt = time.perf_counter() - t0
    rel = lambda g_, r_: float(np.linalg.norm(g_ - r_) / np.linalg.norm(r_))
    a_ref = cofem.m_step(q_g, mu_g.astype(np.float64), s_g.astype(np.float64),
                         alpha.astype(np.float64))
    tc["err_vs_fp64"] = {"pair": [t, c], "mu_rel": rel(mu_g[t, c], X[:, 0]),
                         "s_rel": rel(s_g[t, c], np.mean(pk.T * X[:, 1:], axis=1)),
                         "alpha_mstep_rel": max(rel(alpha_next[j], a_ref[j]) for j in range(wl.C)),
                         "oracle": f"exact Cholesky solves of the pair ({dt:.1f} s); alpha: the "
                                   f"oracle's M-step (Eq. 5, FP64) on the GPU's q, mu, s"}
    tc["ms_per_step_per_task"] = tc["ms_per_step"] / wl.T
    out["bf16x3"] = tc
    del ctx
    # the FP32 SIMT form is ~30x slower here: one EM iteration on tasks 0-3 from the same
    # alpha state, compared per task
    sub = wl.subset(range(4))
    c2 = cmcs.Context(torch.from_numpy(sub.Phi).cuda(), torch.from_numpy(sub.y).cuda(), sub.N,
                      precision="fp32", **kw)
    c2.set_alpha(alpha, it)
    f32 = _time_ctx(c2, 0, 1)
    c2.close()
    f32["tasks"] = "0-3 of 16, one EM iteration from the alpha state of the BF16X3 sample"
    f32["ms_per_step_per_task"] = f32["ms_per_step"] / sub.T
    out["fp32_form"] = f32
    out["bf16x3_speedup_per_task"] = f32["ms_per_step_per_task"] / tc["ms_per_step_per_task"]
    del Phi_d, y_d
    torch.cuda.empty_cache()
    return out


def batching_leg(a) -> dict:
    """The batching workload (T=256 tasks with uneven N_t in [256, 2048], D=4096, C=8, K=16):
    every task in one persistent launch per operator pass (CG chunks replayed from CUDA graphs)
    against a launch loop over the tasks, same precision, same EM iterations."""
    import torch
    from paper_2310_00420_gb300 import cmcs
    wl = _workload("batching", 0)
    kw = dict(C=wl.C, K=wl.K, beta=wl.beta, pi=wl.pi, cg_max_iter=wl.cg_max_iter,
              cg_tol=wl.cg_tol, seed=wl.seed, refine_max=a.refine_max, refine_tol=a.refine_tol,
              refine_steps=0, precision="bf16x3")
    Phi_d = torch.from_numpy(wl.Phi).cuda()
    y_d = torch.from_numpy(wl.y).cuda()
    out = {"workload": f"{wl.name} T={wl.T} C={wl.C} D={wl.D} N_t in [{int(wl.N.min())}, "
                       f"{int(wl.N.max())}] K={wl.K} tol={wl.cg_tol} max_iter={wl.cg_max_iter}"}
    for sched in ("batched", "per_task"):
        c2 = cmcs.Context(Phi_d, y_d, wl.N, schedule=sched, **kw)
        out[sched] = _time_ctx(c2, 1, 1)
        c2.close()
    out["speedup"] = out["batched"]["value"] / out["per_task"]["value"]
    del Phi_d, y_d
    torch.cuda.empty_cache()
    return out


def differentiation_leg(a, n_steps: int = 100) -> dict:
    """The differentiation workload (T=64, C=4, D=2048, N=512, K=32): Phi learned by Adam on
    sum_t ||mu_{t, a_t} - z_t||^2 through PosteriorMeans (forward: one E-step on the current Phi;
    backward: the batched adjoint solve), n_steps timed steps after two warm-up steps, at the
    responsibilities and alpha of the first E-step."""
    import torch
    from paper_2310_00420_gb300 import cmcs
    from paper_2310_00420_gb300.adjoint import posterior_means
    wl = _workload("differentiation", 0)
    kw = dict(C=wl.C, K=wl.K, beta=wl.beta, pi=wl.pi, cg_max_iter=wl.cg_max_iter,
              cg_tol=wl.cg_tol, seed=wl.seed, refine_max=a.refine_max, refine_tol=a.refine_tol,
              refine_steps=0, precision="bf16x3")
    Phi = torch.from_numpy(wl.Phi).cuda().requires_grad_(True)
    y = torch.from_numpy(wl.y).cuda()
    z = torch.from_numpy(wl.z).cuda()
    ctx = cmcs.Context(Phi.detach(), y, wl.N, **kw)
    ctx.estep()
    al = torch.from_numpy(ctx.read(cmcs.OUT_ALPHA)).cuda()
    assign = torch.from_numpy(ctx.read(cmcs.OUT_ASSIGN).astype(np.int64)).cuda()
    rows = torch.arange(wl.T, device="cuda")
    opt = torch.optim.Adam([Phi], lr=1e-4)

    def step():
        mu = posterior_means(ctx, Phi, y, al, 0)
        loss = ((mu[rows, assign] - z) ** 2).sum()
        opt.zero_grad()
        loss.backward()
        opt.step()
        return loss.detach()

    for _ in range(2):
        step()
    losses = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(n_steps):
        losses.append(step())
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    lv = [float(v) for v in losses]
    out = {"workload": f"{wl.name} T={wl.T} C={wl.C} D={wl.D} N={int(wl.N[0])} K={wl.K}",
           "adam_steps": n_steps, "lr": 1e-4, "value": n_steps / (ms / 1000.0),
           "unit": "Adam steps/s", "ms_per_step": ms / n_steps,
           "loss_first": lv[0], "loss_last": lv[-1], "loss_min": min(lv),
           "per_step": "set_data(Phi), E-step (all systems, refined), adjoint solve, Adam update"}
    del Phi, y, z
    torch.cuda.empty_cache()
    return out


def run_ours(a):
    import torch
    from paper_2310_00420_gb300 import cmcs

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    # several GPUs: the tasks of one problem split over them (Sec. 3.3), one all-gather of the
    # M-step rows per EM iteration; or, with --replicas, an independent problem per GPU
    sharded = world > 1 and not a.replicas
    wl = _workload(a.workload, 0 if sharded else rank, a.tasks)
    wl_full = wl
    ranges = None
    if sharded:
        from paper_2310_00420_gb300 import shard
        ranges = shard.partition(wl.N, world)
        wl = wl_full.subset(range(*ranges[rank]))
    fourier = hasattr(wl, "mask")        # Phi_t = Omega_t F, applied by FFT (FP32 only)
    if fourier:
        a.precision = "fp32"
        a.no_fp32_form = True
    kw = dict(C=wl.C, K=wl.K, beta=wl.beta, pi=wl.pi, cg_max_iter=wl.cg_max_iter, cg_tol=wl.cg_tol,
              seed=wl.seed, precision=a.precision, refine_max=a.refine_max, refine_tol=a.refine_tol,
              refine_steps=min(a.refine_steps, wl.cg_max_iter),
              schedule=a.schedule, graphs=not a.no_graphs, precond=a.precond,
              learn_pi=a.learn_pi, probe_share=a.probe_share, warm_start=a.warm_start)
    if sharded:
        kw.update(task_offset=ranges[rank][0], T_total=wl_full.T)
    variant = dict(precond=a.precond, probe_share=a.probe_share)
    if fourier:
        ctx = cmcs.Context.from_fourier(wl, device=True, **kw)
    else:
        Phi_d = torch.from_numpy(wl.Phi).cuda()
        y_d = torch.from_numpy(wl.y).cuda()
        ctx = cmcs.Context(Phi_d, y_d, wl.N, **kw)

    def driver(c_):
        """One EM iteration of the problem: the context's own, or the split one."""
        if not sharded:
            return lambda: c_.em_iter(1)
        em = shard.ShardedEM(c_, ranges, rank, device=True)
        return lambda: em.em_iter(1)

    step = driver(ctx)
    for _ in range(a.warmup):
        step()
    ctx.profile(True)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    summ = ctx.summary()
    ctx.profile(False)
    value, ms_max = aggregate(ms, a.steps, world, units=a.steps if sharded else None)
    systems = wl_full.T * wl.C * (wl.K + 1) if sharded else wl.T * wl.C * (wl.K + 1)

    # operator roofline: algorithmic FLOPs / measured device time of the operator applications
    peaks, src = _peaks()
    op_tflops = prof["operator_flops"] / (prof["operator_ms"] * 1e-3) / 1e12 if prof["operator_ms"] else 0.0
    op_gbs = prof["operator_bytes"] / (prof["operator_ms"] * 1e-3) / 1e9 if prof["operator_ms"] else 0.0
    if fourier:
        # FFT operator fused with the CG update: one CTA per pair of systems, spectra in shared
        # memory; its algorithmic bytes (d, x, r read and written) at the measured HBM bandwidth
        roof = {"bound": "hbm", "achieved": op_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": op_gbs / peaks["hbm_gbs"], "traffic": None,
                "kernel": ("CG step (k_dft_cg_step: FP32 FFT operator of system pairs in shared "
                           "memory fused with the CG update)" if _single_cta_fft(wl.D) else
                           "operator (k_fs_cols_fwd + k_fs_rows + k_fs_cols_inv: four-step FP32 "
                           "FFT of system pairs; d read and A d written counted)"),
                "peak_source": f"MEASURED_PEAKS.json ({src}): HBM {peaks['hbm_gbs']} GB/s",
                "per_launch_flops": prof["operator_flops"] / max(1, prof["operator_calls"]),
                "per_launch_bytes": prof["operator_bytes"] / max(1, prof["operator_calls"]),
                "per_launch_ms": prof["operator_ms"] / max(1, prof["operator_calls"]),
                "fp32_tflops_achieved": op_tflops}
    elif a.precision == "fp32":
        fp32_peak = _fp32_sgemm_peak()
        roof = {"bound": "alu", "achieved": op_tflops, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": op_tflops / fp32_peak,
                "traffic": None,
                "kernel": "operator (k_pass1 + k_pass2, FP32 SIMT)",
                "peak_source": "measured here: cuBLAS SGEMM 8192^3, TF32 off, best of 10",
                "per_launch_flops": prof["operator_flops"] / max(1, prof["operator_calls"]),
                "per_launch_ms": prof["operator_ms"] / max(1, prof["operator_calls"]),
                "hbm_gbs_achieved": op_gbs, "hbm_frac": op_gbs / peaks["hbm_gbs"]}
    else:
        # tensor-core operator: bound by whichever of its algorithmic FLOPs at the measured BF16
        # peak and its algorithmic bytes at the measured HBM bandwidth takes longer
        pk_t = peaks["bf16_tflops_sustained"]
        pk_b = peaks["hbm_gbs"]
        t_flop = prof["operator_flops"] / (pk_t * 1e12)
        t_byte = prof["operator_bytes"] / (pk_b * 1e9)
        per = max(1, prof["operator_calls"])
        common = {"kernel": "operator (k_tc<1> + k_tc<3>, tcgen05 BF16 split; pass 2 reads Phi MN-major)",
                  "per_launch_flops": prof["operator_flops"] / per,
                  "per_launch_bytes": prof["operator_bytes"] / per,
                  "per_launch_ms": prof["operator_ms"] / per,
                  "traffic": _operator_traffic(wl, a.precision),
                  "peak_source": f"MEASURED_PEAKS.json ({src}): HBM {pk_b} GB/s, "
                                 f"BF16 sustained {pk_t} TFLOP/s",
                  "tflops_achieved": op_tflops, "tensor_frac": op_tflops / pk_t}
        if t_byte >= t_flop:
            roof = {"bound": "hbm", "achieved": op_gbs, "peak": pk_b, "unit": "GB/s",
                    "frac": op_gbs / pk_b, **common}
        else:
            roof = {"bound": "tensor", "achieved": op_tflops, "peak": pk_t, "unit": "TFLOP/s",
                    "frac": op_tflops / pk_t, **common}
        roof["hbm_gbs_achieved"] = op_gbs

    # the refinement residual on the tensor cores (k_oz<1> + k_oz<2> and their digit kernels):
    # live time per call and its executed digit-plane MMA work against the sustained BF16
    # peak.  Per 32-system tile, pass 1 multiplies three Phi planes by 4 + 4 + 3 vector planes
    # (352 MMA columns) over D_pad, pass 2 five planes by 3 + 3 + 3 + 2 + 1 (384) over the rows
    res_tc = None
    if (not fourier and a.precision in ("bf16x3", "bf16_mixed") and prof["residual_calls"] > 0
            and os.environ.get("CMCS_OZ", "1") != "0"):
        njt = -(-wl.C * (wl.K + 1) // 32)
        rows = sum(-(-int(n) // 128) * 128 for n in wl.N)
        dpad = -(-wl.D // 128) * 128
        mma = 2.0 * rows * dpad * (352 + 384) * njt
        ms_call = prof["residual_ms"] / prof["residual_calls"]
        pk_t = peaks["bf16_tflops_sustained"]
        res_tc = {"kernels": "k_oz<1> + k_oz<2> (tcgen05, BF16 digit planes) with k_oz_x_digits, "
                             "k_oz_w_digits",
                  "calls_per_step": prof["residual_calls"] / a.steps, "ms_per_call": ms_call,
                  "executed_mma_tflop": mma / 1e12,
                  "tflops_achieved": mma / (ms_call * 1e-3) / 1e12,
                  "tensor_frac": mma / (ms_call * 1e-3) / 1e12 / pk_t,
                  "peak_source": "MEASURED_PEAKS.json: BF16 sustained"}

    # the Lanczos eigen step (Eqs. 9-10) alone, on this E-step's own probe coefficients, through
    # the stand-alone entry point (it runs on a side stream inside the E-step)
    quad_ms = None
    if not fourier:
        gam = ctx.read(cmcs.OUT_GAMMA, device=True).reshape(-1, wl.cg_max_iter)
        xis = ctx.read(cmcs.OUT_XI, device=True).reshape(-1, wl.cg_max_iter)
        stp = ctx.read(cmcs.OUT_STEPS, device=True)[:, :, 1:].contiguous().reshape(-1)
        cmcs.lanczos_quadrature(gam, xis, stp)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record()
        for _ in range(3):
            cmcs.lanczos_quadrature(gam, xis, stp)
        q1.record()
        torch.cuda.synchronize()
        quad_ms = q0.elapsed_time(q1) / 3

    # error vs the FP64 oracle on one sampled (task, cluster) pair, and the CPU baseline
    cpu = None
    err = None
    if rank == 0 and not a.no_cpu and not sharded:
        alpha = ctx.read(cmcs.OUT_ALPHA)
        it = summ["em_iters_done"]
        ctx.set_alpha(alpha, it)
        ctx.estep()
        mu_g = ctx.read(cmcs.OUT_MU)
        s_g = ctx.read(cmcs.OUT_S)
        t_s, c_s = 5, 2 % wl.C
        o, dt = _oracle_pair(wl, alpha, it, t_s, c_s, 1e-12, 40, **variant)
        rel = lambda g_, r_: float(np.linalg.norm(g_ - r_) / np.linalg.norm(r_))
        err = {"pair": [t_s, c_s], "mu_rel": rel(mu_g[t_s, c_s], o["mu"][0, 0]),
               "s_rel": rel(s_g[t_s, c_s], o["s"][0, 0])}
        if world == 1 and not a.no_cpu_baseline:
            from oracle import philox
            alpha0 = philox.alpha_init(wl.seed, wl.C, wl.D)
            pairs = _cpu_pairs(wl)
            times = [_oracle_pair(wl, alpha0, 0, t, c, a.refine_tol, a.refine_max, **variant)[1]
                     for t, c in pairs]
            cpu = _cpu_sample(wl, pairs, times, a.refine_tol, a.refine_max)

    # end to end through the public API with host buffers.  Dense Phi: one context is created
    # before the timed region (set-up); every step then loads that step's Phi and y from pinned
    # host memory (cmcs_set_data: H2D, b0 and the BF16 copies of Phi recomputed), sets alpha,
    # runs one EM iteration and reads q, alpha and the reconstructions (D2H).  Fourier contexts
    # have no set_data, so there each step creates the context from host buffers.
    e2e = None
    if not a.no_e2e:
        if fourier:
            Phi_h = torch.from_numpy(np.ascontiguousarray(wl.mask.astype(np.uint8))).pin_memory()
            y_h = torch.from_numpy(np.ascontiguousarray(
                np.stack([wl.y.real, wl.y.imag], axis=-1).astype(np.float32))).pin_memory()
        else:
            Phi_h = torch.from_numpy(wl.Phi).pin_memory()
            y_h = torch.from_numpy(wl.y).pin_memory()
        alpha_h = torch.from_numpy(ctx.read(cmcs.OUT_ALPHA)).pin_memory()
        it = ctx.summary()["em_iters_done"]
        outs = {"q": torch.empty((wl.T, wl.C), dtype=torch.float64).pin_memory(),
                "alpha": torch.empty((wl.C, wl.D), dtype=torch.float32).pin_memory(),
                "recon": torch.empty((wl.T, wl.D), dtype=torch.float32).pin_memory()}
        c2 = None if fourier else cmcs.Context(Phi_h, y_h, wl.N, **kw)
        c2_step = None if fourier else driver(c2)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            if fourier:
                c3 = cmcs.Context(None, y_h, wl.N, mask=Phi_h, **kw)
                c3.set_alpha(alpha_h, it)
                driver(c3)()
            else:
                c3 = c2
                c3.set_data(Phi_h, y_h)
                c3.set_alpha(alpha_h, it)
                c2_step()
            c3.read(cmcs.OUT_Q, out=outs["q"])
            c3.read(cmcs.OUT_ALPHA, out=outs["alpha"])
            c3.read(cmcs.OUT_RECON, out=outs["recon"])
            if fourier:
                c3.close()
        torch.cuda.synchronize()
        barrier()
        e2e_value, _ = aggregate((time.perf_counter() - t0) * 1e3, a.steps, world,
                                 units=a.steps if sharded else None)
        if c2 is not None:
            c2.close()
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(Phi_h.numel() * Phi_h.element_size() +
                                         y_h.numel() * y_h.element_size() + wl.C * wl.D * 4),
               "d2h_bytes_per_step": int(sum(v.numel() * v.element_size() for v in outs.values())),
               "per_step": ("cmcs_set_data from pinned host Phi and y, cmcs_set_alpha, one EM "
                            "iteration, reads of q, alpha and the reconstructions"
                            if not fourier else
                            "cmcs_create_dft from pinned host mask and y, cmcs_set_alpha, one EM "
                            "iteration, reads of q, alpha and the reconstructions")}

    ctx.close()

    def timed_leg(warmup=None, steps=None, **over):
        """EM iterations/s of another form on the same workload (same warm-up and steps unless
        given)."""
        w_ = a.warmup if warmup is None else warmup
        n_ = a.steps if steps is None else steps
        kw2 = dict(kw)
        kw2.update(over)
        c3 = (cmcs.Context.from_fourier(wl, device=True, **kw2) if fourier
              else cmcs.Context(Phi_d, y_d, wl.N, **kw2))
        out = _time_ctx(c3, w_, n_)
        c3.close()
        out.update({k: v for k, v in over.items()})
        return out

    fp32_form = None
    if a.precision != "fp32" and not a.no_fp32_form and world == 1:
        # the FP32 SIMT form is ~7x slower: a shorter sample (stated in the line)
        fp32_form = timed_leg(warmup=min(a.warmup, 1), steps=min(a.steps, 3), precision="fp32")
        peak32 = _fp32_sgemm_peak()
        fp32_form["fp32_peak_tflops"] = peak32
        fp32_form["fp32_peak_source"] = "measured here: cuBLAS SGEMM 8192^3, TF32 off, best of 10"
        if fp32_form["operator_tflops"]:
            fp32_form["alu_frac"] = fp32_form["operator_tflops"] / peak32
    mixed_form = None
    if a.precision == "bf16x3" and not a.no_fp32_form and world == 1 and not fourier:
        # the mixed path: first solves with Phi as one BF16 plane (half its bytes), refinement
        # with the BF16 pair; its one-plane operator against the measured HBM bandwidth
        # (its refinement keeps the first solve's step cap: with shorter inner solves some
        # systems' refinement diverges from the one-plane first solve)
        mixed_form = timed_leg(warmup=min(a.warmup, 2), steps=min(a.steps, 5),
                               precision="bf16_mixed", refine_steps=0)
        one = sum(2.0 * int(n) * wl.D + 4.0 * wl.C * (wl.K + 1) * (2.0 * wl.D + 2.0 * int(n))
                  for n in wl.N)
        if mixed_form["bf16_plane_ms_per_application"]:
            gbs = one / (mixed_form["bf16_plane_ms_per_application"] * 1e-3) / 1e9
            mixed_form["bf16_plane_bytes_per_application"] = one
            mixed_form["bf16_plane_hbm_gbs"] = gbs
            mixed_form["bf16_plane_hbm_frac"] = gbs / peaks["hbm_gbs"]
        if rank == 0 and not a.no_cpu:
            c4 = cmcs.Context(Phi_d, y_d, wl.N, **dict(kw, precision="bf16_mixed", refine_steps=0))
            c4.em_iter(2)
            al4 = c4.read(cmcs.OUT_ALPHA)
            it4 = c4.summary()["em_iters_done"]
            c4.estep()
            mu4, s4 = c4.read(cmcs.OUT_MU), c4.read(cmcs.OUT_S)
            c4.close()
            o4, _ = _oracle_pair(wl, al4, it4, 5, 2 % wl.C, 1e-12, 40, **variant)
            rel4 = lambda g_, r_: float(np.linalg.norm(g_ - r_) / np.linalg.norm(r_))
            mixed_form["err_vs_fp64"] = {"pair": [5, 2 % wl.C],
                                         "mu_rel": rel4(mu4[5, 2 % wl.C], o4["mu"][0, 0]),
                                         "s_rel": rel4(s4[5, 2 % wl.C], o4["s"][0, 0])}
    per_task = None
    if a.compare_schedule:
        per_task = timed_leg(schedule="per_task")
    precond_form = None
    if a.compare_precond and not a.precond:
        precond_form = timed_leg(precond=True)
    legs = {}
    if rank == 0 and world == 1 and not a.no_legs and a.workload == "plain-scale" and not a.tasks:
        del Phi_d, y_d
        torch.cuda.empty_cache()
        legs["precision_workload"] = precision_leg(a, peaks)
        legs["batching_workload"] = batching_leg(a)
        legs["differentiation_workload"] = differentiation_leg(a)
    if rank == 0:
        line = {"metric": _metric(a.workload, sharded), "value": value, "unit": UNIT,
                "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / a.steps,
                "higher_is_better": True, "scaling": "strong" if sharded else "weak",
                "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16": "bf16+f32", "bf16x3": "bf16x2+f32",
                          "bf16_mixed": "bf16+bf16x2+f32"}[a.precision],
                "data": "synthetic",
                "config": {"workload": f"{wl_full.name} T={wl_full.T} C={wl.C} D={wl.D} "
                                       f"N={int(wl.N[0])} K={wl.K} tol={wl.cg_tol} "
                                       f"max_iter={wl.cg_max_iter}",
                           "precision": a.precision, "refine_max": a.refine_max,
                           "refine_tol": a.refine_tol, "refine_steps": min(a.refine_steps, wl.cg_max_iter) or wl.cg_max_iter,
                           "parallelism": (f"tasks split over {world} GPUs {ranges}, one "
                                           f"all-gather of the M-step rows per EM iteration"
                                           if sharded else f"{world} replicas"),
                           "variants": [v for v, on in (("precond", a.precond),
                                                        ("learn_pi", a.learn_pi),
                                                        ("probe_share", a.probe_share),
                                                        ("warm_start", a.warm_start)) if on],
                           "l2": (f"inputs larger than L2 (CG vectors {5 * systems * wl.D * 4 / 1e9:.1f} GB)"
                                  if fourier else
                                  f"inputs larger than L2 (Phi {wl.Phi.nbytes / 1e9:.1f} GB)")},
                "cg_solves_per_s": value * systems,
                "cg_solves_counted": "refined solves: every system of the E-step, counted once "
                                     "whether its first CG solve converged or stopped at "
                                     "max_iter and was finished by refinement",
                "cg_steps_mean": summ["cg_steps_mean"], "cg_capped": summ["cg_capped"],
                "cg_capped_frac": summ["cg_capped"] / systems,
                "refine_sweeps_max": summ["refine_sweeps_max"],
                "refine_diverged": summ["refine_diverged"], "resid_rel_max": summ["resid_rel_max"],
                "operator_share": prof["operator_ms"] / ms if ms else None,
                "residual_ms_per_step": prof["residual_ms"] / a.steps,
                "residual_tc": res_tc,
                "operator_applies_per_step": prof["operator_calls"] / a.steps,
                "lanczos_quadrature_ms": quad_ms,
                "roofline": roof, "cpu_baseline": cpu, "err_vs_fp64": err, "e2e": e2e,
                "clocks": clk, "gpu_launches": prof["kernel_launches"],
                "fp32_form": fp32_form, "bf16_mixed_form": mixed_form,
                "per_task_schedule": per_task,
                "precond_form": precond_form, **legs}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
