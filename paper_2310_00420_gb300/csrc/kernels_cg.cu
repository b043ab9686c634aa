// Batched conjugate gradient (Alg. 1) over all S = T*C*(K+1) systems, the diagonal estimator
// (Eq. 4) and the set-up kernels (b0 = beta Phi^T y, alpha ~ Uniform(0,1), probes).
//
// One CTA of 256 threads owns one system for the vector updates, so both inner products of a
// CG step (d^T A d and r^T r, or r^T M^-1 r with the Jacobi preconditioner) reduce inside the
// CTA: no grid-wide barrier or spin-wait exists.  With the SIMT and four-step Fourier
// operators d^T A d arrives as per-tile partials from the operator epilogue; with the
// tensor-core operator the update kernel adds alpha_c * d to beta Phi^T Phi d and forms
// d^T A d itself.  Every reduction has a fixed tree order, so results are run-to-run
// deterministic.
// Converged systems are masked (their CTA returns at once) and a task whose systems have all
// converged is skipped by the operator.  Also here: the Jacobi preconditioner's column norms
// and per-E-step diagonal, and the warm start's addition of the previous means.
#include <cuda_bf16.h>
#include <math.h>

#include <vector>

#include "cmcs_internal.cuh"

namespace cmcs {

namespace {

// fixed-order block sum over 256 threads (warp xor-tree, then warp 0 over the 8 warp sums)
template <typename Tv>
__device__ __forceinline__ Tv block_sum(Tv v, Tv* sh) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  Tv tot = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += sh[i];
    sh[32] = tot;
  }
  __syncthreads();
  return sh[32];
}

__device__ __forceinline__ float4 probe4(uint64_t seed, int64_t em, int t, int c, int C, int k0,
                                         int d, int D) {
  const uint32_t bits = probe_bits32(seed, em, t, c, C, k0, d & ~31);
  const int sh = d & 31;
  float v[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) v[e] = (d + e < D) ? (((bits >> (sh + e)) & 1u) ? -1.f : 1.f) : 0.f;
  return make_float4(v[0], v[1], v[2], v[3]);
}

// BF16 pair split x = hi + lo of four values, written for the tensor-core operator
__device__ __forceinline__ void store_split4(__nv_bfloat16* hi, __nv_bfloat16* lo, int64_t i,
                                             float4 v) {
  const float x[4] = {v.x, v.y, v.z, v.w};
  __nv_bfloat16 h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    h[e] = __float2bfloat16_rn(x[e]);
    l[e] = __float2bfloat16_rn(x[e] - __bfloat162float(h[e]));
  }
  *reinterpret_cast<uint2*>(hi + i) = *reinterpret_cast<const uint2*>(h);
  *reinterpret_cast<uint2*>(lo + i) = *reinterpret_cast<const uint2*>(l);
}

}  // namespace

// ---- CG initialisation: x_1 = 0, r_1 = d_1 = b (Alg. 1, first line) ---------------------
// mode 0: b = b0_t (k = 0) or the probe p_{t,c,k} (k >= 1); mode 1: b = the residual
// already in r (refinement), systems no longer refining have r = 0; mode 2: b = a given
// right-hand side already in r (first solve of the adjoint system).
// With the Jacobi preconditioner (pminv != null): probe right-hand sides are sqrt(m) * p,
// d_1 = z_1 = M^-1 r_1 and rr = r^T z.
// warm (mode 0): the mean systems (k = 0) start from the previous means, so r already holds
// b0 - A mu_prev; their tol test keeps the cold start's reference b0^T M^-1 b0, and a system
// already within tol of it takes no step.
__global__ void __launch_bounds__(256)
k_cg_init(int mode, float* __restrict__ x, float* __restrict__ r, float* __restrict__ d,
          const float* __restrict__ b0hi, float* rr, float* bb, int* steps, int* active,
          int* ractive, int* sweeps, float* rrel, int* task_active, int* counters, int R,
          int K, int C, int Dp, int D, uint64_t seed, int64_t em_iter, int toff, int refine,
          __nv_bfloat16* dhi, __nv_bfloat16* dlo, const float* __restrict__ pminv,
          const float* __restrict__ pw, int pshare, int warm, float tol2) {
  __shared__ float sh[33];
  const int64_t sys = blockIdx.x;
  const int t = (int)(sys / R), j = (int)(sys % R), c = j / (K + 1), k = j % (K + 1);
  const bool wm = mode == 0 && warm != 0 && k == 0;      // block-uniform
  float* xs = x + sys * Dp;
  float* rs = r + sys * Dp;
  float* ds = d + sys * Dp;
  const int64_t tcoff = ((int64_t)t * C + c) * Dp;
  float acc = 0.f, accr = 0.f;
  for (int i = threadIdx.x * 4; i < Dp; i += 256 * 4) {
    float4 b;
    if (mode == 0) {
      if (wm) {
        b = *reinterpret_cast<const float4*>(rs + i);           // b0 - A mu_prev
        float4 b0 = *reinterpret_cast<const float4*>(b0hi + (int64_t)t * Dp + i);
        float4 z0 = b0;
        if (pminv != nullptr) {
          const float4 mi = *reinterpret_cast<const float4*>(pminv + tcoff + i);
          z0 = make_float4(b0.x * mi.x, b0.y * mi.y, b0.z * mi.z, b0.w * mi.w);
        }
        accr = fmaf(b0.x, z0.x, accr);
        accr = fmaf(b0.y, z0.y, accr);
        accr = fmaf(b0.z, z0.z, accr);
        accr = fmaf(b0.w, z0.w, accr);
      } else if (k == 0) {
        b = *reinterpret_cast<const float4*>(b0hi + (int64_t)t * Dp + i);
      } else {
        b = probe4(seed, em_iter, t + toff, probe_cluster(c, pshare), C, k - 1, i, D);
        if (pw != nullptr) {
          const float4 w = *reinterpret_cast<const float4*>(pw + tcoff + i);
          b = make_float4(b.x * w.x, b.y * w.y, b.z * w.z, b.w * w.w);
        }
      }
      *reinterpret_cast<float4*>(rs + i) = b;
    } else {
      b = *reinterpret_cast<const float4*>(rs + i);
    }
    float4 z = b;
    if (pminv != nullptr) {
      const float4 mi = *reinterpret_cast<const float4*>(pminv + tcoff + i);
      z = make_float4(b.x * mi.x, b.y * mi.y, b.z * mi.z, b.w * mi.w);
    }
    *reinterpret_cast<float4*>(xs + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(ds + i) = z;
    if (dhi != nullptr) store_split4(dhi, dlo, sys * Dp + i, z);
    acc = fmaf(b.x, z.x, acc);
    acc = fmaf(b.y, z.y, acc);
    acc = fmaf(b.z, z.z, acc);
    acc = fmaf(b.w, z.w, acc);
  }
  const float rr0 = block_sum(acc, sh);
  const float ref = wm ? block_sum(accr, sh) : rr0;
  if (threadIdx.x == 0) {
    rr[sys] = rr0;
    bb[sys] = ref;
    steps[sys] = 0;
    if (mode != 1) {
      ractive[sys] = refine;
      sweeps[sys] = 0;
      rrel[sys] = 0.f;
    }
    const int on = (rr0 > 0.f) && (mode != 1 || ractive[sys] != 0) && !(wm && rr0 <= tol2 * ref);
    active[sys] = on;
    if (on) {
      atomicAdd(&task_active[t], 1);
      atomicAdd(&counters[0], 1);
    }
  }
}

// ---- one CG step after the operator has produced ad = A d (Alg. 1, loop body) ----------
// NV > 0: each thread keeps its NV float4s of r_{u+1} and d_u in registers between the two
// phases (D_pad <= 1024 NV); NV = 0: generic loop that re-reads them.
// RAW = false: ad = A d and d^T A d arrives as per-tile partials from the operator epilogue.
// RAW = true (tensor-core operator): ad = beta Phi^T Phi d only; this kernel adds alpha_c * d
// and forms d^T A d itself, so the operator's epilogue reads neither d nor alpha.
// pminv != null: Jacobi-preconditioned step, z = M^-1 r, rr = r^T z, d = z + xi d.
template <int NV, bool RAW>
__global__ void __launch_bounds__(256)
k_cg_update(float* __restrict__ x, float* __restrict__ r, float* __restrict__ d,
            const float* __restrict__ ad, const float* __restrict__ part,
            const float* __restrict__ alpha, int ndt, float* rr, const float* bb, int* steps,
            int* active, int* task_active, int* counters, float* gam, float* xih, int* psteps,
            int record, int R, int K, int C, int Dp, int S, int U, int cap, float tol2,
            __nv_bfloat16* dhi, __nv_bfloat16* dlo, const float* __restrict__ pminv) {
  __shared__ float sh[33];
  __shared__ float s_dad;
  const int64_t sys = blockIdx.x;
  if (active[sys] == 0) return;
  const int t = (int)(sys / R), j = (int)(sys % R);
  float* xs = x + sys * Dp;
  float* rs = r + sys * Dp;
  float* ds = d + sys * Dp;
  const float* as = ad + sys * Dp;
  const float* al = alpha + (int64_t)(j / (K + 1)) * Dp;
  const float* mi = pminv != nullptr ? pminv + ((int64_t)t * C + j / (K + 1)) * Dp : nullptr;
  // z = M^-1 r for four coordinates (r itself without the preconditioner)
  auto zof = [&](int i, float4 rv) {
    if (mi == nullptr) return rv;
    const float4 m4 = *reinterpret_cast<const float4*>(mi + i);
    return make_float4(rv.x * m4.x, rv.y * m4.y, rv.z * m4.z, rv.w * m4.w);
  };
  float4 dk[NV > 0 ? NV : 1], ak[(RAW && NV > 0) ? NV : 1];
  // A d for four coordinates (RAW: beta Phi^T Phi d + alpha_c * d)
  auto adv = [&](int i, float4 dv) {
    float4 av = *reinterpret_cast<const float4*>(as + i);
    if constexpr (RAW) {
      const float4 a4 = *reinterpret_cast<const float4*>(al + i);
      av.x = fmaf(a4.x, dv.x, av.x); av.y = fmaf(a4.y, dv.y, av.y);
      av.z = fmaf(a4.z, dv.z, av.z); av.w = fmaf(a4.w, dv.w, av.w);
    }
    return av;
  };
  float dad;
  if constexpr (RAW) {
    float a2 = 0.f;
    auto pre = [&](int i, float4& dout, float4& aout) {
      dout = *reinterpret_cast<const float4*>(ds + i);
      aout = adv(i, dout);
      a2 = fmaf(dout.x, aout.x, a2); a2 = fmaf(dout.y, aout.y, a2);
      a2 = fmaf(dout.z, aout.z, a2); a2 = fmaf(dout.w, aout.w, a2);
    };
    if constexpr (NV > 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int i = (threadIdx.x + 256 * q) * 4;
        if (i < Dp) pre(i, dk[q], ak[q]);
      }
    } else {
      float4 d0, a0;
      for (int i = threadIdx.x * 4; i < Dp; i += 256 * 4) pre(i, d0, a0);
    }
    dad = block_sum(a2, sh);                       // d_u^T A d_u
  } else {
    if (threadIdx.x < 32) {
      float v = 0.f;
      for (int q = threadIdx.x; q < ndt; q += 32) v += part[(int64_t)q * S + sys];
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
      if (threadIdx.x == 0) s_dad = v;
    }
    __syncthreads();
    dad = s_dad;
  }
  const float rr0 = rr[sys];
  if (!(dad > 0.f) || !isfinite(dad)) {            // breakdown: stop this system
    if (threadIdx.x == 0) {
      active[sys] = 0;
      atomicSub(&task_active[t], 1);
      atomicSub(&counters[0], 1);
      if (!isfinite(dad)) atomicOr(&counters[2], 1);
    }
    return;
  }
  const float g = rr0 / dad;                       // gamma_u
  float acc = 0.f;
  float4 rk[NV > 0 ? NV : 1];
  auto step1 = [&](int i, int q, float4& ro, float4& dout) {
    float4 xv = *reinterpret_cast<float4*>(xs + i);
    float4 rv = *reinterpret_cast<float4*>(rs + i);
    float4 dv, av;
    if constexpr (RAW && NV > 0) {
      dv = dk[q];
      av = ak[q];
    } else {
      dv = *reinterpret_cast<const float4*>(ds + i);
      av = adv(i, dv);
    }
    xv.x = fmaf(g, dv.x, xv.x); xv.y = fmaf(g, dv.y, xv.y);
    xv.z = fmaf(g, dv.z, xv.z); xv.w = fmaf(g, dv.w, xv.w);
    rv.x = fmaf(-g, av.x, rv.x); rv.y = fmaf(-g, av.y, rv.y);
    rv.z = fmaf(-g, av.z, rv.z); rv.w = fmaf(-g, av.w, rv.w);
    *reinterpret_cast<float4*>(xs + i) = xv;
    *reinterpret_cast<float4*>(rs + i) = rv;
    const float4 zv = zof(i, rv);
    acc = fmaf(rv.x, zv.x, acc);
    acc = fmaf(rv.y, zv.y, acc);
    acc = fmaf(rv.z, zv.z, acc);
    acc = fmaf(rv.w, zv.w, acc);
    ro = zv;
    dout = dv;
  };
  if constexpr (NV > 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int i = (threadIdx.x + 256 * q) * 4;
      if (i < Dp) step1(i, q, rk[q], dk[q]);
    }
  } else {
    for (int i = threadIdx.x * 4; i < Dp; i += 256 * 4) step1(i, 0, rk[0], dk[0]);
  }
  const float rr1 = block_sum(acc, sh);            // r_{u+1}^T z_{u+1} (z = r: r^T r)
  const float xi = rr1 / rr0;                      // xi_u
  auto step2 = [&](int i, float4 rv, float4 dv) {  // rv: z_{u+1}
    dv.x = fmaf(xi, dv.x, rv.x); dv.y = fmaf(xi, dv.y, rv.y);
    dv.z = fmaf(xi, dv.z, rv.z); dv.w = fmaf(xi, dv.w, rv.w);
    *reinterpret_cast<float4*>(ds + i) = dv;
    if (dhi != nullptr) store_split4(dhi, dlo, sys * Dp + i, dv);
  };
  if constexpr (NV > 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int i = (threadIdx.x + 256 * q) * 4;
      if (i < Dp) step2(i, rk[q], dk[q]);
    }
  } else {
    for (int i = threadIdx.x * 4; i < Dp; i += 256 * 4)
      step2(i, zof(i, *reinterpret_cast<const float4*>(rs + i)),
            *reinterpret_cast<const float4*>(ds + i));
  }
  if (threadIdx.x == 0) {
    const int u = steps[sys];
    const int c = j / (K + 1), k = j % (K + 1);
    if (record && k > 0) {
      const int64_t pidx = ((int64_t)t * C + c) * K + (k - 1);
      gam[pidx * U + u] = g;
      xih[pidx * U + u] = xi;
      psteps[pidx] = u + 1;
    }
    steps[sys] = u + 1;
    rr[sys] = rr1;
    if (!isfinite(rr1)) atomicOr(&counters[2], 1);
    const bool done = (rr1 <= tol2 * bb[sys]) || (rr1 == 0.f) || (u + 1 >= cap) || !isfinite(rr1);
    if (done) {
      active[sys] = 0;
      atomicSub(&task_active[t], 1);
      atomicSub(&counters[0], 1);
    }
  }
}

// ---- refinement: xacc += delta; stop once the estimated relative error <= refine_tol ----
__global__ void __launch_bounds__(256)
k_refine_update(float* __restrict__ xacc, const float* __restrict__ delta, int* ractive,
                int* sweeps, float* rrel, int* counters, int Dp, float rtol) {
  __shared__ float sh[33];
  const int64_t sys = blockIdx.x;
  if (ractive[sys] == 0) return;
  float* xa = xacc + sys * Dp;
  const float* de = delta + sys * Dp;
  float a1 = 0.f, a2 = 0.f;
  for (int i = threadIdx.x * 4; i < Dp; i += 256 * 4) {
    float4 xv = *reinterpret_cast<float4*>(xa + i);
    const float4 dv = *reinterpret_cast<const float4*>(de + i);
    xv.x += dv.x; xv.y += dv.y; xv.z += dv.z; xv.w += dv.w;
    *reinterpret_cast<float4*>(xa + i) = xv;
    a1 += dv.x * dv.x + dv.y * dv.y + dv.z * dv.z + dv.w * dv.w;
    a2 += xv.x * xv.x + xv.y * xv.y + xv.z * xv.z + xv.w * xv.w;
  }
  const float dn2 = block_sum(a1, sh);
  const float xn2 = block_sum(a2, sh);
  __shared__ int s_revert;
  if (threadIdx.x == 0) {
    const int sw = sweeps[sys] + 1;
    sweeps[sys] = sw;
    const float rel = xn2 > 0.f ? sqrtf(dn2 / xn2) : 0.f;
    const float prev = rrel[sys];
    // a correction larger than the previous one means the inner solves no longer contract:
    // undo it, stop refining this system and count it
    const int diverged = (sw > 1 && rel > prev) || !isfinite(rel);
    s_revert = diverged;
    if (diverged) {
      ractive[sys] = 0;
      atomicAdd(&counters[3], 1);
    } else {
      rrel[sys] = rel;
      // stop once the remaining relative error is estimated below rtol: the first correction
      // itself, then the next correction predicted from the contraction rho = rel / prev of
      // the last two (the error left is about rho rel / (1 - rho) of ||x||)
      bool stop = rel <= rtol || !(xn2 > 0.f);
      if (!stop && sw > 1 && prev > 0.f) {
        const float rho = rel / prev;
        stop = rho * rel <= rtol * (1.f - rho);
      }
      if (stop) {
        ractive[sys] = 0;
      } else {
        atomicAdd(&counters[1], 1);
      }
    }
  }
  __syncthreads();
  if (s_revert) {
    for (int i = threadIdx.x * 4; i < Dp; i += 256 * 4) {
      float4 xv = *reinterpret_cast<float4*>(xa + i);
      const float4 dv = *reinterpret_cast<const float4*>(de + i);
      xv.x -= dv.x; xv.y -= dv.y; xv.z -= dv.z; xv.w -= dv.w;
      *reinterpret_cast<float4*>(xa + i) = xv;
    }
  }
}

// ---- ||b - A x|| / ||b|| per system from the residual in r ----------------------------
__global__ void __launch_bounds__(256)
k_resid_norm(const float* __restrict__ r, const float* __restrict__ b0hi,
             const float* __restrict__ b0lo, float* rres, int R, int K, int Dp, int D) {
  __shared__ double sh[33];
  const int64_t sys = blockIdx.x;
  const int t = (int)(sys / R), j = (int)(sys % R), k = j % (K + 1);
  if (k != 0) return;                  // the final residual is formed for the mean systems
  const float* rs = r + sys * Dp;
  double a1 = 0.0, a2 = 0.0;
  for (int d = threadIdx.x; d < D; d += 256) {
    const double rv = (double)rs[d];
    a1 += rv * rv;
    if (k == 0) {
      const double bv = (double)b0hi[(int64_t)t * Dp + d] + (double)b0lo[(int64_t)t * Dp + d];
      a2 += bv * bv;
    }
  }
  const double rr = block_sum(a1, sh);
  const double bb = block_sum(a2, sh);
  if (threadIdx.x == 0) rres[sys] = bb > 0.0 ? (float)sqrt(rr / bb) : 0.f;
}

cudaError_t launch_resid_norm(Ctx* c) {
  c->launches += 1;
  k_resid_norm<<<c->S, 256, 0, c->stream>>>(c->r, c->b0hi, c->b0lo, c->rres, c->R, c->K, c->Dp,
                                            c->D);
  return cudaGetLastError();
}

// ---- diagonal estimator s_tc = (1/K) sum_k p_k * x_k (Eq. 4) ----------------------------
__global__ void __launch_bounds__(128)
// With the Jacobi preconditioner the probe systems solve A x_k = sqrt(m) p_k, and
// s = (1/K) sum_k p_k x_k / sqrt(m) (pw = sqrt(m); null: plain probes).
k_sest(const float* __restrict__ xacc, float* __restrict__ sest, int R, int K, int C, int Dp,
       int D, uint64_t seed, int64_t em_iter, int toff, const float* __restrict__ pw,
       int pshare) {
  const int tc = blockIdx.y;
  const int t = tc / C, c = tc % C;
  const int i = (blockIdx.x * 128 + threadIdx.x) * 4;
  if (i >= Dp) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t base = ((int64_t)t * R + (int64_t)c * (K + 1)) * Dp;
  for (int k = 1; k <= K; ++k) {
    const float4 p = probe4(seed, em_iter, t + toff, probe_cluster(c, pshare), C, k - 1, i, D);
    const float4 xv = *reinterpret_cast<const float4*>(xacc + base + (int64_t)k * Dp + i);
    acc.x = fmaf(p.x, xv.x, acc.x);
    acc.y = fmaf(p.y, xv.y, acc.y);
    acc.z = fmaf(p.z, xv.z, acc.z);
    acc.w = fmaf(p.w, xv.w, acc.w);
  }
  const float inv = 1.0f / (float)K;
  float4 sv = make_float4(acc.x * inv, acc.y * inv, acc.z * inv, acc.w * inv);
  if (pw != nullptr) {
    const float4 w = *reinterpret_cast<const float4*>(pw + (int64_t)tc * Dp + i);
    sv = make_float4(sv.x / w.x, sv.y / w.y, sv.z / w.z, sv.w / w.w);
  }
  *reinterpret_cast<float4*>(sest + (int64_t)tc * Dp + i) = sv;
}

// ---- Jacobi preconditioner: m = beta ||Phi_t e_d||^2 + alpha_cd, the diagonal of A_tc ----
__global__ void __launch_bounds__(128)
k_colnorm(const float* __restrict__ phi, const int64_t* drow, float* colnorm, int Dp) {
  const int t = blockIdx.y;
  const int d = blockIdx.x * 128 + threadIdx.x;
  if (d >= Dp) return;
  double acc = 0.0;
  for (int64_t n = drow[t]; n < drow[t + 1]; ++n) {
    const double a = (double)phi[n * Dp + d];
    acc = fma(a, a, acc);
  }
  colnorm[(int64_t)t * Dp + d] = (float)acc;
}

__global__ void __launch_bounds__(256)
k_precond(const float* __restrict__ colnorm, const float* __restrict__ alpha, float* pminv,
          float* pw, double* sumlogm, int C, int Dp, int D, double beta) {
  __shared__ double sh[33];
  const int tc = blockIdx.x, t = tc / C, c = tc % C;
  double acc = 0.0;
  for (int d = threadIdx.x; d < Dp; d += 256) {
    const double m = beta * (double)colnorm[(int64_t)t * Dp + d] + (double)alpha[(int64_t)c * Dp + d];
    pminv[(int64_t)tc * Dp + d] = (float)(1.0 / m);
    pw[(int64_t)tc * Dp + d] = (float)sqrt(m);
    if (d < D) acc += log(m);
  }
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) sumlogm[tc] = tot;
}

// ---- b0_t = beta Phi_t^T y_t, kept as hi + lo (compensated sum, then FP64 scaling) ------
__global__ void __launch_bounds__(128)
k_b0(const float* __restrict__ phi, const float* __restrict__ y, const int64_t* drow,
     float* b0hi, float* b0lo, int Dp, double beta) {
  const int t = blockIdx.y;
  const int d = blockIdx.x * 128 + threadIdx.x;
  if (d >= Dp) return;
  float hi = 0.f, lo = 0.f;
  for (int64_t n = drow[t]; n < drow[t + 1]; ++n) {
    const float a = phi[n * Dp + d], b = y[n];
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bv = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  const double v = beta * ((double)hi + (double)lo);
  const float vh = (float)v;
  b0hi[(int64_t)t * Dp + d] = vh;
  b0lo[(int64_t)t * Dp + d] = (float)(v - (double)vh);
}

// ---- alpha_c ~ Uniform(0,1) (Alg. 2, first step); padded coordinates get 1 ---------------
__global__ void k_alpha_init(float* alpha, int Dp, int D, uint64_t seed) {
  const int c = blockIdx.y;
  const int d = blockIdx.x * 256 + threadIdx.x;
  if (d >= Dp) return;
  float v = 1.0f;
  if (d < D) {
    U4 ctr{(uint32_t)(d >> 2), (uint32_t)c, 0u, kTagAlpha};
    const U4 w = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t word = pick_word(w, d & 3);
    v = ((float)(word >> 9) + 0.5f) * 1.1920928955078125e-07f;   // 2^-23
  }
  alpha[(int64_t)c * Dp + d] = v;
}

// ---- sum_d log alpha_cd in FP64 (Eq. 3) ---------------------------------------------------
__global__ void __launch_bounds__(256)
k_sumlogalpha(const float* alpha, double* out, int Dp, int D) {
  __shared__ double sh[33];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int d = threadIdx.x; d < D; d += 256) acc += log((double)alpha[(int64_t)c * Dp + d]);
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) out[c] = tot;
}

// ---- per-task constant of log p(y_t | alpha_c) = ell/2 - const_t -------------------------
__global__ void __launch_bounds__(256)
k_tconst(const float* y, const int64_t* drow, const int64_t* Nt, double* out, double beta) {
  __shared__ double sh[33];
  const int t = blockIdx.x;
  double acc = 0.0;
  for (int64_t n = drow[t] + threadIdx.x; n < drow[t + 1]; n += 256) acc += (double)y[n] * (double)y[n];
  const double yy = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double N = (double)Nt[t];
    out[t] = 0.5 * (N * 1.8378770664093453 - N * log(beta) + beta * yy);   // log(2 pi)
  }
}

// ---- probes as +-1 floats [T][C][K][D] ----------------------------------------------------
__global__ void k_probes_out(float* dst, int T, int C, int K, int D, uint64_t seed,
                             int64_t em_iter, int toff, int pshare) {
  const int64_t tck = blockIdx.y;
  const int k = (int)(tck % K);
  const int c = (int)((tck / K) % C);
  const int t = (int)(tck / ((int64_t)K * C));
  const int d = blockIdx.x * 256 + threadIdx.x;
  if (d >= D) return;
  const uint32_t bits = probe_bits32(seed, em_iter, t + toff, probe_cluster(c, pshare), C, k,
                                     d & ~31);
  dst[tck * D + d] = ((bits >> (d & 31)) & 1u) ? -1.f : 1.f;
}

// --------------------------------------------------------------------------------------
cudaError_t launch_cg_init(Ctx* c, int mode, int warm) {
  c->launches += 1;
  k_cg_init<<<c->S, 256, 0, c->stream>>>(mode, c->x, c->r, c->d, c->b0hi, c->rr, c->bb,
                                         c->steps, c->active, c->ractive, c->sweeps, c->rrel,
                                         c->task_active, c->counters, c->R, c->K, c->C, c->Dp,
                                         c->D, c->seed, c->em_iter, c->toff,
                                         c->refine_max > 0 ? 1 : 0,
                                         static_cast<__nv_bfloat16*>(c->dhi),
                                         static_cast<__nv_bfloat16*>(c->dlo),
                                         c->precond ? c->pminv : nullptr,
                                         c->precond ? c->pw : nullptr, c->pshare, warm,
                                         (float)(c->cg_tol * c->cg_tol));
  return cudaGetLastError();
}

// ---- warm start: x of the mean systems += the previous means -----------------------------
__global__ void __launch_bounds__(256)
k_add_means(float* __restrict__ x, const float* __restrict__ prev, int R, int K, int C, int Dp) {
  const int tc = blockIdx.x, t = tc / C, c = tc % C;
  const int64_t off = ((int64_t)t * R + (int64_t)c * (K + 1)) * Dp;
  for (int i = threadIdx.x; i < Dp; i += 256) x[off + i] += prev[off + i];
}

cudaError_t launch_add_means(Ctx* c) {
  c->launches += 1;
  k_add_means<<<c->T * c->C, 256, 0, c->stream>>>(c->x, c->xacc, c->R, c->K, c->C, c->Dp);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(Ctx* c, int record) {
  c->launches += 1;
  const float tol2 = (float)(c->cg_tol * c->cg_tol);
  const int nv = (c->Dp + 1023) / 1024;
#define UPD(NV)                                                                                  \
  if (c->tc != nullptr)                                                                          \
    k_cg_update<NV, true><<<c->S, 256, 0, c->stream>>>(                                          \
        c->x, c->r, c->d, c->ad, c->part, c->alpha, c->op == 1 ? c->dft_ndt : c->Dp / 128, c->rr, c->bb, c->steps,        \
        c->active, c->task_active, c->counters, c->gam, c->xi, c->psteps, record, c->R, c->K,    \
        c->C, c->Dp, c->S, c->U, cg_cap(c), tol2, static_cast<__nv_bfloat16*>(c->dhi),         \
        static_cast<__nv_bfloat16*>(c->dlo), c->precond ? c->pminv : nullptr);                   \
  else                                                                                           \
    k_cg_update<NV, false><<<c->S, 256, 0, c->stream>>>(                                         \
        c->x, c->r, c->d, c->ad, c->part, c->alpha, c->op == 1 ? c->dft_ndt : c->Dp / 128, c->rr, c->bb, c->steps,        \
        c->active, c->task_active, c->counters, c->gam, c->xi, c->psteps, record, c->R, c->K,    \
        c->C, c->Dp, c->S, c->U, cg_cap(c), tol2, static_cast<__nv_bfloat16*>(c->dhi),         \
        static_cast<__nv_bfloat16*>(c->dlo), c->precond ? c->pminv : nullptr)
  if (nv <= 1) { UPD(1); }
  else if (nv <= 2) { UPD(2); }
  else if (nv <= 4) { UPD(4); }
  else if (nv <= 8) { UPD(8); }
  else if (nv <= 16) { UPD(16); }
  else { UPD(0); }
#undef UPD
  return cudaGetLastError();
}

cudaError_t launch_refine_update(Ctx* c) {
  c->launches += 1;
  k_refine_update<<<c->S, 256, 0, c->stream>>>(c->xacc, c->x, c->ractive, c->sweeps, c->rrel,
                                               c->counters, c->Dp, (float)c->refine_tol);
  return cudaGetLastError();
}

cudaError_t launch_sest(Ctx* c) {
  c->launches += 1;
  dim3 grid((c->Dp / 4 + 127) / 128, c->T * c->C);
  k_sest<<<grid, 128, 0, c->stream>>>(c->xacc, c->sest, c->R, c->K, c->C, c->Dp, c->D, c->seed,
                                      c->em_iter, c->toff, c->precond ? c->pw : nullptr,
                                      c->pshare);
  return cudaGetLastError();
}

cudaError_t launch_colnorm(Ctx* c) {
  if (!c->precond) return cudaSuccess;
  if (c->op == 1) {
    // Phi_t = Omega_t F with F unitary: every column has ||Phi_t e_d||^2 = N_t / D
    std::vector<float> h((size_t)c->T * c->Dp, 0.f);
    for (int t = 0; t < c->T; ++t)
      for (int d = 0; d < c->D; ++d)
        h[(size_t)t * c->Dp + d] = (float)((double)(c->hN[t] / 2) / (double)c->D);
    cudaError_t e = cudaMemcpyAsync(c->colnorm, h.data(), sizeof(float) * h.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);     // h is released on return
  }
  c->launches += 1;
  dim3 grid(c->Dp / 128, c->T);
  k_colnorm<<<grid, 128, 0, c->stream>>>(c->phi, c->drow, c->colnorm, c->Dp);
  return cudaGetLastError();
}

cudaError_t launch_precond(Ctx* c) {
  if (!c->precond) return cudaSuccess;
  c->launches += 1;
  k_precond<<<c->T * c->C, 256, 0, c->stream>>>(c->colnorm, c->alpha, c->pminv, c->pw, c->sumlogm,
                                                c->C, c->Dp, c->D, c->beta);
  return cudaGetLastError();
}

cudaError_t launch_b0(Ctx* c) {
  if (c->op == 1) return launch_dft_b0(c);
  c->launches += 1;
  dim3 grid(c->Dp / 128, c->T);
  k_b0<<<grid, 128, 0, c->stream>>>(c->phi, c->y, c->drow, c->b0hi, c->b0lo, c->Dp, c->beta);
  return cudaGetLastError();
}

cudaError_t launch_alpha_init(Ctx* c) {
  c->launches += 1;
  dim3 grid((c->Dp + 255) / 256, c->C);
  k_alpha_init<<<grid, 256, 0, c->stream>>>(c->alpha, c->Dp, c->D, c->seed);
  return cudaGetLastError();
}

cudaError_t launch_sumlogalpha(Ctx* c) {
  c->launches += 1;
  k_sumlogalpha<<<c->C, 256, 0, c->stream>>>(c->alpha, c->sumlogalpha, c->Dp, c->D);
  return cudaGetLastError();
}

cudaError_t launch_tconst_dev(Ctx* c, const int64_t* dN) {
  c->launches += 1;
  k_tconst<<<c->T, 256, 0, c->stream>>>(c->y, c->drow, dN, c->tconst, c->beta);
  return cudaGetLastError();
}

cudaError_t launch_probes_out(const Ctx* c, int64_t em_iter, float* dst) {
  dim3 grid((c->D + 255) / 256, (unsigned)((int64_t)c->T * c->C * c->K));
  k_probes_out<<<grid, 256, 0, c->stream>>>(dst, c->T, c->C, c->K, c->D, c->seed, em_iter,
                                            c->toff, c->pshare);
  return cudaGetLastError();
}

}  // namespace cmcs
