// Structured sensing operator of Sec. 4: Phi_t = Omega_t F, with F the unitary D x D DFT and
// Omega_t the rows (frequencies) a 0/1 mask selects.  Sec. 3.3 notes that CG needs only
// products with A, which for this Phi cost O(D log D) by FFT instead of O(N D).
//
// Reading for complex Phi and real z: the real and imaginary parts of y_t are 2 N_t real
// measurements, each with noise precision beta, so
//     A_tc = beta Re(Phi_t^H Phi_t) + diag(alpha_c),    b0_t = beta Re(Phi_t^H y_t).
// Phi^H Phi = F^H diag(m) F, and for real v, Re(F^H diag(m) F v) = ifft(mt .* fft(v)) with the
// symmetrised mask mt_k = (m_k + m_{D-k}) / 2 (real and even, so the product stays real).  One
// complex FFT of v1 + i v2 therefore applies the operator to two systems of a task at once:
// the real part of the result belongs to v1, the imaginary part to v2.
//
// One CTA per pair of systems holds the pair's spectrum in shared memory: a
// decimation-in-frequency FFT (natural order in, bit-reversed out), the mask multiply (the
// mask is stored in bit-reversed order), and a decimation-in-time inverse (bit-reversed in,
// natural out), so no permutation pass is needed.  Each pass over shared memory applies three
// radix-2 stages in registers (eight elements per thread).  The CG operator runs in FP32; the
// refinement residual b - A x runs the same transform in FP64 (the DFT is unitary, so its
// rounding error stays ~log2(D) units of FP64, below the double-single residual of the dense
// path).  Twiddles come from tables computed on the host in FP64.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "cmcs_internal.cuh"

namespace cmcs {

namespace {

constexpr int kDftThreads = 512;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Shared-memory index with one pad element per 32: the passes with small spacing would
// otherwise hit the same banks with power-of-two strides.
__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

template <typename CT> __device__ __forceinline__ CT cmake(double x, double y);
template <> __device__ __forceinline__ float2 cmake<float2>(double x, double y) {
  return make_float2((float)x, (float)y);
}
template <> __device__ __forceinline__ double2 cmake<double2>(double x, double y) {
  return make_double2(x, y);
}

// e^{-2 pi i k / n} for n in {2, 4, 8}, k < n / 2
template <typename CT>
__device__ __forceinline__ CT root_of_unity(int n, int k) {
  const double h = 0.70710678118654752440;       // sqrt(2) / 2
  if (k == 0) return cmake<CT>(1.0, 0.0);
  if (n == 4 || (n == 8 && k == 2)) return cmake<CT>(0.0, -1.0);
  if (k == 1) return cmake<CT>(h, -h);
  return cmake<CT>(-h, -h);
}

// Radix-2 butterflies, R stages per pass over shared memory: each thread loads 2^R elements
// spaced sub apart, applies the R stages in registers and stores them back.  Within a pass
// every twiddle is w^(2^q) times an 8th, 4th or 2nd root of unity, with w = W_span^j for the
// group's offset j: one table load per group and pass.
// Decimation in frequency, stages of half-size 2^s down to 2^(s-R+1):
template <typename CT, int R>
__device__ __forceinline__ void dif_pass(CT* X, const CT* __restrict__ tw, int D, int s) {
  const int lsub = s - R + 1, sub = 1 << lsub, span = 1 << (s + 1);
  for (int g = threadIdx.x; g < (D >> R); g += blockDim.x) {
    const int j = g & (sub - 1);
    const int base = (g >> lsub) * span + j;
    CT wq = tw[j * (D / span)];
    CT x[1 << R];
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) x[m] = X[pad(base + m * sub)];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int step = 1 << (R - 1 - q);
#pragma unroll
      for (int m = 0; m < (1 << R); ++m) {
        if (m & step) continue;
        const int k = m & (step - 1);
        const CT t = k == 0 ? wq : cmul(wq, root_of_unity<CT>(1 << (R - q), k));
        const CT u = x[m], v = x[m + step];
        x[m] = cadd(u, v);
        x[m + step] = cmul(csub(u, v), t);
      }
      wq = cmul(wq, wq);
    }
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) X[pad(base + m * sub)] = x[m];
  }
  __syncthreads();
}

// decimation in time with conjugate twiddles, stages of half-size 2^s up to 2^(s+R-1)
template <typename CT, int R>
__device__ __forceinline__ void dit_pass(CT* X, const CT* __restrict__ tw, int D, int s) {
  const int sub = 1 << s, span = 1 << (s + R);
  for (int g = threadIdx.x; g < (D >> R); g += blockDim.x) {
    const int j = g & (sub - 1);
    const int base = (g >> s) * span + j;
    CT pw[R];                                     // w, w^2, w^4 with w = W_span^j
    pw[0] = tw[j * (D / span)];
#pragma unroll
    for (int q = 1; q < R; ++q) pw[q] = cmul(pw[q - 1], pw[q - 1]);
    CT x[1 << R];
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) x[m] = X[pad(base + m * sub)];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int step = 1 << q;
#pragma unroll
      for (int m = 0; m < (1 << R); ++m) {
        if (m & step) continue;
        const int k = m & (step - 1);
        const CT t = k == 0 ? pw[R - 1 - q] : cmul(pw[R - 1 - q], root_of_unity<CT>(1 << (q + 1), k));
        const CT u = x[m];
        const CT v = cmulc(x[m + step], t);
        x[m] = cadd(u, v);
        x[m + step] = csub(u, v);
      }
    }
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) X[pad(base + m * sub)] = x[m];
  }
  __syncthreads();
}

// forward DFT X_k = sum_n x_n e^{-2 pi i k n / D} in place: natural order in, bit-reversed out;
// tw[k] = e^{-2 pi i k / D}, k < D/2
template <typename CT>
__device__ void fft_dif(CT* X, const CT* __restrict__ tw, int D, int L) {
  int s = L - 1;
  while (s >= 0) {
    if (s >= 2) {
      dif_pass<CT, 3>(X, tw, D, s);
      s -= 3;
    } else if (s == 1) {
      dif_pass<CT, 2>(X, tw, D, s);
      s -= 2;
    } else {
      dif_pass<CT, 1>(X, tw, D, s);
      s -= 1;
    }
  }
}

// unnormalised inverse x_n = sum_k X_k e^{+2 pi i k n / D} in place: bit-reversed in, natural
// order out
template <typename CT>
__device__ void ifft_dit(CT* X, const CT* __restrict__ tw, int D, int L) {
  int s = 0;
  while (s < L) {
    if (L - s >= 3) {
      dit_pass<CT, 3>(X, tw, D, s);
      s += 3;
    } else if (L - s == 2) {
      dit_pass<CT, 2>(X, tw, D, s);
      s += 2;
    } else {
      dit_pass<CT, 1>(X, tw, D, s);
      s += 1;
    }
  }
}

// fixed-order block sum over the CTA (warp xor-tree, then thread 0 over the warp sums)
template <typename Tv>
__device__ Tv dft_block_sum(Tv v, Tv* sh) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    Tv tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += sh[i];
    sh[32] = tot;
  }
  __syncthreads();
  return sh[32];
}

}  // namespace

// ---- A V for pairs of systems (CG operator, FP32) ---------------------------------------
// CTA (t, p) applies A_tc to systems j = 2p and 2p + 1 of task t (the second absent when R is
// odd), writes Z and, when dots is set, the exact d^T A d of each system (the CG update reads
// it as a single partial).
__global__ void __launch_bounds__(kDftThreads)
k_dft_apply(const float* __restrict__ V, float* __restrict__ Z, float* __restrict__ dots,
            const float* __restrict__ mask_br, const float2* __restrict__ tw,
            const float* __restrict__ alpha, const int* __restrict__ task_active,
            unsigned long long* opcount, int R, int K, int Dp, int D, int L, int npair,
            float beta) {
  extern __shared__ float2 Xf[];
  __shared__ float sh[33];
  const int t = blockIdx.x / npair, p = blockIdx.x - t * npair;
  if (task_active != nullptr && task_active[t] == 0) return;
  const int j1 = 2 * p, j2 = 2 * p + 1;
  const bool has2 = j2 < R;
  const int64_t s1 = (int64_t)t * R + j1, s2 = has2 ? s1 + 1 : s1;
  const float* v1 = V + s1 * Dp;
  const float* v2 = V + s2 * Dp;
  for (int i = threadIdx.x; i < D; i += blockDim.x) Xf[pad(i)] = make_float2(v1[i], has2 ? v2[i] : 0.f);
  __syncthreads();
  fft_dif(Xf, tw, D, L);
  const float* m = mask_br + (int64_t)t * D;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const float mk = m[i];
    const float2 v = Xf[pad(i)];
    Xf[pad(i)] = make_float2(v.x * mk, v.y * mk);
  }
  __syncthreads();
  ifft_dit(Xf, tw, D, L);
  const float scale = beta / (float)D;
  const float* a1 = alpha + (int64_t)(j1 / (K + 1)) * Dp;
  const float* a2 = alpha + (int64_t)((has2 ? j2 : j1) / (K + 1)) * Dp;
  float dot1 = 0.f, dot2 = 0.f;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const float x1 = v1[i];
    const float2 xf = Xf[pad(i)];
    const float z1 = fmaf(scale, xf.x, a1[i] * x1);
    Z[s1 * Dp + i] = z1;
    dot1 = fmaf(x1, z1, dot1);
    if (has2) {
      const float x2 = v2[i];
      const float z2 = fmaf(scale, xf.y, a2[i] * x2);
      Z[s2 * Dp + i] = z2;
      dot2 = fmaf(x2, z2, dot2);
    }
  }
  if (dots != nullptr) {
    dot1 = dft_block_sum(dot1, sh);
    dot2 = dft_block_sum(dot2, sh);
    if (threadIdx.x == 0) {
      dots[s1] = dot1;
      if (has2) dots[s2] = dot2;
    }
  }
  if (opcount != nullptr && p == 0 && threadIdx.x == 0) atomicAdd(&opcount[t], 1ull);
}

// ---- one whole CG step (Alg. 1, loop body) for pairs of systems --------------------------
// The CTA holds both systems' full vectors, so the operator, d^T A d, the x and r updates,
// r^T r and the new direction need no second kernel: d is read for the transform and (from
// L2) for the updates; A d and then r stay in the shared buffer between the phases.  The
// per-system bookkeeping is that of the separate CG update kernel (breakdown stop, gamma and
// xi recorded for the first solve, convergence mask, step counts, counters).  With pminv the
// step is Jacobi-preconditioned: z = M^-1 r, rr = r^T z, d = z + xi d.
__global__ void __launch_bounds__(kDftThreads)
k_dft_cg_step(float* __restrict__ x, float* __restrict__ r, float* __restrict__ d,
              const float* __restrict__ mask_br, const float2* __restrict__ tw,
              const float* __restrict__ alpha, float* rr, const float* __restrict__ bb,
              int* steps, int* active, int* task_active, int* counters, float* gam, float* xih,
              int* psteps, unsigned long long* opcount, int record, int R, int K, int C, int Dp,
              int D, int L, int npair, int U, int cap, float beta, float tol2,
              const float* __restrict__ pminv) {
  extern __shared__ float2 Xf[];
  __shared__ float sh[33];
  __shared__ int s_go[2];
  const int t = blockIdx.x / npair, p = blockIdx.x - t * npair;
  if (task_active[t] == 0) return;
  const int j1 = 2 * p, j2 = 2 * p + 1;
  const bool has2 = j2 < R;
  const int64_t s1 = (int64_t)t * R + j1, s2 = has2 ? s1 + 1 : s1;
  const bool act1 = active[s1] != 0, act2 = has2 && active[s2] != 0;
  if (!act1 && !act2) return;                       // block-uniform
  if (opcount != nullptr && p == 0 && threadIdx.x == 0) atomicAdd(&opcount[t], 1ull);
  float* x1 = x + s1 * Dp;
  float* x2 = x + s2 * Dp;
  float* r1 = r + s1 * Dp;
  float* r2 = r + s2 * Dp;
  float* d1 = d + s1 * Dp;
  float* d2 = d + s2 * Dp;
  for (int i = threadIdx.x; i < D; i += blockDim.x) Xf[pad(i)] = make_float2(d1[i], has2 ? d2[i] : 0.f);
  __syncthreads();
  fft_dif(Xf, tw, D, L);
  const float* m = mask_br + (int64_t)t * D;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const float mk = m[i];
    const float2 v = Xf[pad(i)];
    Xf[pad(i)] = make_float2(v.x * mk, v.y * mk);
  }
  __syncthreads();
  ifft_dit(Xf, tw, D, L);
  // A d and d^T A d
  const float scale = beta / (float)D;
  const float* a1 = alpha + (int64_t)(j1 / (K + 1)) * Dp;
  const float* a2 = alpha + (int64_t)((has2 ? j2 : j1) / (K + 1)) * Dp;
  float dad1 = 0.f, dad2 = 0.f;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const float2 xf = Xf[pad(i)];
    const float dv1 = d1[i], dv2 = has2 ? d2[i] : 0.f;
    const float ad1 = fmaf(scale, xf.x, a1[i] * dv1);
    const float ad2 = has2 ? fmaf(scale, xf.y, a2[i] * dv2) : 0.f;
    Xf[pad(i)] = make_float2(ad1, ad2);
    dad1 = fmaf(dv1, ad1, dad1);
    dad2 = fmaf(dv2, ad2, dad2);
  }
  dad1 = dft_block_sum(dad1, sh);
  dad2 = dft_block_sum(dad2, sh);
  // breakdown (d^T A d <= 0 or not finite): stop the system
  bool go1 = act1, go2 = act2;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) {
      const bool act = q == 0 ? act1 : act2;
      const float dad = q == 0 ? dad1 : dad2;
      const int64_t sys = q == 0 ? s1 : s2;
      bool go = act;
      if (act && (!(dad > 0.f) || !isfinite(dad))) {
        active[sys] = 0;
        atomicSub(&task_active[t], 1);
        atomicSub(&counters[0], 1);
        if (!isfinite(dad)) atomicOr(&counters[2], 1);
        go = false;
      }
      s_go[q] = go ? 1 : 0;
    }
  }
  __syncthreads();
  go1 = s_go[0] != 0;
  go2 = s_go[1] != 0;
  if (!go1 && !go2) return;                         // block-uniform
  const float rr01 = rr[s1], rr02 = rr[s2];
  const float g1 = go1 ? rr01 / dad1 : 0.f, g2 = go2 ? rr02 / dad2 : 0.f;   // gamma_u
  // x += gamma d, r -= gamma A d; z = M^-1 r (z = r without the preconditioner); r^T z
  const float* mi1 = pminv != nullptr ? pminv + ((int64_t)t * C + j1 / (K + 1)) * Dp : nullptr;
  const float* mi2 = (pminv != nullptr && has2) ? pminv + ((int64_t)t * C + j2 / (K + 1)) * Dp
                                                : nullptr;
  float q1 = 0.f, q2 = 0.f;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const float2 ad = Xf[pad(i)];
    float zv1 = 0.f, zv2 = 0.f;
    if (go1) {
      x1[i] = fmaf(g1, d1[i], x1[i]);
      const float rv1 = fmaf(-g1, ad.x, r1[i]);
      r1[i] = rv1;
      zv1 = mi1 != nullptr ? rv1 * mi1[i] : rv1;
      q1 = fmaf(rv1, zv1, q1);
    }
    if (go2) {
      x2[i] = fmaf(g2, d2[i], x2[i]);
      const float rv2 = fmaf(-g2, ad.y, r2[i]);
      r2[i] = rv2;
      zv2 = mi2 != nullptr ? rv2 * mi2[i] : rv2;
      q2 = fmaf(rv2, zv2, q2);
    }
    Xf[pad(i)] = make_float2(zv1, zv2);
  }
  const float rr11 = dft_block_sum(q1, sh);
  const float rr12 = dft_block_sum(q2, sh);
  const float xi1 = go1 ? rr11 / rr01 : 0.f, xi2 = go2 ? rr12 / rr02 : 0.f;   // xi_u
  // d = z + xi d
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const float2 rv = Xf[pad(i)];
    if (go1) d1[i] = fmaf(xi1, d1[i], rv.x);
    if (go2) d2[i] = fmaf(xi2, d2[i], rv.y);
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) {
      if (!(q == 0 ? go1 : go2)) continue;
      const int64_t sys = q == 0 ? s1 : s2;
      const int j = q == 0 ? j1 : j2;
      const float g = q == 0 ? g1 : g2, xi = q == 0 ? xi1 : xi2, rr1 = q == 0 ? rr11 : rr12;
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
}

// ---- a whole CG solve (Alg. 1) for pairs of systems, persistent -----------------------------
// The same step as k_dft_cg_step (the same operations in the same order, so the same results
// bit for bit), looped inside the CTA until both systems stop (convergence,
// breakdown or the step cap): the CTA keeps its pair for the whole solve, so the pair's x, r
// and d (192 KiB at D = 8192) stay in L2 between steps and r^T r, the step counts and the
// convergence state stay in registers; no host poll and no launch per step.  maxsteps
// (counters[4]) receives the most steps any pair took, the operator applications the solve
// cost.
__global__ void __launch_bounds__(kDftThreads)
k_dft_cg_solve(float* __restrict__ x, float* __restrict__ r, float* __restrict__ d,
               const float* __restrict__ mask_br, const float2* __restrict__ tw,
               const float* __restrict__ alpha, float* rr, const float* __restrict__ bb,
               int* steps, int* active, int* task_active, int* counters, float* gam, float* xih,
               int* psteps, unsigned long long* opcount, int record, int R, int K, int C, int Dp,
               int D, int L, int npair, int U, int cap, float beta, float tol2,
               const float* __restrict__ pminv) {
  extern __shared__ float2 Xf[];
  __shared__ float sh[33];
  __shared__ int s_go[2];
  const int t = blockIdx.x / npair, p = blockIdx.x - t * npair;
  const int j1 = 2 * p, j2 = 2 * p + 1;
  const bool has2 = j2 < R;
  const int64_t s1 = (int64_t)t * R + j1, s2 = has2 ? s1 + 1 : s1;
  bool go1 = active[s1] != 0, go2 = has2 && active[s2] != 0;
  if (!go1 && !go2) return;                          // block-uniform
  float* x1 = x + s1 * Dp;
  float* x2 = x + s2 * Dp;
  float* r1 = r + s1 * Dp;
  float* r2 = r + s2 * Dp;
  float* d1 = d + s1 * Dp;
  float* d2 = d + s2 * Dp;
  const float* m = mask_br + (int64_t)t * D;
  const float scale = beta / (float)D;
  const float* a1 = alpha + (int64_t)(j1 / (K + 1)) * Dp;
  const float* a2 = alpha + (int64_t)((has2 ? j2 : j1) / (K + 1)) * Dp;
  const float* mi1 = pminv != nullptr ? pminv + ((int64_t)t * C + j1 / (K + 1)) * Dp : nullptr;
  const float* mi2 = (pminv != nullptr && has2) ? pminv + ((int64_t)t * C + j2 / (K + 1)) * Dp
                                                : nullptr;
  float rr01 = rr[s1], rr02 = rr[s2];
  int u1 = steps[s1], u2 = steps[s2];
  int nstep = 0;
  while (go1 || go2) {                               // block-uniform
    if (opcount != nullptr && p == 0 && threadIdx.x == 0) atomicAdd(&opcount[t], 1ull);
    ++nstep;
    for (int i = threadIdx.x; i < D; i += blockDim.x) Xf[pad(i)] = make_float2(d1[i], has2 ? d2[i] : 0.f);
    __syncthreads();
    fft_dif(Xf, tw, D, L);
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
      const float mk = m[i];
      const float2 v = Xf[pad(i)];
      Xf[pad(i)] = make_float2(v.x * mk, v.y * mk);
    }
    __syncthreads();
    ifft_dit(Xf, tw, D, L);
    float dad1 = 0.f, dad2 = 0.f;
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
      const float2 xf = Xf[pad(i)];
      const float dv1 = d1[i], dv2 = has2 ? d2[i] : 0.f;
      const float ad1 = fmaf(scale, xf.x, a1[i] * dv1);
      const float ad2 = has2 ? fmaf(scale, xf.y, a2[i] * dv2) : 0.f;
      Xf[pad(i)] = make_float2(ad1, ad2);
      dad1 = fmaf(dv1, ad1, dad1);
      dad2 = fmaf(dv2, ad2, dad2);
    }
    dad1 = dft_block_sum(dad1, sh);
    dad2 = dft_block_sum(dad2, sh);
    // breakdown (d^T A d <= 0 or not finite): stop the system
    if (threadIdx.x == 0) {
      for (int q = 0; q < 2; ++q) {
        const bool act = q == 0 ? go1 : go2;
        const float dad = q == 0 ? dad1 : dad2;
        const int64_t sys = q == 0 ? s1 : s2;
        bool go = act;
        if (act && (!(dad > 0.f) || !isfinite(dad))) {
          active[sys] = 0;
          atomicSub(&task_active[t], 1);
          atomicSub(&counters[0], 1);
          if (!isfinite(dad)) atomicOr(&counters[2], 1);
          go = false;
        }
        s_go[q] = go ? 1 : 0;
      }
    }
    __syncthreads();
    go1 = s_go[0] != 0;
    go2 = s_go[1] != 0;
    if (!go1 && !go2) break;                         // block-uniform
    const float g1 = go1 ? rr01 / dad1 : 0.f, g2 = go2 ? rr02 / dad2 : 0.f;   // gamma_u
    float q1 = 0.f, q2 = 0.f;
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
      const float2 ad = Xf[pad(i)];
      float zv1 = 0.f, zv2 = 0.f;
      if (go1) {
        x1[i] = fmaf(g1, d1[i], x1[i]);
        const float rv1 = fmaf(-g1, ad.x, r1[i]);
        r1[i] = rv1;
        zv1 = mi1 != nullptr ? rv1 * mi1[i] : rv1;
        q1 = fmaf(rv1, zv1, q1);
      }
      if (go2) {
        x2[i] = fmaf(g2, d2[i], x2[i]);
        const float rv2 = fmaf(-g2, ad.y, r2[i]);
        r2[i] = rv2;
        zv2 = mi2 != nullptr ? rv2 * mi2[i] : rv2;
        q2 = fmaf(rv2, zv2, q2);
      }
      Xf[pad(i)] = make_float2(zv1, zv2);
    }
    const float rr11 = dft_block_sum(q1, sh);
    const float rr12 = dft_block_sum(q2, sh);
    const float xi1 = go1 ? rr11 / rr01 : 0.f, xi2 = go2 ? rr12 / rr02 : 0.f;   // xi_u
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
      const float2 rv = Xf[pad(i)];
      if (go1) d1[i] = fmaf(xi1, d1[i], rv.x);
      if (go2) d2[i] = fmaf(xi2, d2[i], rv.y);
    }
    // per-system bookkeeping, as in the step kernel; every thread takes the same decisions
    bool done1 = false, done2 = false;
    for (int q = 0; q < 2; ++q) {
      if (!(q == 0 ? go1 : go2)) continue;
      const int64_t sys = q == 0 ? s1 : s2;
      const int j = q == 0 ? j1 : j2;
      const float g = q == 0 ? g1 : g2, xi = q == 0 ? xi1 : xi2, rr1 = q == 0 ? rr11 : rr12;
      const int u = q == 0 ? u1 : u2;
      const bool done = (rr1 <= tol2 * bb[sys]) || (rr1 == 0.f) || (u + 1 >= cap) || !isfinite(rr1);
      if (threadIdx.x == 0) {
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
        if (done) {
          active[sys] = 0;
          atomicSub(&task_active[t], 1);
          atomicSub(&counters[0], 1);
        }
      }
      if (q == 0) { u1 = u + 1; rr01 = rr11; done1 = done; }
      else { u2 = u + 1; rr02 = rr12; done2 = done; }
    }
    go1 = go1 && !done1;
    go2 = go2 && !done2;
    __syncthreads();                                 // d and Xf complete before the next step
  }
  if (threadIdx.x == 0) atomicMax(&counters[4], nstep);
}

// ---- refinement residual b - A x in FP64 ------------------------------------------------
// Columns j' < Rc of each task are systems j = j' * jstride (all R, or the means only); pairs
// (2p, 2p+1) share a transform.  b is Bext when given, else b0 (k = 0) or the probe.  Systems
// that stopped refining are skipped (pairs with neither refining do no work), and get 0.
__global__ void __launch_bounds__(kDftThreads)
k_dft_residual(const float* __restrict__ X, const float* __restrict__ Bext,
               const float* __restrict__ b0hi, const float* __restrict__ b0lo,
               float* __restrict__ Rout, const int* __restrict__ ractive,
               const float* __restrict__ mask_br, const double2* __restrict__ tw,
               const float* __restrict__ alpha, int R, int K, int C, int Dp, int D, int L, int Rc,
               int jstride, int npair, double beta, uint64_t seed, int64_t em_iter, int toff,
               const float* __restrict__ pw, int pshare) {
  extern __shared__ double2 Xd[];
  const int t = blockIdx.x / npair, p = blockIdx.x - t * npair;
  const int jp1 = 2 * p, jp2 = 2 * p + 1;
  const bool has2 = jp2 < Rc;
  const int j1 = jp1 * jstride, j2 = has2 ? jp2 * jstride : j1;
  const int64_t s1 = (int64_t)t * R + j1, s2 = (int64_t)t * R + j2;
  const bool on1 = ractive == nullptr || ractive[s1] != 0;
  const bool on2 = has2 && (ractive == nullptr || ractive[s2] != 0);
  if (!on1 && !on2) return;                         // block-uniform
  const float* x1 = X + s1 * Dp;
  const float* x2 = X + s2 * Dp;
  for (int i = threadIdx.x; i < D; i += blockDim.x)
    Xd[pad(i)] = make_double2(on1 ? (double)x1[i] : 0.0, on2 ? (double)x2[i] : 0.0);
  __syncthreads();
  fft_dif(Xd, tw, D, L);
  const float* m = mask_br + (int64_t)t * D;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const double mk = (double)m[i];
    const double2 v = Xd[pad(i)];
    Xd[pad(i)] = make_double2(v.x * mk, v.y * mk);
  }
  __syncthreads();
  ifft_dit(Xd, tw, D, L);
  const double scale = beta / (double)D;
  const int c1 = j1 / (K + 1), k1 = j1 - c1 * (K + 1);
  const int c2 = j2 / (K + 1), k2 = j2 - c2 * (K + 1);
  const float* a1 = alpha + (int64_t)c1 * Dp;
  const float* a2 = alpha + (int64_t)c2 * Dp;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const double b0 = (double)b0hi[(int64_t)t * Dp + i] + (double)b0lo[(int64_t)t * Dp + i];
    for (int q = 0; q < 2; ++q) {
      const bool on = q == 0 ? on1 : on2;
      if (q == 1 && !has2) break;
      const int64_t s = q == 0 ? s1 : s2;
      const int c = q == 0 ? c1 : c2, k = q == 0 ? k1 : k2;
      double rv = 0.0;
      if (on) {
        double b;
        if (Bext != nullptr) {
          b = (double)Bext[s * Dp + i];
        } else if (k == 0) {
          b = b0;
        } else {
          const uint32_t bits = probe_bits32(seed, em_iter, t + toff, probe_cluster(c, pshare),
                                             C, k - 1, i & ~31);
          b = ((bits >> (i & 31)) & 1u) ? -1.0 : 1.0;
          if (pw != nullptr) b *= (double)pw[((int64_t)t * C + c) * Dp + i];   // sqrt(m) p
        }
        const double xv = (double)(q == 0 ? x1[i] : x2[i]);
        const double2 xd = Xd[pad(i)];
        const double z = fma(scale, q == 0 ? xd.x : xd.y, (double)(q == 0 ? a1[i] : a2[i]) * xv);
        rv = b - z;
      }
      Rout[s * Dp + i] = (float)rv;
    }
  }
}

// ---- b0_t = beta Re(Phi_t^H y_t) = beta Re(sum_k Y_k e^{+2 pi i k d / D}) / sqrt(D) ------
// Y is the measured spectrum, zero at the frequencies not sampled; it is scattered straight
// into bit-reversed positions for the decimation-in-time inverse.  Kept as an FP32 pair.
__global__ void __launch_bounds__(kDftThreads)
k_dft_b0(const float2* __restrict__ y, const int* __restrict__ freq,
         const int64_t* __restrict__ off, float* __restrict__ b0hi, float* __restrict__ b0lo,
         const double2* __restrict__ tw, int Dp, int D, int L, double beta) {
  extern __shared__ double2 Xd[];
  const int t = blockIdx.x;
  for (int i = threadIdx.x; i < D; i += blockDim.x) Xd[pad(i)] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int64_t q = off[t] + threadIdx.x; q < off[t + 1]; q += blockDim.x) {
    const int k = freq[q];
    const int pos = (int)(__brev((unsigned)k) >> (32 - L));
    Xd[pad(pos)] = make_double2((double)y[q].x, (double)y[q].y);
  }
  __syncthreads();
  ifft_dit(Xd, tw, D, L);
  const double scale = beta / sqrt((double)D);
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const double b = scale * Xd[pad(i)].x;
    const float hi = (float)b;
    b0hi[(int64_t)t * Dp + i] = hi;
    b0lo[(int64_t)t * Dp + i] = (float)(b - (double)hi);
  }
}

// ---- host side ----------------------------------------------------------------------------
namespace {
bool dft_small_ok(int D) { return D >= 128 && D <= kDftMaxD && (D & (D - 1)) == 0; }
}  // namespace

bool dft_size_ok(int D) { return dft_small_ok(D) || dft_large_ok(D); }

int dft_create(Ctx* c, const uint8_t* mask, const float* y, int on_device) {
  const int T = c->T, D = c->D;
  int L = 0;
  while ((1 << L) < D) ++L;
  c->dft_L = L;
  // CMCS_DFT_FOURSTEP=1 (evaluation switch) takes the four-step path at every supported D
  const char* fsenv = getenv("CMCS_DFT_FOURSTEP");
  const bool force = fsenv != nullptr && fsenv[0] == '1' && dft_large_ok(D);
  c->dft_large = (dft_small_ok(D) && !force) ? 0 : 1;
  c->dft_ndt = 1;
  std::vector<uint8_t> hm((size_t)T * D);
  if (on_device) {
    if (cudaMemcpy(hm.data(), mask, hm.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  } else {
    memcpy(hm.data(), mask, hm.size());
  }
  // sampled frequencies (ascending) and the symmetrised mask in bit-reversed order
  std::vector<int> freq;
  std::vector<int64_t> off((size_t)T + 1, 0);
  std::vector<float> mbr((size_t)T * D);
  for (int t = 0; t < T; ++t) {
    const uint8_t* m = hm.data() + (size_t)t * D;
    for (int k = 0; k < D; ++k)
      if (m[k]) freq.push_back(k);
    off[(size_t)t + 1] = (int64_t)freq.size();
    if (off[(size_t)t + 1] - off[(size_t)t] != c->hN[t] / 2) return 5;
    for (int pos = 0; !c->dft_large && pos < D; ++pos) {
      unsigned k = 0;
      for (int b = 0; b < L; ++b) k |= (unsigned)((pos >> b) & 1) << (L - 1 - b);
      const int kk = (int)k, km = (D - kk) & (D - 1);
      mbr[(size_t)t * D + pos] = 0.5f * (float)((m[kk] ? 1 : 0) + (m[km] ? 1 : 0));
    }
  }
  // twiddles e^{-2 pi i k / D}, k < D/2, evaluated in FP64
  std::vector<float2> tw32((size_t)D / 2);
  std::vector<double2> tw64((size_t)D / 2);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < D / 2; ++k) {
    const double a = -2.0 * pi * (double)k / (double)D;
    tw64[(size_t)k] = make_double2(cos(a), sin(a));
    tw32[(size_t)k] = make_float2((float)cos(a), (float)sin(a));
  }
  const size_t nf = freq.size();
  bool ok = cudaMalloc(reinterpret_cast<void**>(&c->dft_mask), sizeof(float) * mbr.size()) == cudaSuccess &&
            cudaMalloc(&c->dft_tw32, sizeof(float2) * tw32.size()) == cudaSuccess &&
            cudaMalloc(&c->dft_tw64, sizeof(double2) * tw64.size()) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&c->dft_freq), sizeof(int) * (nf > 0 ? nf : 1)) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&c->dft_off), sizeof(int64_t) * off.size()) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&c->dft_y), sizeof(float) * 2 * (nf > 0 ? nf : 1)) == cudaSuccess;
  if (!ok) return 2;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  ok = cudaMemcpy(c->dft_mask, mbr.data(), sizeof(float) * mbr.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->dft_tw32, tw32.data(), sizeof(float2) * tw32.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->dft_tw64, tw64.data(), sizeof(double2) * tw64.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->dft_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok && nf > 0)
    ok = cudaMemcpy(c->dft_freq, freq.data(), sizeof(int) * nf, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->dft_y, y, sizeof(float) * 2 * nf, kin) == cudaSuccess;
  // the real-stacked measurements [Re y_t; Im y_t] for the likelihood constant
  for (int t = 0; ok && t < T; ++t) {
    const int64_t n = off[(size_t)t + 1] - off[(size_t)t];
    if (n == 0) continue;
    const float* src = y + 2 * off[(size_t)t];
    ok = cudaMemcpy2D(c->y + c->hrow[t], sizeof(float), src, 2 * sizeof(float), sizeof(float),
                      (size_t)n, kin) == cudaSuccess &&
         cudaMemcpy2D(c->y + c->hrow[t] + n, sizeof(float), src + 1, 2 * sizeof(float),
                      sizeof(float), (size_t)n, kin) == cudaSuccess;
  }
  if (!ok) return 3;
  if (c->dft_large) return fs_create(c, hm.data());
  const int sm32 = (int)sizeof(float2) * (D + D / 32), sm64 = (int)sizeof(double2) * (D + D / 32);
  if (cudaFuncSetAttribute(k_dft_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, sm32) != cudaSuccess ||
      cudaFuncSetAttribute(k_dft_cg_step, cudaFuncAttributeMaxDynamicSharedMemorySize, sm32) != cudaSuccess ||
      cudaFuncSetAttribute(k_dft_cg_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, sm32) != cudaSuccess ||
      cudaFuncSetAttribute(k_dft_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, sm64) != cudaSuccess ||
      cudaFuncSetAttribute(k_dft_b0, cudaFuncAttributeMaxDynamicSharedMemorySize, sm64) != cudaSuccess)
    return 4;
  return 0;
}

void dft_destroy(Ctx* c) {
  fs_destroy(c);
  void* ptrs[] = {c->dft_mask, c->dft_tw32, c->dft_tw64, c->dft_freq, c->dft_off, c->dft_y};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

cudaError_t launch_dft_apply(Ctx* c, const float* V, float* Z, int with_dots) {
  if (c->dft_large) return fs_apply(c, V, Z, with_dots);
  const int npair = (c->R + 1) / 2;
  c->launches += 1;
  k_dft_apply<<<c->T * npair, kDftThreads, sizeof(float2) * (c->D + c->D / 32), c->stream>>>(
      V, Z, with_dots ? c->part : nullptr, c->dft_mask, static_cast<const float2*>(c->dft_tw32),
      c->alpha, with_dots ? c->task_active : nullptr,
      c->prof_on ? reinterpret_cast<unsigned long long*>(c->opcount) : nullptr, c->R, c->K, c->Dp,
      c->D, c->dft_L, npair, (float)c->beta);
  return cudaGetLastError();
}

cudaError_t launch_dft_residual(Ctx* c, const float* X, const float* Bext, float* Rout,
                                int all_systems, int means_only) {
  if (c->dft_large) return fs_residual(c, X, Bext, Rout, all_systems, means_only);
  const int Rc = means_only ? c->C : c->R;
  const int js = means_only ? c->K + 1 : 1;
  const int npair = (Rc + 1) / 2;
  c->launches += 1;
  k_dft_residual<<<c->T * npair, kDftThreads, sizeof(double2) * (c->D + c->D / 32), c->stream>>>(
      X, Bext, c->b0hi, c->b0lo, Rout, (Bext || all_systems) ? nullptr : c->ractive, c->dft_mask,
      static_cast<const double2*>(c->dft_tw64), c->alpha, c->R, c->K, c->C, c->Dp, c->D, c->dft_L,
      Rc, js, npair, c->beta, c->seed, c->em_iter, c->toff, c->precond ? c->pw : nullptr,
      c->pshare);
  return cudaGetLastError();
}

cudaError_t launch_dft_cg_step(Ctx* c, int record) {
  if (c->dft_large) return cudaErrorInvalidValue;   // the four-step path updates separately
  const int npair = (c->R + 1) / 2;
  c->launches += 1;
  k_dft_cg_step<<<c->T * npair, kDftThreads, sizeof(float2) * (c->D + c->D / 32), c->stream>>>(
      c->x, c->r, c->d, c->dft_mask, static_cast<const float2*>(c->dft_tw32), c->alpha, c->rr,
      c->bb, c->steps, c->active, c->task_active, c->counters, c->gam, c->xi, c->psteps,
      c->prof_on ? reinterpret_cast<unsigned long long*>(c->opcount) : nullptr, record, c->R,
      c->K, c->C, c->Dp, c->D, c->dft_L, npair, c->U, cg_cap(c), (float)c->beta,
      (float)(c->cg_tol * c->cg_tol), c->precond ? c->pminv : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_dft_cg_solve(Ctx* c, int record) {
  if (c->dft_large) return cudaErrorInvalidValue;
  const int npair = (c->R + 1) / 2;
  c->launches += 1;
  k_dft_cg_solve<<<c->T * npair, kDftThreads, sizeof(float2) * (c->D + c->D / 32), c->stream>>>(
      c->x, c->r, c->d, c->dft_mask, static_cast<const float2*>(c->dft_tw32), c->alpha, c->rr,
      c->bb, c->steps, c->active, c->task_active, c->counters, c->gam, c->xi, c->psteps,
      c->prof_on ? reinterpret_cast<unsigned long long*>(c->opcount) : nullptr, record, c->R,
      c->K, c->C, c->Dp, c->D, c->dft_L, npair, c->U, cg_cap(c), (float)c->beta,
      (float)(c->cg_tol * c->cg_tol), c->precond ? c->pminv : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_dft_b0(Ctx* c) {
  if (c->dft_large) return fs_b0(c);
  c->launches += 1;
  k_dft_b0<<<c->T, kDftThreads, sizeof(double2) * (c->D + c->D / 32), c->stream>>>(
      reinterpret_cast<const float2*>(c->dft_y), c->dft_freq, c->dft_off, c->b0hi, c->b0lo,
      static_cast<const double2*>(c->dft_tw64), c->Dp, c->D, c->dft_L, c->beta);
  return cudaGetLastError();
}

}  // namespace cmcs
