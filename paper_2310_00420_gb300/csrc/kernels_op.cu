// Batched operator A_tc V = beta Phi_t^T (Phi_t V) + alpha_c * V (Eq. 7; Sec. 3.3 notes that CG
// needs only this product) for all R = C*(K+1) right-hand sides of every task at once, as two
// FP32 SIMT GEMMs per task, plus the compensated variant that forms the refinement residual.
//
// Pass 1: W[t][j][n] = sum_d Phi_t[n][d] V[t][j][d]   (M = N_t rows, N = R, K = D)
// Pass 2: Z[t][j][d] = beta sum_n Phi_t[n][d] W[t][j][n] + alpha_c[d] V[t][j][d]
//         (M = D, N = R, K = N_t), with the per-system partial d^T A d of each 128-wide
//         coordinate tile written for the CG update (deterministic, no atomics).
// Tiles: 256 threads as 16 x 16; each thread owns 8 rows (two runs of 4, so shared-memory
// reads are conflict-free float4s) by TN columns; BK = 16; the next k-tile is prefetched into
// registers.  The plain kernels double-buffer shared memory; the DS kernels keep one buffer
// (at most ~15 KB), which measured faster for them (fewer registers, more resident CTAs).
// The residual variant ("DS") keeps every accumulator as an unevaluated FP32 pair hi + lo:
// products are split exactly with an FMA (TwoProduct) and added with Knuth's TwoSum, the
// compensated dot product of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26(6), 2005),
// giving about twice FP32's precision; the epilogue forms b - A x in FP64 per element.
#include "cmcs_internal.cuh"

namespace cmcs {

namespace {

// k-steps unrolled in the DS kernels: the fully unrolled body (16 k x TN x 8 compensated
// multiply-adds of ~10 instructions) overflows the instruction cache
#ifndef CMCS_DS_UNROLL
#define CMCS_DS_UNROLL 4
#endif
constexpr int kUnrollDS = CMCS_DS_UNROLL;
#ifndef CMCS_DS_P2_MINB
#define CMCS_DS_P2_MINB 2
#endif
constexpr int kP2MinBlocksDS = CMCS_DS_P2_MINB;     // DS pass 2: two resident CTAs (50.6 vs 51.6 ms)

template <bool DS>
__device__ __forceinline__ void mac(float& hi, float& lo, float a, float b) {
  if constexpr (DS) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);       // a*b = p + e exactly
    const float s = __fadd_rn(hi, p);          // TwoSum(hi, p) = s + err
    const float bv = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  } else {
    hi = fmaf(a, b, hi);
  }
}

// pass 2 of the residual multiplies Phi by (w_hi + w_lo): exact product with w_hi, plain
// product with w_lo folded into the low part
template <bool DS>
__device__ __forceinline__ void mac2(float& hi, float& lo, float a, float bh, float bl) {
  mac<DS>(hi, lo, a, bh);
  if constexpr (DS) lo = __fmaf_rn(a, bl, lo);
}

__device__ __forceinline__ float probe_sign(uint32_t bits, int sh) {
  return ((bits >> sh) & 1u) ? -1.0f : 1.0f;
}

// whether any of the columns j' in [j0, j0 + bn) of task t (systems t R + j' jstride) is
// still refining; block-uniform.  A residual tile with none is skipped: such systems are
// not refined again, so their residual entries are never read.
__device__ __forceinline__ bool tile_refining(const int* ractive, int t, int R, int j0, int bn,
                                              int Rc, int jstride) {
  int any = 0;
  for (int jj = threadIdx.x; jj < bn; jj += blockDim.x)
    if (j0 + jj < Rc && ractive[(int64_t)t * R + (int64_t)(j0 + jj) * jstride] != 0) any = 1;
  return __syncthreads_or(any) != 0;
}

}  // namespace

// --------------------------------------------------------------------------------------
// Pass 1
// --------------------------------------------------------------------------------------
template <int TN, bool DS>
__global__ void __launch_bounds__(256)
k_pass1(const float* __restrict__ phi, const float* __restrict__ V, float* __restrict__ W,
        float* __restrict__ Wlo, const int64_t* __restrict__ drow,
        const int* __restrict__ tile_task, const int* __restrict__ task_active,
        const int* __restrict__ ractive, int R, int Dp, int Rc, int jstride, int g0, int ntiles) {
  // columns j' = 0 .. Rc-1 of the tile are systems j = j' * jstride of the task (all R
  // systems when Rc = R, jstride = 1; the mean systems only when Rc = C, jstride = K + 1)
  constexpr int BN = 16 * TN;
  constexpr int NB = (BN * 4 + 255) / 256;
  constexpr int NBUF = DS ? 1 : 2;     // DS: one shared-memory buffer (see top)
  __shared__ __align__(16) float As[NBUF][16][132];
  __shared__ __align__(16) float Bs[NBUF][16][BN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // tiles (row tile, column tile), column tiles of a row tile adjacent; a grid smaller than
  // the tile count makes the kernel persistent
  const int ncx = (Rc + BN - 1) / BN;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int g = g0 + tile / ncx;
    const int t = tile_task[g];
    if (task_active != nullptr && task_active[t] == 0) continue;
    const int64_t row0 = (int64_t)g * 128;
    const int64_t rbeg = drow[t];
    const int64_t Np = drow[t + 1] - rbeg;
    const int64_t nl0 = row0 - rbeg;
    const int j0 = (tile % ncx) * BN;
    if (DS && ractive != nullptr && !tile_refining(ractive, t, R, j0, BN, Rc, jstride)) continue;
    const float* Ag = phi + row0 * Dp;
    const float* Vg = V + (int64_t)t * R * Dp;

    float hi[8][TN], lo[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int jj = 0; jj < TN; ++jj) hi[i][jj] = lo[i][jj] = 0.f;

    float4 ra[2], rb[NB];
    auto load = [&](int k0) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int idx = tid + 256 * q, row = idx >> 2, c4 = idx & 3;
        ra[q] = *reinterpret_cast<const float4*>(Ag + (int64_t)row * Dp + k0 + c4 * 4);
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const int idx = tid + 256 * q, row = idx >> 2, c4 = idx & 3, j = j0 + row;
        rb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < BN * 4 && j < Rc)
          rb[q] = *reinterpret_cast<const float4*>(Vg + (int64_t)j * jstride * Dp + k0 + c4 * 4);
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int idx = tid + 256 * q, row = idx >> 2, c4 = idx & 3;
        As[buf][c4 * 4 + 0][row] = ra[q].x;
        As[buf][c4 * 4 + 1][row] = ra[q].y;
        As[buf][c4 * 4 + 2][row] = ra[q].z;
        As[buf][c4 * 4 + 3][row] = ra[q].w;
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const int idx = tid + 256 * q, row = idx >> 2, c4 = idx & 3;
        if (idx < BN * 4) {
          Bs[buf][c4 * 4 + 0][row] = rb[q].x;
          Bs[buf][c4 * 4 + 1][row] = rb[q].y;
          Bs[buf][c4 * 4 + 2][row] = rb[q].z;
          Bs[buf][c4 * 4 + 3][row] = rb[q].w;
        }
      }
    };

    load(0);
    store(0);
    __syncthreads();
    const int nk = Dp / 16;
    for (int kt = 0; kt < nk; ++kt) {
      const int buf = NBUF == 2 ? (kt & 1) : 0;
      if (kt + 1 < nk) load((kt + 1) * 16);
#pragma unroll(DS ? kUnrollDS : 16)
      for (int k = 0; k < 16; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][tx * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float b[TN];
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) b[jj] = Bs[buf][k][ty + 16 * jj];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int jj = 0; jj < TN; ++jj) mac<DS>(hi[i][jj], lo[i][jj], a[i], b[jj]);
      }
      if constexpr (NBUF == 1) __syncthreads();
      if (kt + 1 < nk) store(buf ^ (NBUF - 1));
      __syncthreads();
    }

    float* Wt = W + rbeg * Rc;
    float* Wlt = DS ? Wlo + rbeg * Rc : nullptr;
#pragma unroll
    for (int jj = 0; jj < TN; ++jj) {
      const int j = j0 + ty + 16 * jj;
      if (j >= Rc) continue;
      float* wr = Wt + (int64_t)j * Np + nl0;
      *reinterpret_cast<float4*>(wr + tx * 4) = make_float4(hi[0][jj], hi[1][jj], hi[2][jj], hi[3][jj]);
      *reinterpret_cast<float4*>(wr + 64 + tx * 4) = make_float4(hi[4][jj], hi[5][jj], hi[6][jj], hi[7][jj]);
      if constexpr (DS) {
        float* wl = Wlt + (int64_t)j * Np + nl0;
        *reinterpret_cast<float4*>(wl + tx * 4) = make_float4(lo[0][jj], lo[1][jj], lo[2][jj], lo[3][jj]);
        *reinterpret_cast<float4*>(wl + 64 + tx * 4) = make_float4(lo[4][jj], lo[5][jj], lo[6][jj], lo[7][jj]);
      }
    }
  }
}

// --------------------------------------------------------------------------------------
// Pass 2 with the operator epilogue (plain) or the residual epilogue (DS)
// --------------------------------------------------------------------------------------
struct P2Args {
  const float* phi;
  const float* W;
  const float* Wlo;
  const float* V;        // plain: the vectors A is applied to; DS: the solutions x
  float* Z;              // plain: A V; DS: the residual B - A x (FP32-rounded)
  float* part;           // [Dp/128][S] partial v^T A v (plain, may be null)
  const float* alpha;    // [C][Dp]
  const float* b0hi;     // [T][Dp]
  const float* b0lo;     // [T][Dp]
  const float* Bext;     // DS: explicit right-hand sides [S][Dp] or null
  const int* ractive;    // DS: systems still refining (null: all)
  const int64_t* drow;
  const int* task_active;
  unsigned long long* opcount;  // [T] applications per task (plain pass only, may be null)
  int R, K, C, Dp, D, S;
  int Rc, jstride;        // columns processed: systems j = j' * jstride, j' < Rc
  int t0;                 // first task of the launch
  int ntiles;             // (task, coordinate tile, column tile) tiles from task t0 on
  float beta_f;
  double beta_d;
  uint64_t seed;
  int64_t em_iter;
  int toff;               // global index of the context's first task (probe counters)
  const float* pw;        // DS: sqrt(m) [T*C][Dp] scaling the probe right-hand sides, or null
  int pshare;             // DS: probes shared across clusters
};

template <int TN, bool DS>
__global__ void __launch_bounds__(256, DS ? kP2MinBlocksDS : 1) k_pass2(P2Args p) {
  constexpr int BN = 16 * TN;
  constexpr int NB = (BN * 4 + 255) / 256;
  constexpr int NBUF = DS ? 1 : 2;
  __shared__ __align__(16) float As[NBUF][16][128];
  __shared__ __align__(16) float Bs[NBUF][16][BN + 4];
  __shared__ __align__(16) float Bl[NBUF][16][DS ? BN + 4 : 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int ncx = (p.Rc + BN - 1) / BN, ndt = p.Dp / 128;
  for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
    const int t = p.t0 + tile / (ndt * ncx);
    if (p.task_active != nullptr && p.task_active[t] == 0) continue;
    const int dt = (tile / ncx) % ndt;
    const int d0 = dt * 128;
    const int j0 = (tile % ncx) * BN;
    if (DS && p.ractive != nullptr && !tile_refining(p.ractive, t, p.R, j0, BN, p.Rc, p.jstride))
      continue;
    if (!DS && p.opcount != nullptr && j0 == 0 && dt == 0 && threadIdx.x == 0)
      atomicAdd(&p.opcount[t], 1ull);
    const int64_t rbeg = p.drow[t];
    const int64_t Np = p.drow[t + 1] - rbeg;
    const float* Ag = p.phi + rbeg * p.Dp + d0;
    const float* Wt = p.W + rbeg * p.Rc;
    const float* Wlt = DS ? p.Wlo + rbeg * p.Rc : nullptr;

    float hi[8][TN], lo[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int jj = 0; jj < TN; ++jj) hi[i][jj] = lo[i][jj] = 0.f;

    float4 ra[2], rb[NB], rl[DS ? NB : 1];
    auto load = [&](int64_t n0) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int idx = tid + 256 * q, row = idx >> 5, c4 = idx & 31;
        ra[q] = *reinterpret_cast<const float4*>(Ag + (n0 + row) * p.Dp + c4 * 4);
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const int idx = tid + 256 * q, row = idx >> 2, c4 = idx & 3, j = j0 + row;
        rb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (DS) rl[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < BN * 4 && j < p.Rc) {
          rb[q] = *reinterpret_cast<const float4*>(Wt + (int64_t)j * Np + n0 + c4 * 4);
          if constexpr (DS) rl[q] = *reinterpret_cast<const float4*>(Wlt + (int64_t)j * Np + n0 + c4 * 4);
        }
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int idx = tid + 256 * q, row = idx >> 5, c4 = idx & 31;
        *reinterpret_cast<float4*>(&As[buf][row][c4 * 4]) = ra[q];
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const int idx = tid + 256 * q, row = idx >> 2, c4 = idx & 3;
        if (idx < BN * 4) {
          Bs[buf][c4 * 4 + 0][row] = rb[q].x;
          Bs[buf][c4 * 4 + 1][row] = rb[q].y;
          Bs[buf][c4 * 4 + 2][row] = rb[q].z;
          Bs[buf][c4 * 4 + 3][row] = rb[q].w;
          if constexpr (DS) {
            Bl[buf][c4 * 4 + 0][row] = rl[q].x;
            Bl[buf][c4 * 4 + 1][row] = rl[q].y;
            Bl[buf][c4 * 4 + 2][row] = rl[q].z;
            Bl[buf][c4 * 4 + 3][row] = rl[q].w;
          }
        }
      }
    };

    load(0);
    store(0);
    __syncthreads();
    const int64_t nk = Np / 16;
    for (int64_t kt = 0; kt < nk; ++kt) {
      const int buf = NBUF == 2 ? (int)(kt & 1) : 0;
      if (kt + 1 < nk) load((kt + 1) * 16);
#pragma unroll(DS ? kUnrollDS : 16)
      for (int k = 0; k < 16; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][tx * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float b[TN], bl[TN];
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
          b[jj] = Bs[buf][k][ty + 16 * jj];
          bl[jj] = DS ? Bl[buf][k][ty + 16 * jj] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int jj = 0; jj < TN; ++jj) mac2<DS>(hi[i][jj], lo[i][jj], a[i], b[jj], bl[jj]);
      }
      if constexpr (NBUF == 1) __syncthreads();
      if (kt + 1 < nk) store(buf ^ (NBUF - 1));
      __syncthreads();
    }

    // epilogue
#pragma unroll
    for (int jj = 0; jj < TN; ++jj) {
      const int jc = j0 + ty + 16 * jj;
      const bool valid = jc < p.Rc;
      const int j = jc * p.jstride;
      const int64_t sys = (int64_t)t * p.R + j;
      const int c = j / (p.K + 1);
      const int k = j - c * (p.K + 1);
      float dot = 0.f;
      if (valid) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int dd = d0 + half * 64 + tx * 4;
          const float4 v = *reinterpret_cast<const float4*>(p.V + sys * p.Dp + dd);
          const float4 al = *reinterpret_cast<const float4*>(p.alpha + (int64_t)c * p.Dp + dd);
          const float vv[4] = {v.x, v.y, v.z, v.w};
          const float aa[4] = {al.x, al.y, al.z, al.w};
          float out[4];
          if constexpr (!DS) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              out[e] = fmaf(p.beta_f, hi[half * 4 + e][jj], aa[e] * vv[e]);
              dot = fmaf(vv[e], out[e], dot);
            }
          } else {
            const bool on = (p.ractive == nullptr) || (p.ractive[sys] != 0);
            uint32_t bits = 0;
            if (on && p.Bext == nullptr && k > 0)
              bits = probe_bits32(p.seed, p.em_iter, t + p.toff, probe_cluster(c, p.pshare), p.C, k - 1,
                                  dd & ~31);
            const float* wv = (p.pw != nullptr && k > 0)
                                  ? p.pw + ((int64_t)t * p.C + c) * p.Dp : nullptr;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int d = dd + e;
              double b = 0.0;
              if (p.Bext != nullptr) {
                b = (double)p.Bext[sys * p.Dp + d];
              } else if (d < p.D) {
                b = (k == 0) ? (double)p.b0hi[(int64_t)t * p.Dp + d] + (double)p.b0lo[(int64_t)t * p.Dp + d]
                             : (double)probe_sign(bits, (d & 31));
                if (wv != nullptr) b *= (double)wv[d];
              }
              const double z = (double)hi[half * 4 + e][jj] + (double)lo[half * 4 + e][jj];
              const double rv = b - p.beta_d * z - (double)aa[e] * (double)vv[e];
              out[e] = on ? (float)rv : 0.f;
            }
          }
          *reinterpret_cast<float4*>(p.Z + sys * p.Dp + dd) = make_float4(out[0], out[1], out[2], out[3]);
        }
      }
      if constexpr (!DS) {
#pragma unroll
        for (int m = 1; m < 16; m <<= 1) dot += __shfl_xor_sync(0xffffffffu, dot, m);
        if (tx == 0 && valid && p.part != nullptr) p.part[(int64_t)dt * p.S + sys] = dot;
      }
    }
  }
}

// --------------------------------------------------------------------------------------
// Narrow right-hand-side blocks (R <= 8, e.g. the adjoint's C systems per task): the operator
// as two GEMVs.  With so few columns the GEMM tiles above would mostly compute padding, and
// the work is bound by reading Phi: each pass streams Phi once, row segments as float4 loads
// coalesced across the warp.
// Pass 1: a warp takes 8 rows of one task; for every float4 of d it loads the R vectors once
// (L1-cached) and the 8 rows' Phi, keeps 8 x R accumulators and reduces them across the warp.
// Pass 2: a CTA of 128 threads takes 512 coordinates of one task, each thread four of them
// for all R systems; the task's W is staged in shared memory 256 rows at a time.  Epilogue as
// in k_pass2: Z = beta Phi^T W + alpha_c V and the per-128-coordinate partials of v^T A v.
// --------------------------------------------------------------------------------------
constexpr int kGemvMaxR = 8;        // widest right-hand-side block run as two GEMVs
constexpr int kGvRows = 8;          // rows per warp in pass 1
constexpr int kGvWarps = 4;         // warps per CTA in pass 1
constexpr int kGvChunk = 256;       // rows of W staged per step of pass 2

template <int NR>
__global__ void __launch_bounds__(32 * kGvWarps)
k_gemv1(const float* __restrict__ phi, const float* __restrict__ V, float* __restrict__ W,
        const int64_t* __restrict__ drow, const int* __restrict__ tile_task,
        const int* __restrict__ task_active, int R, int Dp, int64_t rows_total) {
  const int lane = threadIdx.x & 31;
  const int64_t n0 = ((int64_t)blockIdx.x * kGvWarps + (threadIdx.x >> 5)) * kGvRows;
  if (n0 >= rows_total) return;
  const int t = tile_task[n0 >> 7];
  if (task_active != nullptr && task_active[t] == 0) return;
  const float* Vt = V + (int64_t)t * R * Dp;
  float acc[kGvRows][NR];
#pragma unroll
  for (int i = 0; i < kGvRows; ++i)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[i][j] = 0.f;
  for (int d = lane * 4; d < Dp; d += 128) {
    float4 v[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = __ldg(reinterpret_cast<const float4*>(Vt + (int64_t)j * Dp + d));
#pragma unroll
    for (int i = 0; i < kGvRows; ++i) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(phi + (n0 + i) * Dp + d));
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        acc[i][j] = fmaf(a.x, v[j].x, acc[i][j]);
        acc[i][j] = fmaf(a.y, v[j].y, acc[i][j]);
        acc[i][j] = fmaf(a.z, v[j].z, acc[i][j]);
        acc[i][j] = fmaf(a.w, v[j].w, acc[i][j]);
      }
    }
  }
  // fixed-order butterfly over the lanes: every lane ends with the full sums
#pragma unroll
  for (int i = 0; i < kGvRows; ++i)
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], m);
  const int64_t rbeg = drow[t], Np = drow[t + 1] - rbeg;
  float* Wt = W + rbeg * R;
  if (lane < kGvRows) {
#pragma unroll
    for (int i = 0; i < kGvRows; ++i)
      if (i == lane)
#pragma unroll
        for (int j = 0; j < NR; ++j) Wt[(int64_t)j * Np + (n0 - rbeg) + i] = acc[i][j];
  }
}

template <int NR>
__global__ void __launch_bounds__(128) k_gemv2(P2Args p) {
  __shared__ float Ws[NR][kGvChunk];
  const int t = blockIdx.y;
  if (p.task_active != nullptr && p.task_active[t] == 0) return;
  const int d = blockIdx.x * 512 + threadIdx.x * 4;
  const bool on = d < p.Dp;          // warp-uniform: D_pad is a multiple of 128
  if (p.opcount != nullptr && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&p.opcount[t], 1ull);
  const int64_t rbeg = p.drow[t], Np = p.drow[t + 1] - rbeg;
  const float* Wt = p.W + rbeg * p.R;
  float4 acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t c0 = 0; c0 < Np; c0 += kGvChunk) {
    const int nc = (int)(Np - c0 < kGvChunk ? Np - c0 : kGvChunk);
    __syncthreads();
    for (int i = threadIdx.x; i < NR * nc; i += 128) {
      const int j = i / nc, n = i - j * nc;
      Ws[j][n] = Wt[(int64_t)j * Np + c0 + n];
    }
    __syncthreads();
    const float* prow = p.phi + (rbeg + c0) * p.Dp + d;
    for (int n = 0; on && n < nc; ++n) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(prow + (int64_t)n * p.Dp));
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const float w = Ws[j][n];
        acc[j].x = fmaf(a.x, w, acc[j].x);
        acc[j].y = fmaf(a.y, w, acc[j].y);
        acc[j].z = fmaf(a.z, w, acc[j].z);
        acc[j].w = fmaf(a.w, w, acc[j].w);
      }
    }
  }
  const int lane = threadIdx.x & 31;
  if (!on) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    if (j >= p.R) break;
    const int64_t sys = (int64_t)t * p.R + j;
    const int c = j / (p.K + 1);
    const float4 v = *reinterpret_cast<const float4*>(p.V + sys * p.Dp + d);
    const float4 al = *reinterpret_cast<const float4*>(p.alpha + (int64_t)c * p.Dp + d);
    float4 z;
    z.x = fmaf(p.beta_f, acc[j].x, al.x * v.x);
    z.y = fmaf(p.beta_f, acc[j].y, al.y * v.y);
    z.z = fmaf(p.beta_f, acc[j].z, al.z * v.z);
    z.w = fmaf(p.beta_f, acc[j].w, al.w * v.w);
    *reinterpret_cast<float4*>(p.Z + sys * p.Dp + d) = z;
    if (p.part != nullptr) {
      float dot = fmaf(v.x, z.x, fmaf(v.y, z.y, fmaf(v.z, z.z, v.w * z.w)));
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, m);
      if (lane == 0) p.part[(int64_t)(d >> 7) * p.S + sys] = dot;
    }
  }
}

// --------------------------------------------------------------------------------------
// host launchers
// --------------------------------------------------------------------------------------
namespace {

// tile width TN (columns per thread) from the supported set minimising padded R, then
// preferring wider tiles (fewer re-reads of Phi)
}  // namespace

int pick_tn(int R, int max_tn) {
  static const int cands[] = {9, 8, 6, 4, 3, 2, 1};
  int best = 1;
  int64_t best_pad = INT64_MAX;
  for (int tn : cands) {
    if (tn > max_tn) continue;
    const int bn = 16 * tn;
    const int64_t pad = (int64_t)((R + bn - 1) / bn) * bn;
    if (pad < best_pad) {
      best_pad = pad;
      best = tn;
    }
  }
  return best;
}

namespace {

// one CTA per tile (the kernels also accept fewer CTAs, looping over the tiles)
template <bool DS>
cudaError_t pass1(Ctx* c, int tn, const float* V, float* W, float* Wlo, const int* mask, int Rc,
                  int jstride, int g0 = 0, int ng = -1, const int* ractive = nullptr) {
  const int bn = 16 * tn;
  if (ng < 0) ng = (int)(c->rows_total / 128);
  const int ntiles = ((Rc + bn - 1) / bn) * ng;
  if (ntiles <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)ntiles;
  cudaStream_t st = c->stream;
#define P1CASE(TN)                                                                          \
  case TN:                                                                                  \
    k_pass1<TN, DS><<<grid, 256, 0, st>>>(c->phi, V, W, Wlo, c->drow, c->tile_task, mask,  \
                                          ractive, c->R, c->Dp, Rc, jstride, g0, ntiles);   \
    break;
  switch (tn) {
    P1CASE(1) P1CASE(2) P1CASE(3) P1CASE(4) P1CASE(6) P1CASE(8) P1CASE(9)
    default: return cudaErrorInvalidValue;
  }
#undef P1CASE
  return cudaGetLastError();
}

template <bool DS>
cudaError_t pass2(Ctx* c, int tn, const P2Args& a0, int nt = -1) {
  const int bn = 16 * tn;
  P2Args a = a0;
  a.ntiles = ((a.Rc + bn - 1) / bn) * (c->Dp / 128) * (nt < 0 ? c->T - a.t0 : nt);
  if (a.ntiles <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)a.ntiles;
  cudaStream_t st = c->stream;
#define P2CASE(TN)                                          \
  case TN:                                                  \
    k_pass2<TN, DS><<<grid, 256, 0, st>>>(a);               \
    break;
  switch (tn) {
    P2CASE(1) P2CASE(2) P2CASE(3) P2CASE(4) P2CASE(6) P2CASE(8) P2CASE(9)
    default: return cudaErrorInvalidValue;
  }
#undef P2CASE
  return cudaGetLastError();
}

// the two GEMV passes for R <= kGemvMaxR (every task in one launch per pass)
cudaError_t gemv_operator(Ctx* c, const P2Args& a, const float* V, const int* mask) {
  const int64_t nwarps = c->rows_total / kGvRows;
  const unsigned g1 = (unsigned)((nwarps + kGvWarps - 1) / kGvWarps);
  const dim3 g2((unsigned)((c->Dp + 511) / 512), (unsigned)c->T);
  cudaStream_t st = c->stream;
#define GVCASE(NR)                                                                              \
  case NR:                                                                                      \
    k_gemv1<NR><<<g1, 32 * kGvWarps, 0, st>>>(c->phi, V, c->w, c->drow, c->tile_task, mask, c->R, \
                                             c->Dp, c->rows_total);                              \
    k_gemv2<NR><<<g2, 128, 0, st>>>(a);                                                         \
    break;
  switch (c->R) {
    GVCASE(1) GVCASE(2) GVCASE(3) GVCASE(4) GVCASE(5) GVCASE(6) GVCASE(7) GVCASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef GVCASE
  c->launches += 2;
  return cudaGetLastError();
}

P2Args base_args(Ctx* c) {
  P2Args a{};
  a.phi = c->phi;
  a.W = c->w;
  a.Wlo = c->wlo;
  a.alpha = c->alpha;
  a.b0hi = c->b0hi;
  a.b0lo = c->b0lo;
  a.drow = c->drow;
  a.R = c->R;
  a.K = c->K;
  a.C = c->C;
  a.Dp = c->Dp;
  a.D = c->D;
  a.S = c->S;
  a.beta_f = (float)c->beta;
  a.beta_d = c->beta;
  a.seed = c->seed;
  a.em_iter = c->em_iter;
  a.toff = c->toff;
  a.pw = c->precond ? c->pw : nullptr;
  a.pshare = c->pshare;
  a.Rc = c->R;
  a.jstride = 1;
  a.t0 = 0;
  return a;
}

}  // namespace

cudaError_t launch_operator(Ctx* c, const float* V, float* Z, int with_dots) {
  if (c->op == 1) return launch_dft_apply(c, V, Z, with_dots);
  if (c->tc != nullptr) return tc_operator(c, V, Z, with_dots);
  const int* mask = with_dots ? c->task_active : nullptr;
  const int tn = c->tn_plain > 0 ? c->tn_plain : pick_tn(c->R, 9);
  P2Args a = base_args(c);
  a.V = V;
  a.Z = Z;
  a.part = with_dots ? c->part : nullptr;
  a.task_active = mask;
  a.opcount = c->prof_on ? reinterpret_cast<unsigned long long*>(c->opcount) : nullptr;
  if (c->per_task) {
    // comparison schedule: one pair of launches per task
    for (int t = 0; t < c->T; ++t) {
      cudaError_t e = pass1<false>(c, tn, V, c->w, nullptr, mask, c->R, 1,
                                   (int)(c->hrow[t] / 128), (int)((c->hrow[t + 1] - c->hrow[t]) / 128));
      if (e != cudaSuccess) return e;
      a.t0 = t;
      e = pass2<false>(c, tn, a, 1);
      if (e != cudaSuccess) return e;
      c->launches += 2;
    }
    return cudaSuccess;
  }
  static int gemv = -1;                // evaluation switch CMCS_GEMV=0: the GEMM tiles at any R
  if (gemv < 0) {
    const char* v = getenv("CMCS_GEMV");
    gemv = v ? atoi(v) != 0 : 1;
  }
  if (gemv && c->R <= kGemvMaxR) return gemv_operator(c, a, V, mask);
  cudaError_t e = pass1<false>(c, tn, V, c->w, nullptr, mask, c->R, 1);
  if (e != cudaSuccess) return e;
  c->launches += 2;
  return pass2<false>(c, tn, a);
}

cudaError_t launch_phi_v(Ctx* c, const float* V, float* W, float* Wlo, int Rc, int jstride) {
  c->launches += 1;
  if (Wlo != nullptr) return pass1<true>(c, pick_tn(Rc, 4), V, W, Wlo, nullptr, Rc, jstride);
  return pass1<false>(c, pick_tn(Rc, 9), V, W, nullptr, nullptr, Rc, jstride);
}

cudaError_t launch_residual(Ctx* c, const float* X, const float* Bext, float* Rout,
                            int all_systems, int means_only) {
  if (c->op == 1) return launch_dft_residual(c, X, Bext, Rout, all_systems, means_only);
  const int Rc = means_only ? c->C : c->R;
  const int js = means_only ? c->K + 1 : 1;
  // the residual of the means feeds ell's data term mu^T (b0 - A mu), where the tensor-core
  // residual's rounding of W (beta Phi^T dW, harmless to refinement) would shift the value by
  // beta (Phi mu)^T dW: it stays on the double-single kernels
  if (c->oz != nullptr && !means_only) return oz_residual(c, X, Bext, Rout, Rc, js);
  const int tn = c->tn_ds > 0 ? c->tn_ds : pick_tn(Rc, 4);
  // systems no longer refining: their tiles are skipped, their residual entries not read
  const int* ractive = (Bext || all_systems) ? nullptr : c->ractive;
  cudaError_t e = pass1<true>(c, tn, X, c->w, c->wlo, nullptr, Rc, js, 0, -1, ractive);
  if (e != cudaSuccess) return e;
  P2Args a = base_args(c);
  a.Rc = Rc;
  a.jstride = js;
  a.V = X;
  a.Z = Rout;
  a.Bext = Bext;
  a.ractive = ractive;
  c->launches += 2;
  return pass2<true>(c, tn, a);
}

}  // namespace cmcs
