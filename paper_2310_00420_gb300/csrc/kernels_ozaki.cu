// Refinement residual r = B - A X (A = beta Phi^T Phi + diag(alpha_c), Eq. 7) on the tensor
// cores, by error-free splitting of the operands into BF16 digit planes (Ozaki, Ogita, Oishi and
// Rump, "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012)).
//
// Each operand is written as a scale (a power of two) times a short sum of digit planes whose
// entries are integers of at most 8 bits times a fixed power of two:
//   Phi[n][d] = u_td 2^-7 sum_{k<5} q_k[n][d],  q_k = e_k 2^-8k,  e_k integer in [-128, 128],
// with u_td the smallest power of two >= max_n |Phi_t[n][d]| (column d of task t), so every FP32
// entry of Phi within 2^-15 of its column's largest is represented exactly, and the vector
// operand likewise with one scale per system over the contraction index: x' = u_t * x in pass 1
// with four planes (32 bits below the system's largest |x'|), W in pass 2 with three (24 bits).
// The product of two digit planes (k, l) is an integer multiple of 2^-8(k+l), each product of
// digits has at most 14 bits, so the FP32 sum of up to 1024 of them in tensor memory is exact.
// The pairs with k + l <= 4 are formed (the rest lie below 2^-32 of the leading pair): per tile
// Phi plane k is multiplied by the first nl(k) stacked vector planes in one MMA of N = 32 nl(k)
// columns into its own TMEM accumulator; after every `chunk` k-blocks the epilogue warps add the
// exact sums into a double-single accumulator per output (Knuth's TwoSum) and the MMA issuer
// starts the next chunk from zero.
//
// Pass 1: W[j][n] = sum_d Phi[n][d] x[j][d]      A = the three leading Phi digit planes, K-major
//                                               (blocked layout)
// Pass 2: R[j][d] = B - alpha x - beta sum_n Phi[n][d] W[j][n]
//                                               A = all five planes read MN-major
// W carries rounding of FP32 size: its digits keep 24 bits below each system's largest |W|, and
// pass 1 takes Phi to 23 bits below its column's largest entry.  Such an error in Phi x reaches
// the solution of A delta = r only through beta Phi^T (amplified by about the condition of Phi_t,
// not of A_tc); Phi^T W itself, whose rounding A^-1 amplifies by kappa(A_tc), is formed without
// rounding from all five planes.  The final combine b - alpha x - beta z runs in
// double-single arithmetic (TwoProduct by FMA, TwoSum), the output is rounded to FP32 once.
//
// Persistent kernels, one CTA (10 warps) per SM: warp 0 lane 0 streams the tiles with TMA
// (128-byte swizzle) through three (pass 1) or two (pass 2) shared-memory stages, warp 1 lane 0
// issues tcgen05.mma, warps 2-9 drain TMEM (two per 32-lane quarter, 16 systems each).  Every
// wait is bounded; on expiry the kernel records status bit 8, stops issuing, waits (bounded)
// for its copies in flight and still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <new>

#include "cmcs_internal.cuh"
#include "tc_ptx.cuh"

namespace cmcs {

using namespace tcx;

namespace {

constexpr int kOzK = 5;                          // digit planes of Phi
constexpr int kOzL1 = 4;                         // digit planes of x' (pass 1)
constexpr int kOzL2 = 3;                         // digit planes of W (pass 2)
constexpr int kOzJT = 32;                        // systems per tile
constexpr int kOzTmem = 512;                     // TMEM columns allocated (352 or 384 used)
constexpr int kOzEpiWarps = 8;
constexpr int kOzThreads = 64 + 32 * kOzEpiWarps;
// pass 1 forms W, whose errors the refinement sees only through beta Phi^T (see above), from
// the three leading Phi planes in three 64 KiB stages; pass 2 uses all five in two of 92 KiB
__host__ __device__ constexpr int oz_nk(int pass) { return pass == 1 ? 3 : kOzK; }
__host__ __device__ constexpr int oz_stages(int pass) { return pass == 1 ? 3 : 2; }
constexpr int kOzABytes = kTileM * kTileK * 2;   // 16 KiB per Phi plane
constexpr int kOzBBytes = kOzJT * kTileK * 2;    // 4 KiB per vector plane
__host__ __device__ constexpr int oz_nl_max(int pass) { return pass == 1 ? kOzL1 : kOzL2; }
__host__ __device__ constexpr int oz_stage_bytes(int pass) {
  return oz_nk(pass) * kOzABytes + oz_nl_max(pass) * kOzBBytes;
}
// vector planes multiplied by Phi plane k (pairs k + l <= 4) and its accumulator's first column
__host__ __device__ constexpr int oz_nl(int pass, int k) {
  return oz_nl_max(pass) < 5 - k ? oz_nl_max(pass) : 5 - k;
}
__host__ __device__ constexpr int oz_col(int pass, int k) {
  return k == 0 ? 0 : oz_col(pass, k - 1) + kOzJT * oz_nl(pass, k - 1);
}
static_assert(oz_col(1, oz_nk(1)) <= kOzTmem && oz_col(2, oz_nk(2)) <= kOzTmem, "TMEM columns");
constexpr int kOzSmem1 = oz_stages(1) * oz_stage_bytes(1) + 1024 + 128;
constexpr int kOzSmem2 = oz_stages(2) * oz_stage_bytes(2) + 1024 + 128;
static_assert(kOzSmem1 <= 227 * 1024 && kOzSmem2 <= 227 * 1024, "shared memory per CTA");
constexpr int kOzMaxChunk = 16;                  // k-blocks per exact chunk: 16 x 64 x 2^14 = 2^24

struct OzMaps {
  CUtensorMap a[kOzK];
  CUtensorMap b[kOzL1];        // pass 2 uses the first kOzL2
};

struct OzArgs {
  const int* tile_task;       // [rows / 128]
  const int64_t* drow;        // [T + 1] padded row offsets
  int R, K, C, Dp, D, S;
  int Rc, jstride;            // columns j' < Rc of a task: systems j = j' jstride (all R systems,
                              // or the C means); digits, W and scales are indexed compactly
  int64_t rows_total;
  int njt;                    // system tiles per task (of Rc columns)
  int ntiles;
  int chunk;                  // k-blocks summed exactly in TMEM before a drain
  const float* xs;            // pass 1: [S] scale of x' = u_t x
  float* wf;                  // pass 1 output: W [R][rows_total]
  unsigned int* wmax;         // pass 1: [S] bits of max_n |W|
  const float* u;             // [T][Dp] column scales of Phi
  const float* X;             // pass 2: [S][Dp] the solutions
  const float* Bext;          // pass 2: [S][Dp] right-hand sides, or null (b0 and the probes)
  float* Rout;                // pass 2: [S][Dp]
  const float* alpha;         // [C][Dp]
  const float *b0hi, *b0lo;   // [T][Dp]
  float beta_hi, beta_lo;     // beta as an unevaluated FP32 pair
  uint64_t seed;
  int64_t em_iter;
  int toff;
  const float* pw;            // [T*C][Dp] or null (probe scaling of the preconditioned form)
  int pshare;
  int* status;
};

// scale of the digits: the smallest power of two >= m (1 for m = 0), as its exponent
__device__ __forceinline__ int scale_exp(float m) {
  int e = 0;
  frexpf(m, &e);                 // m = f 2^e, f in [0.5, 1)
  return m > 0.f ? e : 0;
}

// digits of a with |a| <= 2^e: a = 2^e 2^-7 sum_{i<n} e_i 2^-8i, written as BF16 values
// e_i 2^-8i (exact: |e_i| <= 128); the remainder after n digits is dropped
template <int NDIG>
__device__ __forceinline__ void make_digits(float a, int e, __nv_bfloat16* out, int64_t stride) {
  float y = ldexpf(a, 7 - e);    // |y| <= 128, exact
  float sc = 1.f;
#pragma unroll
  for (int i = 0; i < NDIG; ++i) {
    const float di = rintf(y);
    out[i * stride] = __float2bfloat16_rn(di * sc);
    y = (y - di) * 256.f;        // exact: the fraction of y, scaled by a power of two
    sc *= 0.00390625f;           // 2^-8
  }
}

// ---- set-up: column scales and digit planes of Phi -----------------------------------------
__global__ void k_oz_colscale(const float* __restrict__ phi, const int64_t* __restrict__ drow,
                              float* __restrict__ u, int Dp) {
  const int t = blockIdx.y;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= Dp) return;
  float m = 0.f;
  for (int64_t n = drow[t]; n < drow[t + 1]; ++n) m = fmaxf(m, fabsf(phi[n * Dp + d]));
  u[(int64_t)t * Dp + d] = ldexpf(1.f, scale_exp(m));
}

// plane k of element (n, d) at k * plane + ((n / 128) (Dp / 64) + d / 64) 8192 + (n % 128) 64 + d % 64
__global__ void k_oz_phi_digits(const float* __restrict__ phi, const float* __restrict__ u,
                                const int* __restrict__ tile_task, __nv_bfloat16* __restrict__ dig,
                                int64_t rows, int Dp) {
  const int64_t n_el = rows * Dp, plane = rows * Dp;
  const int nkb = Dp / 64;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_el;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i / Dp;
    const int d = (int)(i - n * Dp);
    const int t = tile_task[n >> 7];
    const int e = ilogbf(u[(int64_t)t * Dp + d]);
    const int64_t o = ((n >> 7) * nkb + (d >> 6)) * 8192 + (n & 127) * 64 + (d & 63);
    make_digits<kOzK>(phi[i], e, dig + o, plane);
  }
}

// ---- per residual: digits of x' = u_t x (one CTA per system) and of W ----------------------
__global__ void __launch_bounds__(256) k_oz_x_digits(const float* __restrict__ X,
                                                     const float* __restrict__ u,
                                                     __nv_bfloat16* __restrict__ dig,
                                                     float* __restrict__ xs, int R, int Rc,
                                                     int jstride, int Dp, int64_t plane) {
  __shared__ float red[8];
  const int64_t sys = blockIdx.x;                    // compact index t Rc + j'
  const int t = (int)(sys / Rc);
  const float* x = X + ((int64_t)t * R + (sys - (int64_t)t * Rc) * jstride) * Dp;
  const float* ut = u + (int64_t)t * Dp;
  float m = 0.f;
  for (int d = threadIdx.x; d < Dp; d += blockDim.x) m = fmaxf(m, fabsf(ut[d] * x[d]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
  const int e = scale_exp(m);
  if (threadIdx.x == 0) xs[sys] = ldexpf(1.f, e);
  for (int d = threadIdx.x; d < Dp; d += blockDim.x)
    make_digits<kOzL1>(ut[d] * x[d], e, dig + sys * Dp + d, plane);
}

__global__ void k_oz_w_digits(const float* __restrict__ wf, const unsigned int* __restrict__ wmax,
                              const int* __restrict__ tile_task, __nv_bfloat16* __restrict__ dig,
                              int Rc, int64_t rows, int64_t plane) {
  const int64_t n_el = (int64_t)Rc * rows;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_el;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / rows, n = i - j * rows;
    const int t = tile_task[n >> 7];
    const int e = scale_exp(__uint_as_float(wmax[(int64_t)t * Rc + j]));
    make_digits<kOzL2>(wf[i], e, dig + i, plane);
  }
}

// ---- the digit-plane GEMM ------------------------------------------------------------------
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bv = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ bool oz_epi_any(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(32 * kOzEpiWarps)
      : "memory");
  return r != 0;
}

struct OzTile {
  int t, a_row, j0, kx, nk;
};

// tile = A tile * njt + system tile: the system tiles of one A tile run on neighbouring CTAs at
// the same time, so the later reads of the A tile come from L2
template <int PASS>
__device__ __forceinline__ OzTile oz_tile(const OzArgs& p, int tile) {
  OzTile ti;
  const int at = tile / p.njt;
  ti.j0 = (tile - at * p.njt) * kOzJT;
  if (PASS == 1) {
    ti.t = p.tile_task[at];
    ti.a_row = at * kTileM;
    ti.kx = 0;
    ti.nk = p.Dp / kTileK;
  } else {
    const int ndt = p.Dp / kTileM;
    ti.t = at / ndt;
    ti.a_row = (at - ti.t * ndt) * kTileM;
    ti.kx = (int)p.drow[ti.t];
    ti.nk = (int)((p.drow[ti.t + 1] - p.drow[ti.t]) / kTileK);
  }
  return ti;
}

template <int PASS>
__global__ void __launch_bounds__(kOzThreads, 1)
k_oz(const __grid_constant__ OzMaps maps, const OzArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  constexpr int kStage = oz_stage_bytes(PASS);
  constexpr int NL = oz_nl_max(PASS);
  constexpr int NK = oz_nk(PASS);
  constexpr int kOzStages = oz_stages(PASS);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kOzStages * kStage);
  uint64_t* empty = full + kOzStages;
  uint64_t* tfull = empty + kOzStages;        // a chunk's sums are ready for the epilogue
  uint64_t* tempty = tfull + 1;               // the epilogue has read them
  uint64_t* mdone = tempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (*reinterpret_cast<volatile int*>(p.status) & 8) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 32 * kOzEpiWarps);
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, kOzTmem);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t issued = 0;

  if (warp == 0) {
    // ---- TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      bool stop = false;
      for (int tile = blockIdx.x; tile < p.ntiles && !stop && !*abort_flag; tile += gridDim.x) {
        const OzTile ti = oz_tile<PASS>(p, tile);
        const int brow = PASS == 1 ? ti.t * p.Rc + ti.j0 : ti.j0;
        for (int kb = 0; kb < ti.nk; ++kb, ++it) {
          const int s = (int)(it % kOzStages);
          if (it >= (uint32_t)kOzStages && !mbar_wait(&empty[s], ((it / kOzStages) - 1) & 1)) {
            *abort_flag = 1;
            atomicOr(p.status, 8);
            stop = true;
            break;
          }
          if (*abort_flag) {
            stop = true;
            break;
          }
          uint8_t* st = smem + (size_t)s * kStage;
          mbar_expect_tx(&full[s], (uint32_t)kStage);
          const int kcol = ti.kx + kb * kTileK;
#pragma unroll
          for (int k = 0; k < NK; ++k) {
            uint8_t* ad = st + k * kOzABytes;
            if (PASS == 1) {
              tma_load_4d(ad, &maps.a[k], 0, 0, kcol / kTileK, ti.a_row / kTileM, &full[s]);
            } else {
              // rows n = kcol .. kcol + 63 of the 128-row block, columns d = a_row .. a_row + 127
              tma_load_4d(ad, &maps.a[k], 0, kcol & (kTileM - 1), ti.a_row / kTileK, kcol / kTileM,
                          &full[s]);
              tma_load_4d(ad + kOzABytes / 2, &maps.a[k], 0, kcol & (kTileM - 1), ti.a_row / kTileK + 1,
                          kcol / kTileM, &full[s]);
            }
          }
          uint8_t* bst = st + NK * kOzABytes;
#pragma unroll
          for (int l = 0; l < NL; ++l) tma_load_2d(bst + l * kOzBBytes, &maps.b[l], kcol, brow, &full[s]);
          issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t amaj = PASS == 2 ? (1u << 15) : 0u;      // A MN-major in pass 2
      uint32_t it = 0, q = 0;
      bool stop = false;
      for (int tile = blockIdx.x; tile < p.ntiles && !stop && !*abort_flag; tile += gridDim.x) {
        const OzTile ti = oz_tile<PASS>(p, tile);
        for (int kb = 0; kb < ti.nk; ++kb, ++it) {
          const bool cstart = (kb % p.chunk) == 0;
          if (cstart) {
            // the epilogue has read the previous chunk's sums
            if (q > 0 && !mbar_wait(tempty, (q - 1) & 1)) {
              *abort_flag = 1;
              atomicOr(p.status, 8);
              stop = true;
              break;
            }
            tc_fence_after();
          }
          const int s = (int)(it % kOzStages);
          if (!mbar_wait(&full[s], (it / kOzStages) & 1)) {
            *abort_flag = 1;
            atomicOr(p.status, 8);
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + (size_t)s * kStage);
#pragma unroll
          for (int kk = 0; kk < kTileK / 16; ++kk) {
            const uint64_t bd = smem_desc(st + NK * kOzABytes + kk * 32);
#pragma unroll
            for (int k = 0; k < NK; ++k) {
              const uint64_t ad = PASS == 1 ? smem_desc(st + k * kOzABytes + kk * 32)
                                            : smem_desc_mn(st + k * kOzABytes + kk * 2048, 8192, 1024);
              mma_bf16(tmem + (uint32_t)oz_col(PASS, k), ad, bd,
                       idesc_bf16(kTileM, kOzJT * oz_nl(PASS, k)) | amaj, (cstart && kk == 0) ? 0u : 1u);
            }
          }
          mma_commit(&empty[s]);
          if ((kb % p.chunk) == p.chunk - 1 || kb == ti.nk - 1) {
            mma_commit(tfull);
            ++q;
          }
        }
      }
      mma_commit(mdone);
      if (!mbar_wait(mdone, 0)) atomicOr(p.status, 8);
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, systems 16 jh .. + 15
    const int lg = warp & 3;
    const int jh = (warp - 2) >> 2;
    uint32_t q = 0;
    bool bad = false;
    for (int tile = blockIdx.x; tile < p.ntiles && !bad; tile += gridDim.x) {
      const OzTile ti = oz_tile<PASS>(p, tile);
      float hi[16], lo[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) hi[i] = lo[i] = 0.f;
      const int nch = (ti.nk + p.chunk - 1) / p.chunk;
      const uint32_t trow = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(16 * jh);
      for (int ch = 0; ch < nch; ++ch, ++q) {
        const bool ok = mbar_wait(tfull, q & 1);
        if (!ok) {
          *abort_flag = 1;
          if (lane == 0) atomicOr(p.status, 8);
        }
        if (oz_epi_any(!ok || *abort_flag)) {
          bad = true;
          break;
        }
        tc_fence_after();
        // the exact sums of the pairs (k, l), most significant Phi planes first
#pragma unroll
        for (int k = 0; k < NK; ++k) {
#pragma unroll
          for (int l = 0; l < oz_nl(PASS, k); ++l) {
            float v[16];
            tmem_ld16(trow + (uint32_t)(oz_col(PASS, k) + l * kOzJT), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) two_sum_acc(hi[i], lo[i], v[i]);
          }
        }
        tc_fence_before();
        mbar_arrive(tempty);
      }
      if (bad) break;
      if (PASS == 1) {
        const int64_t n = (int64_t)ti.a_row + 32 * lg + lane;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = ti.j0 + 16 * jh + i;
          if (j >= p.Rc) break;                     // uniform across the warp
          const int64_t sys = (int64_t)ti.t * p.Rc + j;  // compact
          // W = 2^-14 s (hi + lo): s and 2^-14 are powers of two
          const float w = __fadd_rn(hi[i], lo[i]) * (p.xs[sys] * 6.103515625e-05f);
          p.wf[(int64_t)j * p.rows_total + n] = w;
          float m = fabsf(w);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
          if (lane == 0) atomicMax(p.wmax + sys, __float_as_uint(m));
        }
      } else {
        const int d = ti.a_row + 32 * lg + lane;
        const float ud = p.u[(int64_t)ti.t * p.Dp + d];
        // probe bits of the 16 systems for this warp's 32 coordinates: lane i draws system i's
        uint32_t mybits = 0;
        {
          const int j = (ti.j0 + 16 * jh + (lane & 15)) * p.jstride;
          if (p.Bext == nullptr && j < p.R) {
            const int c = j / (p.K + 1), k = j - c * (p.K + 1);
            if (k > 0)
              mybits = probe_bits32(p.seed, p.em_iter, ti.t + p.toff, probe_cluster(c, p.pshare), p.C,
                                    k - 1, d & ~31);
          }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int jc = ti.j0 + 16 * jh + i;        // compact column
          const uint32_t bits = __shfl_sync(0xffffffffu, mybits, i);
          if (jc >= p.Rc) break;                    // uniform across the warp
          const int j = jc * p.jstride;
          const int64_t sys = (int64_t)ti.t * p.R + j;
          const int c = j / (p.K + 1), k = j - c * (p.K + 1);
          // z = Phi^T W = 2^-14 u_d v_j (hi + lo), exact scaling by powers of two
          const float sc = ud * ldexpf(6.103515625e-05f,
                                       scale_exp(__uint_as_float(p.wmax[(int64_t)ti.t * p.Rc + jc])));
          const float zh = hi[i] * sc, zl = lo[i] * sc;
          float bh = 0.f, bl = 0.f;
          if (p.Bext != nullptr) {
            bh = p.Bext[sys * p.Dp + d];
          } else if (d < p.D) {
            if (k == 0) {
              bh = p.b0hi[(int64_t)ti.t * p.Dp + d];
              bl = p.b0lo[(int64_t)ti.t * p.Dp + d];
            } else {
              bh = ((bits >> (d & 31)) & 1u) ? -1.f : 1.f;
              if (p.pw != nullptr) bh *= p.pw[((int64_t)ti.t * p.C + c) * p.Dp + d];
            }
          }
          const float xv = p.X[sys * p.Dp + d];
          const float av = p.alpha[(int64_t)c * p.Dp + d];
          // alpha x = p1 + e1 and beta z ~ p2 + e2 (TwoProduct by FMA)
          const float p1 = __fmul_rn(av, xv);
          const float e1 = __fmaf_rn(av, xv, -p1);
          const float p2 = __fmul_rn(p.beta_hi, zh);
          const float e2 = __fmaf_rn(p.beta_hi, zh, -p2) + __fmaf_rn(p.beta_hi, zl, p.beta_lo * zh);
          // b - p1 - p2 by TwoSum, then the small parts
          float s1 = bh, t1 = 0.f;
          two_sum_acc(s1, t1, -p1);
          two_sum_acc(s1, t1, -p2);
          const float r = s1 + (((t1 + bl) - e1) - e2);
          p.Rout[sys * p.Dp + d] = r;
        }
      }
    }
  }

  // ---- teardown: no copy may still be landing in shared memory when the CTA exits
  __syncwarp();
  if (*abort_flag && warp == 0 && lane == 0) {
    for (uint32_t k = issued; k > 0 && k + kOzStages > issued; --k)
      mbar_wait(&full[(k - 1) % kOzStages], ((k - 1) / kOzStages) & 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kOzTmem);
}

struct OzState {
  __nv_bfloat16* phid;        // [5][rows][Dp] digit planes of Phi, blocked
  float* u;                   // [T][Dp]
  __nv_bfloat16* xd;          // [4][S][Dp]
  float* xs;                  // [S]
  float* wf;                  // [R][rows]
  unsigned int* wmax;         // [S]
  __nv_bfloat16* wd;          // [3][R][rows]
  OzMaps m1, m2;              // pass 1 and pass 2 tensor maps
  int chunk;
};

}  // namespace

int oz_create(Ctx* c) {
  OzState* s = new (std::nothrow) OzState();
  if (!s) return 1;
  c->oz = s;
  const int64_t rows = c->rows_total, Dp = c->Dp, S = c->S, R = c->R;
  {
    const char* cv = getenv("CMCS_OZ_CHUNK");    // evaluation switch: k-blocks per exact chunk
    s->chunk = cv ? atoi(cv) : 16;
    if (s->chunk < 1 || s->chunk > kOzMaxChunk) s->chunk = 16;
  }
  auto al = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
  bool ok = al(reinterpret_cast<void**>(&s->phid), sizeof(__nv_bfloat16) * (size_t)(kOzK * rows * Dp)) &&
            al(reinterpret_cast<void**>(&s->u), sizeof(float) * (size_t)(c->T * Dp)) &&
            al(reinterpret_cast<void**>(&s->xd), sizeof(__nv_bfloat16) * (size_t)(kOzL1 * S * Dp)) &&
            al(reinterpret_cast<void**>(&s->xs), sizeof(float) * (size_t)S) &&
            al(reinterpret_cast<void**>(&s->wf), sizeof(float) * (size_t)(R * rows)) &&
            al(reinterpret_cast<void**>(&s->wmax), sizeof(unsigned int) * (size_t)S) &&
            al(reinterpret_cast<void**>(&s->wd), sizeof(__nv_bfloat16) * (size_t)(kOzL2 * R * rows));
  if (!ok) {
    snprintf(c->err, sizeof(c->err), "tensor-core residual: device allocation failed");
    return 1;
  }
  for (int k = 0; k < kOzK && ok; ++k) {
    const __nv_bfloat16* base = s->phid + (size_t)k * rows * Dp;
    ok = encode_blocked(&s->m1.a[k], base, Dp, rows, kTileM) && encode_blocked(&s->m2.a[k], base, Dp, rows, 64);
  }
  for (int l = 0; l < kOzL1 && ok; ++l) ok = encode_2d(&s->m1.b[l], s->xd + (size_t)l * S * Dp, Dp, S, kOzJT);
  for (int l = 0; l < kOzL2 && ok; ++l) ok = encode_2d(&s->m2.b[l], s->wd + (size_t)l * R * rows, rows, R, kOzJT);
  if (!ok) {
    snprintf(c->err, sizeof(c->err), "tensor-core residual: tensor map encoding failed");
    return 1;
  }
  cudaError_t e = cudaFuncSetAttribute(k_oz<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem1);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_oz<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem2);
  if (e == cudaSuccess) e = oz_refresh(c);
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "tensor-core residual set-up: %s", cudaGetErrorString(e));
    return 1;
  }
  return 0;
}

cudaError_t oz_refresh(Ctx* c) {
  OzState* s = static_cast<OzState*>(c->oz);
  if (!s) return cudaSuccess;
  k_oz_colscale<<<dim3((unsigned)(c->Dp / 128), (unsigned)c->T), 128, 0, c->stream>>>(c->phi, c->drow, s->u,
                                                                                    c->Dp);
  k_oz_phi_digits<<<4096, 256, 0, c->stream>>>(c->phi, s->u, c->tile_task, s->phid, c->rows_total, c->Dp);
  c->launches += 2;
  return cudaGetLastError();
}

void oz_destroy(Ctx* c) {
  OzState* s = static_cast<OzState*>(c->oz);
  if (!s) return;
  void* ptrs[] = {s->phid, s->u, s->xd, s->xs, s->wf, s->wmax, s->wd};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete s;
  c->oz = nullptr;
}

cudaError_t oz_residual(Ctx* c, const float* X, const float* Bext, float* Rout, int Rc, int jstride) {
  OzState* s = static_cast<OzState*>(c->oz);
  if (!s) return cudaErrorNotSupported;
  const int64_t rows = c->rows_total;
  OzArgs a{};
  a.tile_task = c->tile_task;
  a.drow = c->drow;
  a.R = c->R;
  a.K = c->K;
  a.C = c->C;
  a.Dp = c->Dp;
  a.D = c->D;
  a.S = c->S;
  a.rows_total = rows;
  a.Rc = Rc;
  a.jstride = jstride;
  a.njt = (Rc + kOzJT - 1) / kOzJT;
  a.chunk = s->chunk;
  a.xs = s->xs;
  a.wf = s->wf;
  a.wmax = s->wmax;
  a.u = s->u;
  a.X = X;
  a.Bext = Bext;
  a.Rout = Rout;
  a.alpha = c->alpha;
  a.b0hi = c->b0hi;
  a.b0lo = c->b0lo;
  a.beta_hi = (float)c->beta;
  a.beta_lo = (float)(c->beta - (double)a.beta_hi);
  a.seed = c->seed;
  a.em_iter = c->em_iter;
  a.toff = c->toff;
  a.pw = c->precond ? c->pw : nullptr;
  a.pshare = c->pshare;
  a.status = &c->counters[2];
  const int sms = c->sm_count > 0 ? c->sm_count : 1;
  const int nsys = c->T * Rc;
  cudaError_t e = cudaMemsetAsync(s->wmax, 0, sizeof(unsigned int) * (size_t)nsys, c->stream);
  if (e != cudaSuccess) return e;
  k_oz_x_digits<<<(unsigned)nsys, 256, 0, c->stream>>>(X, s->u, s->xd, s->xs, c->R, Rc, jstride,
                                                       c->Dp, (int64_t)c->S * c->Dp);
  a.ntiles = (int)(rows / kTileM) * a.njt;
  k_oz<1><<<a.ntiles < sms ? a.ntiles : sms, kOzThreads, kOzSmem1, c->stream>>>(s->m1, a);
  k_oz_w_digits<<<4096, 256, 0, c->stream>>>(s->wf, s->wmax, c->tile_task, s->wd, Rc, rows,
                                             (int64_t)c->R * rows);
  a.ntiles = c->T * (c->Dp / kTileM) * a.njt;
  k_oz<2><<<a.ntiles < sms ? a.ntiles : sms, kOzThreads, kOzSmem2, c->stream>>>(s->m2, a);
  c->launches += 4;
  return cudaGetLastError();
}

}  // namespace cmcs
