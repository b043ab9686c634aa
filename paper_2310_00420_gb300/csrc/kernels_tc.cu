// Tensor-core operator for CMCS_BF16_REFINE and CMCS_BF16X3 (tcgen05 MMA, TMA, TMEM; sm_103a).
//
// Same two passes as the FP32 operator (Eq. 7 applied to all R = C*(K+1) right-hand sides of a
// task), BF16 GEMMs with FP32 accumulation in tensor memory:
//   pass 1: W[j][n] = sum_d Phi[n][d] V[j][d]       A = Phi [rows][D_pad] K-major, B = V [S][D_pad]
//   pass 2: Z[j][d] = beta sum_n Phi[n][d] W[j][n] (+ alpha_c[d] V[j][d])
//                                                   A = the same Phi planes read MN-major,
//                                                   B = W [R][rows]
// In a CG step pass 2 stores beta Phi^T W only and the CG update adds alpha_c d (and forms
// d^T A d); cmcs_apply gets the full A V.  FP32 operands enter as unevaluated BF16 pairs
// x = x_hi + x_lo.  BF16_REFINE multiplies the BF16-rounded Phi by (V_hi + V_lo) (two MMAs per
// k-step); BF16X3 also splits Phi and adds Phi_lo V_hi (three MMAs), about 16 significant bits
// per product.
//
// Persistent kernel, one CTA (6 warps) per SM, looping over output tiles of 128 rows by up to
// 256 columns (R wider than 256 is split into column tiles).  Warp 0 lane 0 streams A and B
// tiles with TMA (128-byte swizzle) through a ring of shared-memory stages; warp 1 lane 0
// issues tcgen05.mma from shared-memory descriptors into one of two TMEM accumulators; warps
// 2-5 drain the other accumulator (tcgen05.ld, 32 rows each), so a tile's epilogue overlaps
// the next tile's mainloop.  Pass 2 is launched programmatically: its CTAs start on the SMs
// pass 1 frees, take tiles from a global counter (the producer queues each tile index in
// shared memory for the MMA issuer and the epilogue) and wait per tile for their task's
// pass-1 tiles.  Every wait is bounded: on expiry the kernel records status bit 8, stops
// issuing, waits (bounded) for its copies and MMAs in flight and still frees its TMEM.
// Kept for comparison (CMCS_TC_MODE): pass 2 on a transposed copy of Phi (2) and both passes
// in one fused launch (0).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cmcs_internal.cuh"
#include "tc_ptx.cuh"

namespace cmcs {

using namespace tcx;

namespace {

constexpr int kBM = 128;                   // rows of an output tile (MMA M)
constexpr int kBK = 64;                    // K per stage: one 128-byte row of BF16
constexpr int kEpiWarps = 4;               // warps 2..5 drain TMEM
constexpr int kTcThreads = 64 + 32 * kEpiWarps;
constexpr int kTq = 4;                      // tile queue slots (dynamically scheduled pass 2)
constexpr int kTqBytes = 2 * kTq * 8 + kTq * 4 + 48;
constexpr uint64_t kWaitNs = 2000000000ull; // wall time before an mbarrier wait is declared stuck
constexpr int kSmemBudget = 225 * 1024;

struct TcArgs {
  const int* tile_task;
  const int64_t* drow;
  const int* task_active;
  int R, K, C, Dp, D, S;
  int64_t rows_total;
  int Rpad, BR, nbox, stages, stage_bytes;
  int ntiles, nbuf;
  int tile_lo;            // tiles tile_lo .. ntiles-1 (a single task's range when per task)
  int ncol;               // column tiles per row tile (Rpad columns each)
  uint32_t tmem_cols;     // columns of one accumulator buffer
  uint32_t tmem_alloc;    // columns allocated (nbuf buffers)
  __nv_bfloat16* w_hi;    // pass 1 output, [R][rows_total]
  __nv_bfloat16* w_lo;
  const float* V;         // pass 2 epilogue: the FP32 vectors A is applied to, [S][D_pad]
  float* Z;               // pass 2 output A V, [S][D_pad]
  float* part;            // [D_pad/128][S] partial v^T A v, or null
  const float* alpha;     // [C][D_pad]
  float beta;
  unsigned long long* opcount;
  int* status;
  const int* stall;       // test hook: nonzero makes the MMA warp wait on a barrier nothing arrives at
  uint32_t mn_lbo, mn_sbo; // MN-major A descriptor strides (pass 2 reading Phi directly)
  int raw;                 // pass 2 stores beta Phi^T W only (the CG update adds alpha * V and
                           // forms d^T A d itself); otherwise the full A V, with partials if part
  int early;               // pass 1 counts its finished tiles per task and lets pass 2 launch at
                           // once; pass 2 waits per tile on those counts instead of the grid
  const int* tile_code;    // fused launches: per tile (local << 2) | (pass - 1)
  const int* tile_task2;   // fused launches: task of each tile
  int* p1done;             // fused or early launches: finished pass-1 tiles per task (zeroed per
                           // application)
  int* tile_ctr;           // early pass 2: next tile to hand out (zeroed per launch)
  const int* n1;           // fused or early launches: pass-1 tiles per task
  // one-read schedule (PASS 4): work units in order, pass-1 units split along K
  const int* u_code;       // per unit: (g << 4) | (split << 1) for pass 1, (d-tile << 1) | 1 for pass 2
  const int* u_task;       // per unit: its task
  int splitk;              // K splits of a pass-1 row tile
  int nslot;               // row tiles whose partial sums can be held at once
  float* wpart;            // [nslot][splitk][Rpad][128] FP32 partial W of pass-1 units
  int* p1cnt;              // [row tiles] pass-1 units that reached their epilogue (zeroed per launch)
  int* p1st;               // [row tiles] pass-1 units whose partial is stored (zeroed per launch)
  int* wready;             // [row tiles] 1 once the row tile's W is reduced and stored
  int pf;                  // prefetch the Phi tile this many k-blocks ahead into L2 (0: off)
  int tiled;               // the Phi planes are stored blocked ([row tile][k-block][128][64]):
                           // every A tile of pass 1 is one contiguous 16 KiB and every
                           // MN-major box of pass 2 one contiguous 8 KiB (4-D tensor maps)
};

// all tensor maps of the operator: a[pass-1][hi/lo] (pass 2 reads Phi MN-major), b[pass-1][hi/lo]
struct TcMaps {
  CUtensorMap a[2][2];
  CUtensorMap b[2][2];
};

}  // namespace

// ---- the GEMM kernel (persistent, two TMEM accumulators) --------------------------------
struct TileInfo {
  int pass;                       // 1: W = Phi V;  2: Z = beta Phi^T W + alpha V
  int t, a_row, b_row, kx, nk, dtile, col0;
  int split;                      // PASS 4 pass-1 unit: which K split of row tile dtile
};

// Tile decoding.  Single-pass launches (PASS 1, 2 or 3; 3 is pass 2 reading Phi MN-major):
// tile = row_tile * ncol + column_tile, so the column tiles of one row tile run on
// neighbouring CTAs at the same time and the second read of the A tile is served by L2.
// Fused launches (PASS 0): tile_code[tile] = (local << 2) | (pass - 1) with tasks in order,
// each task's pass-1 tiles before its pass-2 tiles; task = tile_task2[tile].
// One-read launches (PASS 4): unit u of task u_task[u] is either the K split `split` of pass-1
// row tile g (global index; k-blocks [split nkb / splitk, (split + 1) nkb / splitk) of the
// nkb = D_pad / 64) or the whole pass-2 tile of d-tile `local`.
template <int PASS>
__device__ __forceinline__ bool tile_info(const TcArgs& p, int tile_in, TileInfo& ti) {
  if (PASS == 4) {
    const int code = p.u_code[tile_in];
    ti.t = p.u_task[tile_in];
    ti.col0 = 0;
    ti.split = 0;
    if ((code & 1) == 0) {
      const int g = code >> 4, sp = (code >> 1) & 7;
      const int nkb = p.Dp / kBK;
      const int kb0 = sp * nkb / p.splitk, kb1 = (sp + 1) * nkb / p.splitk;
      ti.pass = 1;
      ti.a_row = g * kBM;
      ti.b_row = ti.t * p.R;
      ti.kx = kb0 * kBK;
      ti.nk = kb1 - kb0;
      ti.dtile = g;
      ti.split = sp;
    } else {
      ti.pass = 2;
      ti.dtile = code >> 1;
      ti.a_row = ti.dtile * kBM;
      ti.b_row = 0;
      ti.kx = (int)p.drow[ti.t];
      ti.nk = (int)((p.drow[ti.t + 1] - p.drow[ti.t]) / kBK);
    }
    return p.task_active == nullptr || p.task_active[ti.t] != 0;
  }
  int pass = PASS == 1 ? 1 : 2, local = tile_in;
  if (PASS == 0) {
    const int code = p.tile_code[tile_in];
    pass = (code & 3) + 1;
    local = code >> 2;
  }
  ti.pass = pass;
  const int tile = local / p.ncol;
  ti.col0 = (local - tile * p.ncol) * p.Rpad;
  if (pass == 1) {
    // row tiles are numbered within the whole Phi (fused: within the task, offset below)
    const int g = PASS == 0 ? (int)(p.drow[p.tile_task2[tile_in]] / kBM) + tile : tile;
    ti.t = p.tile_task[g];
    ti.a_row = g * kBM;
    ti.b_row = ti.t * p.R;
    ti.kx = 0;
    ti.nk = p.Dp / kBK;
    ti.dtile = 0;
  } else {
    const int ndt = p.Dp / kBM;
    ti.t = PASS == 0 ? p.tile_task2[tile_in] : tile / ndt;
    ti.dtile = PASS == 0 ? tile : tile - ti.t * ndt;
    ti.a_row = ti.dtile * kBM;
    ti.b_row = 0;
    ti.kx = (int)p.drow[ti.t];
    ti.nk = (int)((p.drow[ti.t + 1] - p.drow[ti.t]) / kBK);
  }
  return p.task_active == nullptr || p.task_active[ti.t] != 0;
}

// release / acquire of the per-task count of finished pass-1 tiles (fused or early launches); W is
// written with generic stores and read by TMA (async proxy), hence the proxy fences
__device__ __forceinline__ void signal_pass1_done(int* cnt) {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __threadfence();
  atomicAdd(cnt, 1);
}
__device__ __forceinline__ bool wait_pass1_done(const int* cnt, int want) {
  const volatile int* v = cnt;
  if (*v < want) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; *v < want; ++i)
      if ((i & 255u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
  __threadfence();
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return true;
}

// bounded wait until *f becomes nonzero (a row tile of W published with the release pattern
// of signal_pass1_done); the fences order the later reads, TMA (async proxy) included
__device__ __forceinline__ bool wait_flag(const int* f) {
  const volatile int* v = f;
  if (*v == 0) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; *v == 0; ++i)
      if ((i & 255u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
  __threadfence();
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return true;
}

// bounded wait until *f >= want (peers that have already arrived finishing their stores)
__device__ __forceinline__ bool wait_count(const int* f, int want) {
  const volatile int* v = f;
  if (*v < want) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; *v < want; ++i)
      if ((i & 255u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
  __threadfence();
  return true;
}

// acc[0..15] = sum over splits sp = 0..SK-1 in order of the partials of columns c0..c0+15 of
// `row` ([split][row][Rpad] FP32), with split `mine` taken from own[] (still in TMEM when the
// others were stored).  SK = 0: run-time split count sk.
template <int SK>
__device__ __forceinline__ void reduce_chunk(const float* part, int Rpad, int row, int c0, int mine,
                                             const float* own, float* acc, int sk = SK) {
  const int nsp = SK > 0 ? SK : sk;
  float4 buf[(SK > 0 ? SK : 1) * 4];
  if (SK > 0) {
#pragma unroll
    for (int sp = 0; sp < (SK > 0 ? SK : 1); ++sp) {
      if (sp == mine) continue;
      const float4* src = reinterpret_cast<const float4*>(part + ((size_t)sp * kBM + row) * Rpad + c0);
#pragma unroll
      for (int i = 0; i < 4; ++i) buf[sp * 4 + i] = __ldcg(src + i);
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  for (int sp = 0; sp < nsp; ++sp) {
    float v[16];
    if (sp == mine) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = own[i];
    } else {
      float4 q[4];
      if (SK > 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = buf[(SK > 0 ? sp : 0) * 4 + i];
      } else {
        const float4* src = reinterpret_cast<const float4*>(part + ((size_t)sp * kBM + row) * Rpad + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = __ldcg(src + i);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v[4 * i] = q[i].x;
        v[4 * i + 1] = q[i].y;
        v[4 * i + 2] = q[i].z;
        v[4 * i + 3] = q[i].w;
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] += v[i];
  }
}

__device__ __forceinline__ float warp_reduce16(float* v, int lane) {
#pragma unroll
  for (int w = 8, off = 16; w >= 1; w >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float send = up ? v[i] : v[i + w];
      const float keep = up ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ int reduce16_index(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

__device__ __forceinline__ void epi_bar() {   // the four epilogue warps only
  asm volatile("bar.sync 1, 128;" ::: "memory");
}
// barrier of the four epilogue warps that also returns whether any of them passed true, so
// every epilogue thread takes the same branch
__device__ __forceinline__ bool epi_bar_any(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred)
      : "memory");
  return r != 0;
}

template <int PASS, int NA, int NB>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc(const __grid_constant__ TcMaps maps, const TcArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)p.stages * p.stage_bytes);
  uint64_t* empty = full + p.stages;
  uint64_t* tfull = empty + p.stages;        // [2] accumulator ready for the epilogue
  uint64_t* tempty = tfull + 2;              // [2] accumulator drained
  uint64_t* mdone = tempty + 2;              // every MMA issued has completed
  uint64_t* never = mdone + 1;               // test hook: no thread ever arrives here
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);          // [4][Rpad] (pass 2)
  // early pass 2 hands its tiles out dynamically (CTAs start at different times): the producer
  // takes the next tile from a global counter and queues its index for the MMA issuer and
  // the epilogue; -1 ends the sequence
  uint64_t* tq_full = reinterpret_cast<uint64_t*>(red + 4 * p.Rpad);
  uint64_t* tq_empty = tq_full + kTq;
  volatile int* tq = reinterpret_cast<volatile int*>(tq_empty + kTq);
  const bool dyn = (PASS == 3 && p.early) || PASS == 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // once a wait has expired in this E-step, later launches do nothing (the host reports it)
  if (*reinterpret_cast<volatile int*>(p.status) & 8) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 32 * kEpiWarps);
    }
    mbar_init(mdone, 1);
    mbar_init(never, 1);
    for (int q = 0; q < kTq; ++q) {
      mbar_init(&tq_full[q], 1);
      mbar_init(&tq_empty[q], 1 + 32 * kEpiWarps);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, p.tmem_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // pass 2 may be scheduled now: its CTAs take the SMs this grid frees, and each of its tiles
  // waits for the pass-1 tiles of its own task (all CTAs of this grid are resident by then)
  if (PASS == 1 && p.early) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t a_bytes = kBM * kBK * 2;                  // 16 KiB per A operand
  const uint32_t b_bytes = (uint32_t)p.Rpad * kBK * 2;     // per B operand
  uint32_t issued = 0;                                      // k-blocks the producer issued
  // next queued tile (bounded wait; -2 if it expired, which takes the abort path)
  auto tq_pop = [&](uint32_t& q) -> int {
    const uint32_t slot = q % kTq;
    if (!mbar_wait(&tq_full[slot], (q / kTq) & 1)) {
      *abort_flag = 1;
      atomicOr(p.status, 8);
      return -2;
    }
    const int v = tq[slot];
    mbar_arrive(&tq_empty[slot]);
    ++q;
    return v;
  };

  if (warp == 0) {
    // ---- TMA producer
    if (lane == 0) {
      uint32_t it = 0, qi = 0;
      bool stop = false;
      auto next = [&](int cur) {
        return dyn ? p.tile_lo + atomicAdd(p.tile_ctr, 1) : cur + (int)gridDim.x;
      };
      auto push = [&](int v) {
        const uint32_t slot = qi % kTq;
        if (qi >= (uint32_t)kTq && !mbar_wait(&tq_empty[slot], ((qi / kTq) - 1) & 1)) return false;
        tq[slot] = v;
        mbar_arrive(&tq_full[slot]);
        ++qi;
        return true;
      };
      for (int tile = dyn ? next(0) : p.tile_lo + (int)blockIdx.x;
           tile < p.ntiles && !stop && !*abort_flag; tile = next(tile)) {
        TileInfo ti;
        if (!tile_info<PASS>(p, tile, ti)) continue;
        if (dyn && !push(tile)) {
          *abort_flag = 1;
          atomicOr(p.status, 8);
          break;
        }
        const bool a_mn = PASS == 3 || ((PASS == 0 || PASS == 4) && ti.pass == 2);
        const int pi = ti.pass - 1;
        if (((PASS == 0 && ti.pass == 2) || (PASS == 3 && p.early)) &&
            !wait_pass1_done(&p.p1done[ti.t], p.n1[ti.t])) {
          *abort_flag = 1;                 // W of this task never completed
          atomicOr(p.status, 8);
          break;
        }
        for (int kb = 0; kb < ti.nk; ++kb, ++it) {
          const int s = (int)(it % p.stages);
          if (it >= (uint32_t)p.stages && !mbar_wait(&empty[s], ((it / p.stages) - 1) & 1)) {
            *abort_flag = 1;
            atomicOr(p.status, 8);
            stop = true;
            break;
          }
          if (*abort_flag) {
            stop = true;
            break;
          }
          // one-read pass 2: each 128-row tile of W (two k-blocks) is used once its pass-1
          // units have been reduced
          if (PASS == 4 && ti.pass == 2 && (kb & 1) == 0 &&
              !wait_flag(&p.wready[(ti.kx + kb * kBK) / kBM])) {
            *abort_flag = 1;
            atomicOr(p.status, 8);
            stop = true;
            break;
          }
          uint8_t* st = smem + (size_t)s * p.stage_bytes;
          mbar_expect_tx(&full[s], (uint32_t)p.stage_bytes);
          const int kcol = ti.kx + kb * kBK;
#pragma unroll
          for (int h = 0; h < NA; ++h) {
            uint8_t* ad = st + h * a_bytes;
            if (a_mn) {
              // Phi itself (rows n = kcol .., columns d = a_row ..): two 64-column boxes
              if (p.tiled) {
                tma_load_4d(ad, &maps.a[1][h], 0, kcol & (kBM - 1), ti.a_row / kBK, kcol / kBM, &full[s]);
                tma_load_4d(ad + a_bytes / 2, &maps.a[1][h], 0, kcol & (kBM - 1), ti.a_row / kBK + 1,
                            kcol / kBM, &full[s]);
              } else {
                tma_load_2d(ad, &maps.a[1][h], ti.a_row, kcol, &full[s]);
                tma_load_2d(ad + a_bytes / 2, &maps.a[1][h], ti.a_row + 64, kcol, &full[s]);
              }
            } else if (PASS == 2 || (PASS == 0 && pi == 1)) {
              tma_load_2d(ad, &maps.a[1][h], kcol, ti.a_row, &full[s]);
            } else if (p.tiled) {
              tma_load_4d(ad, &maps.a[0][h], 0, 0, kcol / kBK, ti.a_row / kBM, &full[s]);
            } else {
              tma_load_2d(ad, &maps.a[0][h], kcol, ti.a_row, &full[s]);
            }
          }
          // the Phi tile pf k-blocks ahead into L2, so that its load then comes from L2
          if (p.pf > 0 && kb + p.pf < ti.nk) {
            const int kpf = kcol + p.pf * kBK;
#pragma unroll
            for (int h = 0; h < NA; ++h) {
              if (a_mn && p.tiled) {
                tma_prefetch_4d(&maps.a[1][h], 0, kpf & (kBM - 1), ti.a_row / kBK, kpf / kBM);
                tma_prefetch_4d(&maps.a[1][h], 0, kpf & (kBM - 1), ti.a_row / kBK + 1, kpf / kBM);
              } else if (a_mn) {
                tma_prefetch_2d(&maps.a[1][h], ti.a_row, kpf);
                tma_prefetch_2d(&maps.a[1][h], ti.a_row + 64, kpf);
              } else if (PASS == 2 || (PASS == 0 && pi == 1)) {
                tma_prefetch_2d(&maps.a[1][h], kpf, ti.a_row);
              } else if (p.tiled) {
                tma_prefetch_4d(&maps.a[0][h], 0, 0, kpf / kBK, ti.a_row / kBM);
              } else {
                tma_prefetch_2d(&maps.a[0][h], kpf, ti.a_row);
              }
            }
          }
          // constant indices into the parameter block keep the maps in parameter space
          uint8_t* bst = st + NA * a_bytes;
          const int brow = ti.b_row + ti.col0;
          if (pi == 0) {
            tma_load_2d(bst, &maps.b[0][0], kcol, brow, &full[s]);
            if (NB == 2) tma_load_2d(bst + b_bytes, &maps.b[0][1], kcol, brow, &full[s]);
          } else {
            tma_load_2d(bst, &maps.b[1][0], kcol, brow, &full[s]);
            if (NB == 2) tma_load_2d(bst + b_bytes, &maps.b[1][1], kcol, brow, &full[s]);
          }
          issued = it + 1;
        }
      }
      if (dyn && !push(-1)) {          // the end of the sequence
        *abort_flag = 1;
        atomicOr(p.status, 8);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc_k = idesc_bf16(kBM, p.BR);
      const uint32_t idesc_mn = idesc_k | (1u << 15);      // A transposed (MN-major)
      uint32_t it = 0, lt = 0;
      if (p.stall != nullptr && *p.stall != 0 && !mbar_wait(never, 0)) {
        *abort_flag = 1;               // the bounded wait expired: take the abort path
        atomicOr(p.status, 8);
      }
      uint32_t qm = 0;
      for (int tile = dyn ? tq_pop(qm) : p.tile_lo + (int)blockIdx.x;
           tile >= 0 && tile < p.ntiles && !*abort_flag;
           tile = dyn ? tq_pop(qm) : tile + (int)gridDim.x) {
        TileInfo ti;
        if (!tile_info<PASS>(p, tile, ti)) continue;
        const bool a_mn = PASS == 3 || ((PASS == 0 || PASS == 4) && ti.pass == 2);
        const uint32_t idesc = a_mn ? idesc_mn : idesc_k;
        const int b = (int)(lt % p.nbuf);
        if (lt >= (uint32_t)p.nbuf && !mbar_wait(&tempty[b], ((lt / p.nbuf) - 1) & 1)) {
          *abort_flag = 1;
          atomicOr(p.status, 8);
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)b * p.tmem_cols;
        bool stop = false;
        for (int kb = 0; kb < ti.nk; ++kb, ++it) {
          const int s = (int)(it % p.stages);
          if (!mbar_wait(&full[s], (it / p.stages) & 1)) {
            *abort_flag = 1;
            atomicOr(p.status, 8);
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + (size_t)s * p.stage_bytes);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            // K-major: the next 16 k are 32 bytes along the swizzled row; MN-major: 16 rows down
            const uint64_t a0 = a_mn ? smem_desc_mn(st + kk * 2048, p.mn_lbo, p.mn_sbo)
                                     : smem_desc(st + kk * 32);
            const uint64_t a1 = a_mn ? smem_desc_mn(st + a_bytes + kk * 2048, p.mn_lbo, p.mn_sbo)
                                     : smem_desc(st + a_bytes + kk * 32);
            const uint32_t bo = st + NA * a_bytes + kk * 32;
            mma_bf16(dt, a0, smem_desc(bo), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            if (NB == 2) mma_bf16(dt, a0, smem_desc(bo + b_bytes), idesc, 1u);
            if (NA == 2) mma_bf16(dt, a1, smem_desc(bo), idesc, 1u);
          }
          mma_commit(&empty[s]);
        }
        if (stop) break;
        mma_commit(&tfull[b]);
        ++lt;
      }
      mma_commit(mdone);
      if (!mbar_wait(mdone, 0)) atomicOr(p.status, 8);
    }
  } else {
    // ---- epilogue: warp w may read TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31
    const int lg = warp & 3;
    const int etid = threadIdx.x - 64;                 // 0..127 among the epilogue warps
    uint32_t lt = 0, qe = 0;
    for (int tile = dyn ? tq_pop(qe) : p.tile_lo + (int)blockIdx.x;;
         tile = dyn ? tq_pop(qe) : tile + (int)gridDim.x) {
      if (dyn ? epi_bar_any(tile < 0) : tile >= p.ntiles) break;   // uniform over the warps
      TileInfo ti;
      if (!tile_info<PASS>(p, tile, ti)) continue;
      const int b = (int)(lt % p.nbuf);
      const bool ok = mbar_wait(&tfull[b], (lt / p.nbuf) & 1);
      if (!ok) {
        *abort_flag = 1;
        if (lane == 0) atomicOr(p.status, 8);
      }
      if (epi_bar_any(!ok || *abort_flag)) break;   // uniform across the epilogue warps
      tc_fence_after();
      const uint32_t trow = tmem + (uint32_t)b * p.tmem_cols + ((uint32_t)(32 * lg) << 16);
      if (PASS == 4 && ti.pass == 1) {
        // K split of a pass-1 row tile.  The last of the row tile's splitk units to arrive sums
        // the partials in split order (its own still in TMEM, the others' stored by them) and
        // stores the row tile of W as BF16 hi + lo; the others store their FP32 partials.  The
        // sums are the same whichever unit arrives last.
        const int g = ti.dtile, row = 32 * lg + lane;
        const int slot = g % p.nslot;
        volatile int* bc = reinterpret_cast<volatile int*>(tmem_slot + 2);
        float* part = p.wpart + (size_t)slot * p.splitk * kBM * p.Rpad;   // [split][row][Rpad]
        if (etid == 0) *bc = atomicAdd(&p.p1cnt[g], 1);
        epi_bar();
        const bool last = *bc == p.splitk - 1;
        epi_bar();                                 // every thread has read the role
        bool ok = true;
        if (!last) {
          // the slot's previous row tile must have been reduced (its partials read)
          if (etid == 0 && g >= p.nslot &&
              (p.task_active == nullptr || p.task_active[p.tile_task[g - p.nslot]]))
            ok = wait_flag(&p.wready[g - p.nslot]);
        } else {
          // the other units have arrived, so they are storing: wait for all of them
          if (etid == 0) ok = wait_count(&p.p1st[g], p.splitk - 1);
        }
        if (epi_bar_any(!ok)) {
          *abort_flag = 1;
          if (etid == 0) atomicOr(p.status, 8);
          break;
        }
        if (!last) {
          float4* mine = reinterpret_cast<float4*>(part + ((size_t)ti.split * kBM + row) * p.Rpad);
          for (int c0 = 0; c0 < p.Rpad; c0 += 16) {
            float v[16];
            tmem_ld16(trow + c0, v);
#pragma unroll
            for (int i = 0; i < 4; ++i)
              mine[c0 / 4 + i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
          }
          tc_fence_before();
          mbar_arrive(&tempty[b]);
          ++lt;
          __threadfence();
          epi_bar();
          if (etid == 0) atomicAdd(&p.p1st[g], 1);
          continue;
        }
        __threadfence();
        const int64_t n = (int64_t)ti.a_row + row;
        for (int c0 = 0; c0 < p.Rpad; c0 += 16) {
          float own[16], acc[16];
          tmem_ld16(trow + c0, own);
          switch (p.splitk) {
            case 2: reduce_chunk<2>(part, p.Rpad, row, c0, ti.split, own, acc); break;
            case 4: reduce_chunk<4>(part, p.Rpad, row, c0, ti.split, own, acc); break;
            default: reduce_chunk<0>(part, p.Rpad, row, c0, ti.split, own, acc, p.splitk); break;
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int j = c0 + i;
            if (j < p.R) {
              const __nv_bfloat16 hi = __float2bfloat16_rn(acc[i]);
              const __nv_bfloat16 lo = __float2bfloat16_rn(acc[i] - __bfloat162float(hi));
              p.w_hi[(int64_t)j * p.rows_total + n] = hi;
              p.w_lo[(int64_t)j * p.rows_total + n] = lo;
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[b]);
        ++lt;
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __threadfence();
        epi_bar();
        if (etid == 0) atomicExch(&p.wready[g], 1);
        continue;
      }
      if (ti.pass == 1) {
        const int64_t n = (int64_t)ti.a_row + 32 * lg + lane;     // global row of Phi
        for (int c0 = 0; c0 < p.Rpad; c0 += 16) {
          float v[16];
          tmem_ld16(trow + c0, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int j = ti.col0 + c0 + i;
            if (j < p.R) {
              const __nv_bfloat16 hi = __float2bfloat16_rn(v[i]);
              const __nv_bfloat16 lo = __float2bfloat16_rn(v[i] - __bfloat162float(hi));
              p.w_hi[(int64_t)j * p.rows_total + n] = hi;
              p.w_lo[(int64_t)j * p.rows_total + n] = lo;
            }
          }
        }
        if (PASS == 0 || (PASS == 1 && p.early)) {
          // publish this tile's part of W for the task's pass-2 tiles
          tc_fence_before();
          asm volatile("fence.proxy.async.global;" ::: "memory");
          __threadfence();
          epi_bar();
          if (etid == 0) signal_pass1_done(&p.p1done[ti.t]);
        }
      } else {
        const int d = ti.a_row + 32 * lg + lane;
        if (p.opcount != nullptr && ti.dtile == 0 && ti.col0 == 0 && etid == 0)
          atomicAdd(&p.opcount[ti.t], 1ull);
        if (p.raw) {
          // beta Phi^T W only: one TMEM read and one coalesced store per column
          for (int c0 = 0; c0 < p.Rpad; c0 += 16) {
            float acc[16];
            tmem_ld16(trow + c0, acc);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int j = ti.col0 + c0 + i;
              if (j < p.R) p.Z[((int64_t)ti.t * p.R + j) * p.Dp + d] = p.beta * acc[i];
            }
          }
        } else {
          for (int c0 = 0; c0 < p.Rpad; c0 += 16) {
            float vv[16], aa[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int j = ti.col0 + c0 + i;
              const int jj = j < p.R ? j : 0;
              const int64_t sys = (int64_t)ti.t * p.R + jj;
              vv[i] = j < p.R ? __ldg(p.V + sys * p.Dp + d) : 0.f;
              aa[i] = j < p.R ? __ldg(p.alpha + (int64_t)(jj / (p.K + 1)) * p.Dp + d) : 0.f;
            }
            float acc[16], dot[16];
            tmem_ld16(trow + c0, acc);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int j = ti.col0 + c0 + i;
              const float ad = fmaf(p.beta, acc[i], aa[i] * vv[i]);
              if (j < p.R) p.Z[((int64_t)ti.t * p.R + j) * p.Dp + d] = ad;
              dot[i] = vv[i] * ad;
            }
            const float tot = warp_reduce16(dot, lane);
            if ((lane & 1) == 0) red[lg * p.Rpad + c0 + reduce16_index(lane)] = tot;
          }
          epi_bar();
          if (p.part != nullptr) {
            for (int jl = etid; jl < p.Rpad && ti.col0 + jl < p.R; jl += 128)
              p.part[(int64_t)ti.dtile * p.S + (int64_t)ti.t * p.R + ti.col0 + jl] =
                  ((red[jl] + red[p.Rpad + jl]) + red[2 * p.Rpad + jl]) + red[3 * p.Rpad + jl];
          }
          epi_bar();
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[b]);
      ++lt;
    }
  }

  // ---- teardown: no copy may still be landing in shared memory when the CTA exits
  __syncwarp();
  if (*abort_flag && warp == 0 && lane == 0) {
    for (uint32_t k = issued; k > 0 && k + p.stages > issued; --k)
      mbar_wait(&full[(k - 1) % p.stages], ((k - 1) / p.stages) & 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, p.tmem_alloc);
}

// ---- set-up kernels ----------------------------------------------------------------------
// x = hi + lo with hi = bf16(x), lo = bf16(x - hi)
__global__ void k_split_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = src[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[i] = h;
    if (lo) lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// the same split written blocked: element (n, d) of Phi [rows][Dp] at
// ((n / 128) (Dp / 64) + d / 64) 8192 + (n % 128) 64 + d % 64
__global__ void k_split_bf16_tiled(const float* __restrict__ src, __nv_bfloat16* __restrict__ hi,
                                   __nv_bfloat16* __restrict__ lo, int64_t rows, int Dp) {
  const int64_t n_el = rows * Dp;
  const int nkb = Dp / 64;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_el;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i / Dp;
    const int d = (int)(i - n * Dp);
    const int64_t o = ((n >> 7) * nkb + (d >> 6)) * 8192 + (n & 127) * 64 + (d & 63);
    const float x = src[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[o] = h;
    if (lo) lo[o] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// PhiT[d][n] = Phi[n][d] split into BF16 pairs, 32 x 32 tiles through shared memory
__global__ void k_transpose_split(const float* __restrict__ phi, __nv_bfloat16* __restrict__ thi,
                                  __nv_bfloat16* __restrict__ tlo, int64_t rows, int Dp) {
  __shared__ float tile[32][33];
  const int64_t n0 = (int64_t)blockIdx.y * 32;
  const int d0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) tile[r][threadIdx.x] = phi[(n0 + r) * Dp + d0 + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const float x = tile[threadIdx.x][r];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const int64_t o = (int64_t)(d0 + r) * rows + n0 + threadIdx.x;
    thi[o] = h;
    if (tlo) tlo[o] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// ---- host side ---------------------------------------------------------------------------
namespace {

struct TcState {
  int NA, NB;
  int Rpad, BR, nbox, stages, stage_bytes, smem_bytes, nbuf, ncol;
  uint32_t tmem_cols, tmem_alloc;
  __nv_bfloat16 *phi_hi, *phi_lo, *phit_hi, *phit_lo, *w_hi, *w_lo;
  CUtensorMap tm_phi[2], tm_phit[2], tm_d[2], tm_w[2], tm_phimn[2];
  // 3 (default): two persistent launches, pass 2 reading Phi itself as an MN-major operand;
  // 2: two launches, pass 2 reading a transposed copy of Phi (twice the device memory);
  // 0: both passes of every task in one launch, pass-2 tiles waiting on per-task counters
  int mode;
  uint32_t mn_lbo, mn_sbo;
  int *tile_code, *tile_task2, *n1, *p1done;   // fused tile list; per-task counts [T] + tile counter
  int early;                                   // mode 3: pass 2 launched programmatically
  int pf;                                      // L2 prefetch distance of the Phi tiles (k-blocks)
  int tiled;                                   // Phi planes stored blocked (see TcArgs)
  std::vector<int> tstart;                     // first fused tile of each task (host)
  // mode 4 (one read of Phi per application): unit list, split-K partials and counters
  int *u_code, *u_task, nunits, splitk, nslot;
  std::vector<int> ustart;                     // first unit of each task (per-task launches)
  float* wpart;
  int* m4;                                     // [3 row tiles + 1]: p1cnt, wready, p1st, unit counter
};


template <int PASS, int NA, int NB>
cudaError_t set_smem_attr(int bytes) {
  return cudaFuncSetAttribute(k_tc<PASS, NA, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

TcArgs base_args(Ctx* c, TcState* s) {
  TcArgs a{};
  a.tile_task = c->tile_task;
  a.drow = c->drow;
  a.R = c->R;
  a.K = c->K;
  a.C = c->C;
  a.Dp = c->Dp;
  a.D = c->D;
  a.S = c->S;
  a.rows_total = c->rows_total;
  a.Rpad = s->Rpad;
  a.BR = s->BR;
  a.nbox = s->nbox;
  a.stages = s->stages;
  a.stage_bytes = s->stage_bytes;
  a.tmem_cols = s->tmem_cols;
  a.tmem_alloc = s->tmem_alloc;
  a.nbuf = s->nbuf;
  a.ncol = s->ncol;
  a.mn_lbo = s->mn_lbo;
  a.mn_sbo = s->mn_sbo;
  a.w_hi = s->w_hi;
  a.w_lo = s->w_lo;
  a.alpha = c->alpha;
  a.beta = (float)c->beta;
  a.status = &c->counters[2];
  a.stall = c->stall_flag;
  a.pf = s->pf;
  a.tiled = s->tiled;
  return a;
}

template <int NA, int NB>
cudaError_t run_passes(Ctx* c, TcState* s, const float* V, float* Z, int with_dots) {
  TcArgs a = base_args(c, s);
  // the bytes one stage receives: NA planes of the Phi tile and NB of the vector tile (a
  // CMCS_BF16_MIXED context runs NA = 1 in its first solve inside stages sized for NA = 2)
  a.stage_bytes = NA * kBM * kBK * 2 + NB * s->Rpad * kBK * 2;
  a.task_active = with_dots ? c->task_active : nullptr;
  // per-task application counts: the first T for the BF16 pair, the next T for one plane
  a.opcount = c->prof_on ? reinterpret_cast<unsigned long long*>(c->opcount) + (NA == 1 ? c->T : 0)
                         : nullptr;
  a.V = V;
  a.Z = Z;
  a.raw = with_dots;             // the CG step: its update kernel completes A d and d^T A d
  a.part = nullptr;
  a.tile_code = s->tile_code;
  a.tile_task2 = s->tile_task2;
  a.n1 = s->n1;
  a.p1done = s->p1done;
  a.tile_ctr = s->p1done + c->T;
  const int sms = c->sm_count > 0 ? c->sm_count : 1;
  const int ndt = c->Dp / kBM;
  const int nloop = c->per_task ? c->T : 1;
  TcMaps maps;
  maps.a[0][0] = s->tm_phi[0];
  maps.a[0][1] = s->tm_phi[NA - 1];
  maps.a[1][0] = s->mode == 2 ? s->tm_phit[0] : s->tm_phimn[0];
  maps.a[1][1] = s->mode == 2 ? s->tm_phit[NA - 1] : s->tm_phimn[NA - 1];
  maps.b[0][0] = s->tm_d[0];
  maps.b[0][1] = s->tm_d[NB - 1];
  maps.b[1][0] = s->tm_w[0];
  maps.b[1][1] = s->tm_w[NB - 1];
  if (s->mode == 4) {
    // one persistent launch per application: pass-1 units split along K and pass-2 tiles,
    // task after task, handed out in order from a counter; a task's Phi is read from HBM by
    // its pass-1 units and again, from L2, by its pass-2 tiles shortly after
    const int ntl = (int)(c->rows_total / kBM);
    cudaError_t e = cudaMemsetAsync(s->m4, 0, sizeof(int) * (3 * (size_t)ntl + 1), c->stream);
    if (e != cudaSuccess) return e;
    a.u_code = s->u_code;
    a.u_task = s->u_task;
    a.splitk = s->splitk;
    a.nslot = s->nslot;
    a.wpart = s->wpart;
    a.p1cnt = s->m4;
    a.wready = s->m4 + ntl;
    a.p1st = s->m4 + 2 * ntl;
    a.tile_ctr = s->m4 + 3 * ntl;
    for (int t = 0; t < nloop; ++t) {
      // every unit in one launch, or (comparison schedule) the units of one task per launch
      a.tile_lo = c->per_task ? s->ustart[(size_t)t] : 0;
      a.ntiles = c->per_task ? s->ustart[(size_t)t + 1] : s->nunits;
      const int n = a.ntiles - a.tile_lo;
      if (c->per_task && t > 0) {    // the unit counter restarts at each task's first unit
        e = cudaMemsetAsync(a.tile_ctr, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) return e;
      }
      k_tc<4, NA, NB><<<n < sms ? n : sms, kTcThreads, s->smem_bytes, c->stream>>>(maps, a);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      c->launches += 1;
    }
    return cudaSuccess;
  }
  for (int t = 0; t < nloop; ++t) {
    // all tasks in one persistent launch, or (comparison schedule) one launch per task
    if (s->mode == 0) {
      cudaError_t e = cudaMemsetAsync(s->p1done, 0, sizeof(int) * c->T, c->stream);
      if (e != cudaSuccess) return e;
      a.tile_lo = c->per_task ? s->tstart[t] : 0;
      a.ntiles = c->per_task ? s->tstart[t + 1] : s->tstart[c->T];
      const int n = a.ntiles - a.tile_lo;
      k_tc<0, NA, NB><<<n < sms ? n : sms, kTcThreads, s->smem_bytes, c->stream>>>(maps, a);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      c->launches += 1;
      continue;
    }
    // default schedule: pass 2 launched programmatically, its tiles starting on the SMs that
    // pass 1's partial last wave leaves idle (the per-task counters order the data)
    a.early = (s->mode == 3 && !c->per_task && s->early) ? 1 : 0;
    if (a.early) {       // the per-task counts and the tile counter (p1done[T])
      cudaError_t e = cudaMemsetAsync(s->p1done, 0, sizeof(int) * ((size_t)c->T + 1), c->stream);
      if (e != cudaSuccess) return e;
    }
    a.tile_lo = (c->per_task ? (int)(c->hrow[t] / kBM) : 0) * s->ncol;
    a.ntiles = (c->per_task ? (int)(c->hrow[t + 1] / kBM) : (int)(c->rows_total / kBM)) * s->ncol;
    int n = a.ntiles - a.tile_lo;
    k_tc<1, NA, NB><<<n < sms ? n : sms, kTcThreads, s->smem_bytes, c->stream>>>(maps, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    a.tile_lo = (c->per_task ? t * ndt : 0) * s->ncol;
    a.ntiles = (c->per_task ? (t + 1) * ndt : c->T * ndt) * s->ncol;
    n = a.ntiles - a.tile_lo;
    if (a.early) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(n < sms ? n : sms));
      cfg.blockDim = dim3(kTcThreads);
      cfg.dynamicSmemBytes = (size_t)s->smem_bytes;
      cfg.stream = c->stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, k_tc<3, NA, NB>, maps, a);
    } else if (s->mode == 3) {
      k_tc<3, NA, NB><<<n < sms ? n : sms, kTcThreads, s->smem_bytes, c->stream>>>(maps, a);
    } else {
      k_tc<2, NA, NB><<<n < sms ? n : sms, kTcThreads, s->smem_bytes, c->stream>>>(maps, a);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    c->launches += 2;
  }
  return cudaSuccess;
}

}  // namespace

int tc_create(Ctx* c) {
  TcState* s = new (std::nothrow) TcState();
  if (!s) return 1;
  c->tc = s;
  s->NA = (c->precision == CMCS_BF16X3 || c->precision == CMCS_BF16_MIXED) ? 2 : 1;
  s->NB = 2;
  // columns: tiles of at most 256 (one MMA width), so two accumulators always fit in TMEM
  s->ncol = (c->R + 255) / 256;
  s->nbox = 1;
  s->BR = (int)round_up((c->R + s->ncol - 1) / s->ncol, 16);
  s->Rpad = s->BR;
  s->tmem_cols = 32;
  while ((int)s->tmem_cols < s->Rpad) s->tmem_cols <<= 1;
  s->nbuf = 2 * s->tmem_cols <= 512 ? 2 : 1;     // double-buffer the accumulator when it fits
  s->tmem_alloc = s->tmem_cols * (uint32_t)s->nbuf;
  s->stage_bytes = s->NA * kBM * kBK * 2 + s->NB * s->Rpad * kBK * 2;
  const int extra = 1024 + (2 * 6 + 5) * 8 + 16 + 4 * s->Rpad * 4 + 64 + kTqBytes;
  s->stages = (kSmemBudget - extra) / s->stage_bytes;
  if (s->stages > 6) s->stages = 6;
  if (s->stages < 2) {
    snprintf(c->err, sizeof(c->err), "tensor-core operator: stage of %d bytes does not fit", s->stage_bytes);
    return 1;
  }
  {
    const char* sv = getenv("CMCS_TC_STAGES");   // evaluation switch: a shallower pipeline
    const int v = sv ? atoi(sv) : 0;
    if (v >= 2 && v < s->stages) s->stages = v;
  }
  s->smem_bytes = s->stages * s->stage_bytes + 1024 + (2 * s->stages + 6) * 8 + 16 + 4 * s->Rpad * 4 + 64 + kTqBytes;

  const int64_t rows = c->rows_total, Dp = c->Dp, S = c->S, R = c->R;
  auto alloc = [&](__nv_bfloat16** p, int64_t n) {
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(__nv_bfloat16) * (size_t)n) == cudaSuccess;
  };
  {
    const char* mv = getenv("CMCS_TC_MODE");     // evaluation switch between the schedules
    s->mode = mv ? atoi(mv) : 3;
    if (s->mode != 0 && s->mode != 2 && s->mode != 4) s->mode = 3;
    // the one-read schedule handles one column tile and the batched launch
    if (s->mode == 4 && s->ncol != 1) s->mode = 3;
    const char* ev = getenv("CMCS_TC_EARLY");    // evaluation switch: 0 launches pass 2 plainly
    s->early = ev ? atoi(ev) != 0 : 1;
    const char* pv = getenv("CMCS_TC_PREFETCH"); // evaluation switch: L2 prefetch distance
    s->pf = pv ? atoi(pv) : 0;
    if (s->pf < 0) s->pf = 0;
    const char* tv = getenv("CMCS_TC_TILED");    // evaluation switch: 0 keeps Phi row-major
    s->tiled = tv ? atoi(tv) != 0 : 1;
  }
  s->mn_lbo = 8192;      // 64-column halves of the MN-major A tile are 8 KiB apart
  s->mn_sbo = 1024;      // groups of 8 k rows are 1 KiB apart
  bool okm = alloc(&s->phi_hi, rows * Dp) &&
             alloc(reinterpret_cast<__nv_bfloat16**>(&c->dhi), S * Dp) &&
             alloc(reinterpret_cast<__nv_bfloat16**>(&c->dlo), S * Dp) && alloc(&s->w_hi, R * rows) &&
             alloc(&s->w_lo, R * rows);
  if (okm && s->NA == 2) okm = alloc(&s->phi_lo, rows * Dp);
  if (okm && s->mode == 2) okm = alloc(&s->phit_hi, rows * Dp) && (s->NA == 1 || alloc(&s->phit_lo, rows * Dp));
  // fused tile list.  The pass-1 tiles of task t + L go ahead of the pass-2 tiles of task t
  // (lookahead L; every pass-2 tile comes after all pass-1 tiles of its task, so a CTA only
  // ever waits on tiles earlier in the list).  L >= T - 1 puts all pass-1 tiles first: pass-2
  // tiles of finished tasks then fill the last, partial wave of pass 1.
  if (okm) {
    const int ndt = (int)(Dp / kBM);
    const char* lv = getenv("CMCS_TC_LOOKAHEAD");
    int L = lv ? atoi(lv) : c->T;
    if (L < 0) L = 0;
    if (c->per_task) L = 0;     // one launch per task: its pass-1 tiles, then its pass-2 tiles
    std::vector<int> code, task2, n1((size_t)c->T);
    s->tstart.assign((size_t)c->T + 1, 0);
    auto emit1 = [&](int t) {
      s->tstart[(size_t)t] = (int)code.size();     // per-task launches: P1(t), P2(t) contiguous
      const int nr = (int)(c->hNp[t] / kBM) * s->ncol;
      n1[(size_t)t] = nr;
      for (int i = 0; i < nr; ++i) {
        code.push_back(i << 2);
        task2.push_back(t);
      }
    };
    for (int t = 0; t <= L && t < c->T; ++t) emit1(t);
    for (int t = 0; t < c->T; ++t) {
      for (int i = 0; i < ndt * s->ncol; ++i) {
        code.push_back((i << 2) | 1);
        task2.push_back(t);
      }
      if (t + L + 1 < c->T) emit1(t + L + 1);
    }
    s->tstart[(size_t)c->T] = (int)code.size();
    okm = cudaMalloc(reinterpret_cast<void**>(&s->tile_code), sizeof(int) * code.size()) == cudaSuccess &&
          cudaMalloc(reinterpret_cast<void**>(&s->tile_task2), sizeof(int) * task2.size()) == cudaSuccess &&
          cudaMalloc(reinterpret_cast<void**>(&s->n1), sizeof(int) * (size_t)c->T) == cudaSuccess &&
          cudaMalloc(reinterpret_cast<void**>(&s->p1done), sizeof(int) * ((size_t)c->T + 1)) == cudaSuccess;
    if (okm) {
      cudaMemcpyAsync(s->tile_code, code.data(), sizeof(int) * code.size(), cudaMemcpyHostToDevice, c->stream);
      cudaMemcpyAsync(s->tile_task2, task2.data(), sizeof(int) * task2.size(), cudaMemcpyHostToDevice, c->stream);
      cudaMemcpyAsync(s->n1, n1.data(), sizeof(int) * (size_t)c->T, cudaMemcpyHostToDevice, c->stream);
      cudaStreamSynchronize(c->stream);    // the host vectors go out of scope
    }
  }
  if (okm && s->mode == 4) {
    // unit list: all pass-1 units of task 0, then per task t the first L pass-1 units of task
    // t + 1, the pass-2 tiles of task t and the rest of task t + 1's pass-1 units (a pass-2
    // tile only ever waits on units earlier in the list)
    const char* kv = getenv("CMCS_TC_SPLITK");   // evaluation switches of the one-read schedule
    const char* lv = getenv("CMCS_TC_LOOKAHEAD");
    const int nkb = (int)(Dp / kBK);
    s->splitk = kv ? atoi(kv) : 4;
    if (s->splitk < 1) s->splitk = 1;
    if (s->splitk > 8) s->splitk = 8;
    if (s->splitk > nkb) s->splitk = nkb;
    int L = lv ? atoi(lv) : 64;
    if (L < 0 || c->per_task) L = 0;   // per-task launches: each task's units contiguous
    const int ndt = (int)(Dp / kBM);
    std::vector<std::vector<int>> p1((size_t)c->T);
    for (int t = 0; t < c->T; ++t)
      for (int64_t g = c->hrow[t] / kBM; g < c->hrow[t + 1] / kBM; ++g)
        for (int sp = 0; sp < s->splitk; ++sp) p1[(size_t)t].push_back((int)(g << 4) | (sp << 1));
    std::vector<int> code, task;
    auto put = [&](int t, int v) {
      code.push_back(v);
      task.push_back(t);
    };
    s->ustart.assign((size_t)c->T + 1, 0);
    for (int v : p1[0]) put(0, v);
    for (int t = 0; t < c->T; ++t) {
      const bool nxt = t + 1 < c->T;
      const size_t l = nxt ? std::min((size_t)L, p1[(size_t)t + 1].size()) : 0;
      for (size_t i = 0; i < l; ++i) put(t + 1, p1[(size_t)t + 1][i]);
      for (int j = 0; j < ndt; ++j) put(t, (j << 1) | 1);
      if (nxt)
        for (size_t i = l; i < p1[(size_t)t + 1].size(); ++i) put(t + 1, p1[(size_t)t + 1][i]);
    }
    s->nunits = (int)code.size();
    // first unit of each task (meaningful with L = 0, where a task's units are contiguous)
    for (int t = 0, u = 0; t < c->T; ++t) {
      while (u < s->nunits && task[(size_t)u] != t) ++u;
      s->ustart[(size_t)t] = u;
    }
    s->ustart[(size_t)c->T] = s->nunits;
    // partials of about three tasks' row tiles in flight (a slot waits for its previous row
    // tile's reduction, so fewer only costs time)
    const int ntl = (int)(rows / kBM);
    s->nslot = std::min(ntl, 64);
    okm = cudaMalloc(reinterpret_cast<void**>(&s->u_code), sizeof(int) * code.size()) == cudaSuccess &&
          cudaMalloc(reinterpret_cast<void**>(&s->u_task), sizeof(int) * task.size()) == cudaSuccess &&
          cudaMalloc(reinterpret_cast<void**>(&s->m4), sizeof(int) * (3 * (size_t)ntl + 1)) == cudaSuccess &&
          cudaMalloc(reinterpret_cast<void**>(&s->wpart),
                     sizeof(float) * (size_t)s->nslot * s->splitk * s->Rpad * kBM) == cudaSuccess;
    if (okm) {
      cudaMemcpyAsync(s->u_code, code.data(), sizeof(int) * code.size(), cudaMemcpyHostToDevice, c->stream);
      cudaMemcpyAsync(s->u_task, task.data(), sizeof(int) * task.size(), cudaMemcpyHostToDevice, c->stream);
      cudaStreamSynchronize(c->stream);    // the host vectors go out of scope
    }
  }
  if (!okm) {
    snprintf(c->err, sizeof(c->err), "tensor-core operator: device allocation failed");
    return 1;
  }
  if (s->tiled)
    k_split_bf16_tiled<<<4096, 256, 0, c->stream>>>(c->phi, s->phi_hi, s->phi_lo, rows, (int)Dp);
  else
    k_split_bf16<<<4096, 256, 0, c->stream>>>(c->phi, s->phi_hi, s->phi_lo, rows * Dp);
  if (s->mode == 2)
    k_transpose_split<<<dim3(Dp / 32, (unsigned)(rows / 32)), dim3(32, 8), 0, c->stream>>>(
        c->phi, s->phit_hi, s->phit_lo, rows, (int)Dp);
  cudaMemsetAsync(c->dhi, 0, sizeof(__nv_bfloat16) * S * Dp, c->stream);
  cudaMemsetAsync(c->dlo, 0, sizeof(__nv_bfloat16) * S * Dp, c->stream);
  auto enc_phi = [&](CUtensorMap* m, const __nv_bfloat16* base, uint32_t box_rows) {
    return s->tiled ? encode_blocked(m, base, Dp, rows, box_rows) : encode_2d(m, base, Dp, rows, box_rows);
  };
  bool ok = enc_phi(&s->tm_phi[0], s->phi_hi, kBM) &&
            (s->mode != 2 || encode_2d(&s->tm_phit[0], s->phit_hi, rows, Dp, kBM)) &&
            encode_2d(&s->tm_d[0], c->dhi, Dp, S, s->BR) && encode_2d(&s->tm_d[1], c->dlo, Dp, S, s->BR) &&
            encode_2d(&s->tm_w[0], s->w_hi, rows, R, s->BR) && encode_2d(&s->tm_w[1], s->w_lo, rows, R, s->BR);
  if (ok && s->NA == 2)
    ok = enc_phi(&s->tm_phi[1], s->phi_lo, kBM) &&
         (s->mode != 2 || encode_2d(&s->tm_phit[1], s->phit_lo, rows, Dp, kBM));
  if (ok) ok = enc_phi(&s->tm_phimn[0], s->phi_hi, 64);
  if (ok && s->NA == 2) ok = enc_phi(&s->tm_phimn[1], s->phi_lo, 64);
  if (!ok) {
    snprintf(c->err, sizeof(c->err), "tensor-core operator: tensor map encoding failed");
    return 1;
  }
  // both plane counts: a CMCS_BF16_MIXED context (NA = 2 storage) also runs the one-plane kernels
  cudaError_t e = set_smem_attr<1, 1, 2>(s->smem_bytes);
  if (e == cudaSuccess) e = set_smem_attr<2, 1, 2>(s->smem_bytes);
  if (e == cudaSuccess) e = set_smem_attr<3, 1, 2>(s->smem_bytes);
  if (e == cudaSuccess) e = set_smem_attr<0, 1, 2>(s->smem_bytes);
  if (e == cudaSuccess) e = set_smem_attr<4, 1, 2>(s->smem_bytes);
  if (e == cudaSuccess && s->NA == 2) e = set_smem_attr<1, 2, 2>(s->smem_bytes);
  if (e == cudaSuccess && s->NA == 2) e = set_smem_attr<2, 2, 2>(s->smem_bytes);
  if (e == cudaSuccess && s->NA == 2) e = set_smem_attr<3, 2, 2>(s->smem_bytes);
  if (e == cudaSuccess && s->NA == 2) e = set_smem_attr<0, 2, 2>(s->smem_bytes);
  if (e == cudaSuccess && s->NA == 2) e = set_smem_attr<4, 2, 2>(s->smem_bytes);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "tensor-core operator set-up: %s", cudaGetErrorString(e));
    return 1;
  }
  c->launches += 2;
  return 0;
}

void tc_destroy(Ctx* c) {
  TcState* s = static_cast<TcState*>(c->tc);
  if (!s) return;
  void* ptrs[] = {s->phi_hi, s->phi_lo, s->phit_hi, s->phit_lo, s->w_hi, s->w_lo, c->dhi, c->dlo,
                  s->tile_code, s->tile_task2, s->n1, s->p1done, s->u_code, s->u_task, s->m4,
                  s->wpart};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->dhi = c->dlo = nullptr;
  delete s;
  c->tc = nullptr;
}

int tc_max_stages(Ctx* c) {
  TcState* s = static_cast<TcState*>(c->tc);
  if (!s) return 0;
  const int extra = 1024 + (2 * 6 + 5) * 8 + 16 + 4 * s->Rpad * 4 + 64 + kTqBytes;
  int m = (kSmemBudget - extra) / s->stage_bytes;
  return m > 6 ? 6 : m;
}

int tc_set_stages(Ctx* c, int stages) {
  TcState* s = static_cast<TcState*>(c->tc);
  if (!s) return 0;
  if (stages >= 2 && stages <= tc_max_stages(c)) {
    s->stages = stages;
    s->smem_bytes = s->stages * s->stage_bytes + 1024 + (2 * s->stages + 6) * 8 + 16 + 4 * s->Rpad * 4 + 64 + kTqBytes;
  }
  return s->stages;
}

cudaError_t tc_refresh(Ctx* c) {
  TcState* s = static_cast<TcState*>(c->tc);
  if (!s) return cudaSuccess;
  const int64_t rows = c->rows_total, Dp = c->Dp;
  if (s->tiled)
    k_split_bf16_tiled<<<4096, 256, 0, c->stream>>>(c->phi, s->phi_hi, s->phi_lo, rows, (int)Dp);
  else
    k_split_bf16<<<4096, 256, 0, c->stream>>>(c->phi, s->phi_hi, s->phi_lo, rows * Dp);
  if (s->mode == 2)
    k_transpose_split<<<dim3(Dp / 32, (unsigned)(rows / 32)), dim3(32, 8), 0, c->stream>>>(
        c->phi, s->phit_hi, s->phit_lo, rows, (int)Dp);
  c->launches += 2;
  return cudaGetLastError();
}

cudaError_t tc_split_vectors(Ctx* c, const float* V) {
  k_split_bf16<<<4096, 256, 0, c->stream>>>(V, static_cast<__nv_bfloat16*>(c->dhi),
                                            static_cast<__nv_bfloat16*>(c->dlo), (int64_t)c->S * c->Dp);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t tc_operator(Ctx* c, const float* V, float* Z, int with_dots) {
  TcState* s = static_cast<TcState*>(c->tc);
  if (!s) return cudaErrorNotSupported;
  // one BF16 plane of Phi (CMCS_BF16_REFINE; the first solve of CMCS_BF16_MIXED, whose storage
  // keeps both planes) or the BF16 pair
  return (s->NA == 2 && !one_plane(c)) ? run_passes<2, 2>(c, s, V, Z, with_dots)
                                        : run_passes<1, 2>(c, s, V, Z, with_dots);
}

}  // namespace cmcs
