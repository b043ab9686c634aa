// Structured sensing Phi_t = Omega_t F (Sec. 4) for signal lengths beyond one CTA's shared
// memory, and for lengths D = 2^a 5^b that are not powers of two (the paper's timings reach
// D = 100,000 = 2^5 5^5).
//
// The transform of length D = n1 * n2 is split in the four-step way: with the input index
// n = n2 * i1 + i2 (i1 < n1, i2 < n2) and the frequency k = k1 + n1 * k2,
//     X[k1 + n1 k2] = sum_i2 W_n2^{i2 k2} W_D^{i2 k1} sum_i1 W_n1^{i1 k1} x[n2 i1 + i2],
// W_M = e^{-2 pi i / M}.  One application of A = beta Re(F^H diag(m) F) + diag(alpha) to a
// pair of real systems (packed as v1 + i v2, as in the single-CTA path) is three launches:
//   1. column pass: length-n1 transforms over i1 for a block of nb columns i2, times the
//      twiddle W_D^{i2 k1}, stored as Y[k1][i2] (i2 fastest);
//   2. row pass: per row k1, the length-n2 transform over i2 (frequencies k1 + n1 k2), the
//      symmetrised mask, the inverse length-n2 transform and the conjugate twiddle;
//   3. inverse column pass: length-n1 inverse transforms over k1, then the epilogue:
//      A d and the per-block partial d^T A d (CG), the FP64 residual b - A x (refinement),
//      or b0 = beta Re(F^H y) (set-up; it enters at the row pass with the measured spectrum).
// Every sub-transform runs in shared memory as a Stockham autosort FFT with radix 4, 2 and 5
// passes (natural order in and out), twiddles from tables evaluated in FP64 on the host.
// The CG operator runs in FP32, the residual and b0 in FP64.  No CTA waits on another.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "cmcs_internal.cuh"

namespace cmcs {
namespace {

constexpr int kFsThreads = 256;
constexpr int kFsMaxLen = 1024;          // longest sub-transform
constexpr int kFsMaxRadices = 12;
constexpr size_t kFsSmemBudget = 140 * 1024;   // shared memory of one FP64 CTA

template <typename CT>
struct Cx;
template <>
struct Cx<float2> {
  using R = float;
  __device__ __forceinline__ static float2 mk(float a, float b) { return make_float2(a, b); }
};
template <>
struct Cx<double2> {
  using R = double;
  __device__ __forceinline__ static double2 mk(double a, double b) { return make_double2(a, b); }
};

template <typename CT>
__device__ __forceinline__ CT fs_mul(CT a, CT b) {
  return Cx<CT>::mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename CT>
__device__ __forceinline__ CT fs_mulc(CT a, CT b) {   // a * conj(b)
  return Cx<CT>::mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename CT>
__device__ __forceinline__ CT fs_add(CT a, CT b) { return Cx<CT>::mk(a.x + b.x, a.y + b.y); }
template <typename CT>
__device__ __forceinline__ CT fs_sub(CT a, CT b) { return Cx<CT>::mk(a.x - b.x, a.y - b.y); }

}  // namespace

// radices of one sub-transform of length L (product of r[0..n)), and for pass q the
// multiply-high reciprocals of L / r[q] and of Ns = r[0] ... r[q-1] (see fs_div)
struct FsRadix {
  int L, n;
  int r[kFsMaxRadices];
  uint64_t mM[kFsMaxRadices], mN[kFsMaxRadices];
};

// the split D = n1 * n2 and the CTA shapes of the three passes
struct FsPlan {
  int n1, n2;
  int nb;     // columns i2 per CTA in the FP64 column passes (divides n2, a power of two)
  int nb32;   // the same for the FP32 column passes
  int nbr;    // rows k1 per CTA in the FP64 row pass (the last block may be partial)
  int nbr32;  // the same for the FP32 row pass
  uint64_t mn2;   // reciprocal of n2
  FsRadix p1, p2;
};

// which systems a launch covers: pairs (2p, 2p+1) of columns j' < Rc, system j = j' * jstride
struct FsPairs {
  int R, K, C, Dp, D, Rc, jstride, npair;
};

namespace {

// floor(n / d) for 0 <= n < 2^15 and 1 <= d <= 1024 from m = ceil(2^32 / d): the high word of
// n * m (m = 2^32 for d = 1).  Exact over that whole range (checked exhaustively on the host).
__device__ __forceinline__ int fs_div(int n, uint64_t m) {
  return (int)(__umulhi((unsigned)n, (unsigned)m) + ((m >> 32) != 0 ? (unsigned)n : 0u));
}

// one Stockham pass of radix RX over nseq sequences of length L (stride ls) from src to dst:
// for j < L / RX, k = j mod Ns: v_r = src[j + r L/RX] W_{Ns RX}^{k r}, then the RX-point DFT,
// written to dst[floor(j / Ns) Ns RX + k + r Ns]
template <int RX, typename CT, bool INV>
__device__ __forceinline__ void fs_pass(const CT* __restrict__ src, CT* __restrict__ dst, int L,
                                        int Ns, uint64_t mM, uint64_t mN, int nseq, int ls,
                                        const CT* __restrict__ tab) {
  const int M = L / RX, ts = L / (Ns * RX);
  // 5-point DFT constants W_5 = (c1, -s1), W_5^2 = (c2, -s2), from the table
  CT w51, w52;
  if constexpr (RX == 5) {
    w51 = tab[L / 5];
    w52 = tab[2 * (L / 5)];
  }
  for (int idx = threadIdx.x; idx < nseq * M; idx += blockDim.x) {
    const int s = fs_div(idx, mM), j = idx - s * M;
    const int jq = fs_div(j, mN), k = j - jq * Ns;
    const CT* in = src + s * ls;
    CT* out = dst + s * ls;
    CT v[RX];
    v[0] = in[j];
#pragma unroll
    for (int r = 1; r < RX; ++r) {
      const CT w = tab[k * r * ts];
      v[r] = INV ? fs_mulc(in[j + r * M], w) : fs_mul(in[j + r * M], w);
    }
    CT y[RX];
    if constexpr (RX == 2) {
      y[0] = fs_add(v[0], v[1]);
      y[1] = fs_sub(v[0], v[1]);
    } else if constexpr (RX == 4) {
      const CT t0 = fs_add(v[0], v[2]), t1 = fs_sub(v[0], v[2]);
      const CT t2 = fs_add(v[1], v[3]), t3 = fs_sub(v[1], v[3]);
      // forward W_4 = -i: y1 = t1 - i t3, y3 = t1 + i t3 (inverse: signs swapped)
      const CT mit3 = Cx<CT>::mk(t3.y, -t3.x);
      y[0] = fs_add(t0, t2);
      y[2] = fs_sub(t0, t2);
      y[1] = INV ? fs_sub(t1, mit3) : fs_add(t1, mit3);
      y[3] = INV ? fs_add(t1, mit3) : fs_sub(t1, mit3);
    } else {
      // 5-point DFT in symmetric form: with t1 = v1 + v4, t2 = v2 + v3, t3 = v1 - v4,
      // t4 = v2 - v3, cos/sin c_q, s_q of 2 pi q / 5:
      //   y0 = v0 + t1 + t2,  y1, y4 = a1 -+ i b1,  y2, y3 = a2 -+ i b2 (forward; inverse +-)
      //   a1 = v0 + c1 t1 + c2 t2, a2 = v0 + c2 t1 + c1 t2, b1 = s1 t3 + s2 t4, b2 = s2 t3 - s1 t4
      using RT = typename Cx<CT>::R;
      const RT c1 = w51.x, s1 = -w51.y, c2 = w52.x, s2 = -w52.y;
      const CT t1 = fs_add(v[1], v[4]), t2 = fs_add(v[2], v[3]);
      const CT t3 = fs_sub(v[1], v[4]), t4 = fs_sub(v[2], v[3]);
      y[0] = fs_add(v[0], fs_add(t1, t2));
      const CT a1 = Cx<CT>::mk(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
      const CT a2 = Cx<CT>::mk(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
      const CT b1 = Cx<CT>::mk(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
      const CT b2 = Cx<CT>::mk(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
      // -i b = (b.y, -b.x)
      const CT mb1 = Cx<CT>::mk(b1.y, -b1.x), mb2 = Cx<CT>::mk(b2.y, -b2.x);
      y[1] = INV ? fs_sub(a1, mb1) : fs_add(a1, mb1);
      y[4] = INV ? fs_add(a1, mb1) : fs_sub(a1, mb1);
      y[2] = INV ? fs_sub(a2, mb2) : fs_add(a2, mb2);
      y[3] = INV ? fs_add(a2, mb2) : fs_sub(a2, mb2);
    }
    const int base = jq * Ns * RX + k;
#pragma unroll
    for (int r = 0; r < RX; ++r) out[base + r * Ns] = y[r];
  }
}

// the whole sub-transform (natural order in and out); returns the buffer holding the result
template <typename CT, bool INV>
__device__ CT* fs_fft(CT* a, CT* b, const FsRadix& p, int nseq, int ls, const CT* __restrict__ tab) {
  int Ns = 1;
  for (int q = 0; q < p.n; ++q) {
    const int R = p.r[q];
    if (R == 4) fs_pass<4, CT, INV>(a, b, p.L, Ns, p.mM[q], p.mN[q], nseq, ls, tab);
    else if (R == 2) fs_pass<2, CT, INV>(a, b, p.L, Ns, p.mM[q], p.mN[q], nseq, ls, tab);
    else fs_pass<5, CT, INV>(a, b, p.L, Ns, p.mM[q], p.mN[q], nseq, ls, tab);
    __syncthreads();
    CT* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// W_D^m for m < D <= 2^20 from three small tables in shared memory:
// W_D^m = top[m >> 12] mid[(m >> 6) & 63] lo[m & 63], with top[a] = W_D^(4096 a),
// mid[b] = W_D^(64 b), lo[c] = W_D^c
constexpr int kFsTwTop = 256;               // 2^20 / 4096
constexpr int kFsTwSmem = 64 + 64 + kFsTwTop;
template <typename CT>
__device__ __forceinline__ CT fs_twD(const CT* tw3, int64_t m) {
  const int mi = (int)m;
  return fs_mul(fs_mul(tw3[128 + (mi >> 12)], tw3[64 + ((mi >> 6) & 63)]), tw3[mi & 63]);
}

// the sub-transform's table (L entries) and the three W_D tables (lo, mid, top: see fs_twD)
// into shared memory
template <typename CT>
__device__ __forceinline__ void fs_stage_tables(CT* tw, CT* tw3, const CT* __restrict__ tab,
                                                int L, const CT* __restrict__ tabD, int D) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = tab[i];
  for (int i = threadIdx.x; i < kFsTwSmem; i += blockDim.x) {
    int64_t e = i < 64 ? i : (i < 128 ? (int64_t)(i - 64) * 64 : (int64_t)(i - 128) * 4096);
    if (e >= D) e = 0;          // beyond the table: never read (m < D)
    tw3[i] = tabD[e];
  }
}

// the two systems of pair p of task t, and whether each takes part
struct FsSys {
  int t, j1, j2;
  int64_t s1, s2;
  bool has2, on1, on2;
};

__device__ __forceinline__ FsSys fs_sys(const FsPairs& pp, int pi, const int* flags) {
  FsSys q;
  q.t = pi / pp.npair;
  const int p = pi - q.t * pp.npair;
  q.has2 = 2 * p + 1 < pp.Rc;
  q.j1 = 2 * p * pp.jstride;
  q.j2 = q.has2 ? (2 * p + 1) * pp.jstride : q.j1;
  q.s1 = (int64_t)q.t * pp.R + q.j1;
  q.s2 = (int64_t)q.t * pp.R + q.j2;
  q.on1 = flags == nullptr || flags[q.s1] != 0;
  q.on2 = q.has2 && (flags == nullptr || flags[q.s2] != 0);
  return q;
}

// ---- pass 1: length-n1 transforms of nb columns, times W_D^{i2 k1} -> Y[k1][i2] -----------
template <typename CT>
__global__ void __launch_bounds__(kFsThreads)
k_fs_cols_fwd(const float* __restrict__ X, CT* __restrict__ Y, const CT* __restrict__ tab1,
              const CT* __restrict__ tabD, FsPlan pl, FsPairs pp, const int* __restrict__ flags,
              const int* __restrict__ task_active) {
  extern __shared__ __align__(16) unsigned char fs_sm[];
  const int nb = sizeof(CT) == sizeof(float2) ? pl.nb32 : pl.nb, lnb = __ffs(nb) - 1;
  const int ls = pl.n1 + 1;
  CT* A = reinterpret_cast<CT*>(fs_sm);
  CT* B = A + nb * ls;
  CT* tw = B + nb * ls;
  CT* tw3 = tw + pl.n1;
  const int pi = blockIdx.x;
  const FsSys q = fs_sys(pp, pi, flags);
  if (task_active != nullptr && task_active[q.t] == 0) return;     // block-uniform
  if (!q.on1 && !q.on2) return;
  fs_stage_tables(tw, tw3, tab1, pl.n1, tabD, pp.D);
  const int c0 = blockIdx.y * nb;
  const float* x1 = X + q.s1 * pp.Dp;
  const float* x2 = X + q.s2 * pp.Dp;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < pl.n1 * nb; idx += blockDim.x) {
    const int i1 = idx >> lnb, cc = idx & (nb - 1);
    const int64_t n = (int64_t)pl.n2 * i1 + c0 + cc;
    A[cc * ls + i1] = Cx<CT>::mk(q.on1 ? x1[n] : 0.f, q.on2 ? x2[n] : 0.f);
  }
  __syncthreads();
  const CT* res = fs_fft<CT, false>(A, B, pl.p1, nb, ls, tw);
  CT* Yp = Y + (int64_t)pi * pp.D;
  for (int idx = threadIdx.x; idx < pl.n1 * nb; idx += blockDim.x) {
    const int k1 = idx >> lnb, cc = idx & (nb - 1), i2 = c0 + cc;
    Yp[(int64_t)k1 * pl.n2 + i2] = fs_mul(res[cc * ls + k1], fs_twD(tw3, (int64_t)i2 * k1));
  }
}

// ---- pass 2: per row k1, transform over i2, mask, inverse transform, conjugate twiddle -----
// SPEC: the rows start from a spectrum spec[t][k] in natural frequency order (b0: only the
// inverse half runs).
template <typename CT, bool SPEC>
__global__ void __launch_bounds__(kFsThreads)
k_fs_rows(CT* __restrict__ Y, const CT* __restrict__ spec, const CT* __restrict__ tab2,
          const CT* __restrict__ tabD, const float* __restrict__ mask, FsPlan pl, FsPairs pp,
          const int* __restrict__ flags, const int* __restrict__ task_active) {
  extern __shared__ __align__(16) unsigned char fs_sm[];
  const int ls = pl.n2 + 1;
  const int nbr = sizeof(CT) == sizeof(float2) ? pl.nbr32 : pl.nbr;
  CT* A = reinterpret_cast<CT*>(fs_sm);
  CT* B = A + nbr * ls;
  CT* tw = B + nbr * ls;
  CT* tw3 = tw + pl.n2;
  const int pi = blockIdx.x;
  const FsSys q = fs_sys(pp, pi, flags);
  if (task_active != nullptr && task_active[q.t] == 0) return;     // block-uniform
  if (!q.on1 && !q.on2) return;
  fs_stage_tables(tw, tw3, tab2, pl.n2, tabD, pp.D);
  const int r0 = blockIdx.y * nbr;
  CT* Yp = Y + (int64_t)pi * pp.D;
  // the last row block may run past n1: its extra rows transform zeros and are not stored
#pragma unroll 4
  for (int idx = threadIdx.x; idx < nbr * pl.n2; idx += blockDim.x) {
    const int rr = fs_div(idx, pl.mn2), i2 = idx - rr * pl.n2, k1 = r0 + rr;
    CT v = Cx<CT>::mk(0, 0);
    if (k1 < pl.n1)
      v = SPEC ? spec[(int64_t)q.t * pp.D + k1 + (int64_t)pl.n1 * i2] : Yp[(int64_t)k1 * pl.n2 + i2];
    A[rr * ls + i2] = v;
  }
  __syncthreads();
  CT* cur = A;
  CT* oth = B;
  if constexpr (!SPEC) {
    cur = fs_fft<CT, false>(A, B, pl.p2, nbr, ls, tw);
    oth = cur == A ? B : A;
    const float* mt = mask + (int64_t)q.t * pp.D;
    for (int idx = threadIdx.x; idx < nbr * pl.n2; idx += blockDim.x) {
      const int rr = fs_div(idx, pl.mn2), k2 = idx - rr * pl.n2, k1 = r0 + rr;
      if (k1 >= pl.n1) continue;
      const typename Cx<CT>::R mk = (typename Cx<CT>::R)mt[k1 + (int64_t)pl.n1 * k2];
      const CT v = cur[rr * ls + k2];
      cur[rr * ls + k2] = Cx<CT>::mk(v.x * mk, v.y * mk);
    }
    __syncthreads();
  }
  const CT* res = fs_fft<CT, true>(cur, oth, pl.p2, nbr, ls, tw);
  for (int idx = threadIdx.x; idx < nbr * pl.n2; idx += blockDim.x) {
    const int rr = fs_div(idx, pl.mn2), i2 = idx - rr * pl.n2, k1 = r0 + rr;
    if (k1 < pl.n1)
      Yp[(int64_t)k1 * pl.n2 + i2] = fs_mulc(res[rr * ls + i2], fs_twD(tw3, (int64_t)i2 * k1));
  }
}

// ---- pass 3: inverse length-n1 transforms of nb columns, then the epilogue -----------------
enum { kFsOp = 0, kFsResidual = 1, kFsB0 = 2 };

struct FsEpi {
  // kFsOp: Z = beta/D z + alpha * V (V the vectors), partial V^T Z per column block
  const float* V;
  float* Z;
  float* part;           // [n2 / nb][S] or null
  const float* alpha;
  int S;
  unsigned long long* opcount;
  // kFsResidual: Rout = B - A X in FP64 (X = V); B = Bext, or b0 (k = 0) / the probe
  const float* Bext;
  const float* b0hi;
  const float* b0lo;
  float* Rout;
  const float* pw;       // sqrt(m) [T*C][Dp] scaling the probes (Jacobi), or null
  int pshare;
  uint64_t seed;
  int64_t em_iter;
  int toff;               // global index of the context's first task (probe counters)
  double beta;
  // kFsB0: b0 = beta Re(F^H y) as an FP32 pair
  float* hi;
  float* lo;
};

template <typename CT, int MODE>
__global__ void __launch_bounds__(kFsThreads)
k_fs_cols_inv(const CT* __restrict__ Y, const CT* __restrict__ tab1, FsPlan pl, FsPairs pp,
              const int* __restrict__ flags, const int* __restrict__ task_active, FsEpi ep) {
  extern __shared__ __align__(16) unsigned char fs_sm[];
  __shared__ double red[2][kFsThreads / 32];
  const int nb = sizeof(CT) == sizeof(float2) ? pl.nb32 : pl.nb, lnb = __ffs(nb) - 1;
  const int ls = pl.n1 + 1;
  CT* A = reinterpret_cast<CT*>(fs_sm);
  CT* B = A + nb * ls;
  CT* tw = B + nb * ls;
  const int pi = blockIdx.x;
  const FsSys q = fs_sys(pp, pi, flags);
  if (task_active != nullptr && task_active[q.t] == 0) return;     // block-uniform
  if (!q.on1 && !q.on2) return;
  for (int i = threadIdx.x; i < pl.n1; i += blockDim.x) tw[i] = tab1[i];
  const int c0 = blockIdx.y * nb;
  const CT* Yp = Y + (int64_t)pi * pp.D;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < pl.n1 * nb; idx += blockDim.x) {
    const int k1 = idx >> lnb, cc = idx & (nb - 1);
    A[cc * ls + k1] = Yp[(int64_t)k1 * pl.n2 + c0 + cc];
  }
  __syncthreads();
  const CT* res = fs_fft<CT, true>(A, B, pl.p1, nb, ls, tw);
  const int D = pp.D, Dp = pp.Dp;
  if constexpr (MODE == kFsOp) {
    const float scale = (float)(ep.beta / (double)D);
    const int c1 = q.j1 / (pp.K + 1), c2 = q.j2 / (pp.K + 1);
    const float* a1 = ep.alpha + (int64_t)c1 * Dp;
    const float* a2 = ep.alpha + (int64_t)c2 * Dp;
    const float* v1 = ep.V + q.s1 * Dp;
    const float* v2 = ep.V + q.s2 * Dp;
    float* z1 = ep.Z + q.s1 * Dp;
    float* z2 = ep.Z + q.s2 * Dp;
    float dot1 = 0.f, dot2 = 0.f;
    for (int idx = threadIdx.x; idx < pl.n1 * nb; idx += blockDim.x) {
      const int i1 = idx >> lnb, cc = idx & (nb - 1);
      const int64_t n = (int64_t)pl.n2 * i1 + c0 + cc;
      const CT zc = res[cc * ls + i1];
      if (q.on1) {
        const float v = v1[n];
        const float z = fmaf(scale, (float)zc.x, a1[n] * v);
        z1[n] = z;
        dot1 = fmaf(v, z, dot1);
      }
      if (q.on2) {
        const float v = v2[n];
        const float z = fmaf(scale, (float)zc.y, a2[n] * v);
        z2[n] = z;
        dot2 = fmaf(v, z, dot2);
      }
    }
    if (ep.part != nullptr) {
      // fixed-order block sums of the two partial inner products
      double d1 = dot1, d2 = dot2;
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) {
        d1 += __shfl_xor_sync(0xffffffffu, d1, m);
        d2 += __shfl_xor_sync(0xffffffffu, d2, m);
      }
      if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = d1;
        red[1][threadIdx.x >> 5] = d2;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < kFsThreads / 32; ++w) {
          t1 += red[0][w];
          t2 += red[1][w];
        }
        if (q.on1) ep.part[(int64_t)blockIdx.y * ep.S + q.s1] = (float)t1;
        if (q.on2) ep.part[(int64_t)blockIdx.y * ep.S + q.s2] = (float)t2;
      }
    }
    const int p = pi - q.t * pp.npair;
    if (ep.opcount != nullptr && p == 0 && blockIdx.y == 0 && threadIdx.x == 0)
      atomicAdd(&ep.opcount[q.t], 1ull);
  } else if constexpr (MODE == kFsResidual) {
    const double scale = ep.beta / (double)D;
    for (int idx = threadIdx.x; idx < pl.n1 * nb; idx += blockDim.x) {
      const int i1 = idx >> lnb, cc = idx & (nb - 1);
      const int64_t n = (int64_t)pl.n2 * i1 + c0 + cc;
      const CT zc = res[cc * ls + i1];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !q.has2) continue;
        const bool on = h == 0 ? q.on1 : q.on2;
        const int64_t s = h == 0 ? q.s1 : q.s2;
        if (!on) {                     // the idle system of a half-active pair
          ep.Rout[s * Dp + n] = 0.f;
          continue;
        }
        const int j = h == 0 ? q.j1 : q.j2;
        const int c = j / (pp.K + 1), k = j - c * (pp.K + 1);
        double b;
        if (ep.Bext != nullptr) {
          b = (double)ep.Bext[s * Dp + n];
        } else if (k == 0) {
          b = (double)ep.b0hi[(int64_t)q.t * Dp + n] + (double)ep.b0lo[(int64_t)q.t * Dp + n];
        } else {
          const uint32_t bits = probe_bits32(ep.seed, ep.em_iter, q.t + ep.toff, probe_cluster(c, ep.pshare),
                                             pp.C, k - 1, (int)(n & ~(int64_t)31));
          b = ((bits >> (n & 31)) & 1u) ? -1.0 : 1.0;
          if (ep.pw != nullptr) b *= (double)ep.pw[((int64_t)q.t * pp.C + c) * Dp + n];
        }
        const double xv = (double)ep.V[s * Dp + n];
        const double z = fma(scale, (double)(h == 0 ? zc.x : zc.y),
                             (double)ep.alpha[(int64_t)c * Dp + n] * xv);
        ep.Rout[s * Dp + n] = (float)(b - z);
      }
    }
  } else {
    // b0 = beta Re(F^H Y) = beta / sqrt(D) Re(sum_k Y_k e^{+2 pi i k n / D})
    const double scale = ep.beta / sqrt((double)D);
    for (int idx = threadIdx.x; idx < pl.n1 * nb; idx += blockDim.x) {
      const int i1 = idx >> lnb, cc = idx & (nb - 1);
      const int64_t n = (int64_t)pl.n2 * i1 + c0 + cc;
      const double b = scale * (double)res[cc * ls + i1].x;
      const float h = (float)b;
      ep.hi[(int64_t)q.t * Dp + n] = h;
      ep.lo[(int64_t)q.t * Dp + n] = (float)(b - (double)h);
    }
  }
}

// the measured coefficients placed at their frequencies: spec[t][freq] = y (FP64)
__global__ void k_fs_scatter(const float2* __restrict__ y, const int* __restrict__ freq,
                             const int64_t* __restrict__ off, double2* spec, int D) {
  const int t = blockIdx.y;
  for (int64_t i = off[t] + blockIdx.x * 256 + threadIdx.x; i < off[t + 1]; i += 256 * gridDim.x)
    spec[(int64_t)t * D + freq[i]] = make_double2((double)y[i].x, (double)y[i].y);
}

// ---- host side ---------------------------------------------------------------------------
struct FsState {
  FsPlan pl;
  float2 *tab1_32, *tab2_32, *tabD_32;
  double2 *tab1_64, *tab2_64, *tabD_64;
  float* mask;        // [T][D] symmetrised mask, natural frequency order
  void* work;         // pair spectra Y: [max(npair, 2) * T][D] double2 (float2 when FP32)
};

int v2of(int64_t x) {
  int a = 0;
  while (x > 0 && x % 2 == 0) {
    x /= 2;
    ++a;
  }
  return a;
}

bool only_2_5(int64_t x) {
  if (x < 1) return false;
  while (x % 2 == 0) x /= 2;
  while (x % 5 == 0) x /= 5;
  return x == 1;
}

uint64_t recip(int d) { return ((uint64_t)1 << 32) / (uint64_t)d + (((uint64_t)1 << 32) % (uint64_t)d != 0); }

FsRadix make_radix(int L) {
  FsRadix p{};
  p.L = L;
  int m = L;
  while (m % 4 == 0 && p.n < kFsMaxRadices) { p.r[p.n++] = 4; m /= 4; }
  while (m % 2 == 0 && p.n < kFsMaxRadices) { p.r[p.n++] = 2; m /= 2; }
  while (m % 5 == 0 && p.n < kFsMaxRadices) { p.r[p.n++] = 5; m /= 5; }
  if (m != 1) {
    p.n = -1;
    return p;
  }
  int Ns = 1;
  for (int q = 0; q < p.n; ++q) {
    p.mM[q] = recip(L / p.r[q]);
    p.mN[q] = recip(Ns);
    Ns *= p.r[q];
  }
  return p;
}

int pow2_share(int n, int cap, int len) {   // largest 2^a dividing n, <= cap, fitting in smem
  int b = 1;
  while (b * 2 <= cap && n % (b * 2) == 0 &&
         (size_t)2 * (b * 2) * (len + 1) * sizeof(double2) <= kFsSmemBudget)
    b *= 2;
  return b;
}

// D = n1 * n2 with both <= 1024 and of the form 2^a 5^b; n2 keeps 16 | n2 so that a column
// block is 16 consecutive floats; the most balanced split, then the shorter column transform
bool make_plan(int D, FsPlan* out) {
  if (D < 128 || D > (1 << 20) || D % 16 != 0 || !only_2_5(D)) return false;
  int best2 = 0;
  for (int n2 = 16; n2 <= kFsMaxLen; ++n2) {
    if (D % n2 != 0 || v2of(n2) < 4 || !only_2_5(n2)) continue;
    const int n1 = D / n2;
    if (n1 < 8 || n1 > kFsMaxLen) continue;
    if (best2 == 0) {
      best2 = n2;
      continue;
    }
    const int b1 = D / best2;
    const int key = n1 > n2 ? n1 : n2, bkey = b1 > best2 ? b1 : best2;
    if (key < bkey || (key == bkey && n1 < b1)) best2 = n2;
  }
  if (best2 == 0) return false;
  FsPlan pl{};
  pl.n2 = best2;
  pl.n1 = D / best2;
  pl.nb = pow2_share(pl.n2, 16, pl.n1);
  // FP32 column passes: 8 columns (32-byte rows) unless the rule below picks another, as long
  // as n2 / nb32 partial sums fit the D / 128 slots
  pl.nb32 = (pl.nb >= 8 && pl.n1 * 8 >= 128) ? 8 : pl.nb;
  pl.nbr = 1;
  while (pl.nbr < 8 && (size_t)2 * (pl.nbr * 2) * (pl.n2 + 1) * sizeof(double2) <= kFsSmemBudget)
    pl.nbr *= 2;
  // FP32 passes: about 2048 complex values per CTA (two 16 KiB buffers), so that several CTAs
  // share an SM; measured best at n2 = 400 (4 rows) and at 128 x 128 (16 rows, 16 columns)
  pl.nbr32 = 1;
  while (pl.nbr32 < 32 && pl.nbr32 < pl.n1 && pl.nbr32 * 2 * pl.n2 <= 2048) pl.nbr32 *= 2;
  {
    int nb = 1;
    while (nb < 16 && pl.n2 % (nb * 2) == 0 && nb * 2 * pl.n1 <= 2048) nb *= 2;
    if ((int64_t)pl.n1 * nb >= 128) pl.nb32 = nb;
  }
  {
    // evaluation switches: FP32 columns per column-pass CTA and rows per row-pass CTA
    const char* v = getenv("CMCS_FS_NB32");
    const int nbv = v ? atoi(v) : 0;
    if (nbv >= 1 && nbv <= 16 && (nbv & (nbv - 1)) == 0 && pl.n2 % nbv == 0 &&
        (int64_t)pl.n1 * nbv >= 128 &&
        (size_t)2 * nbv * (pl.n1 + 1) * sizeof(float2) <= kFsSmemBudget)
      pl.nb32 = nbv;
    const char* r = getenv("CMCS_FS_NBR32");
    const int nr = r ? atoi(r) : 0;
    if (nr >= 1 && nr <= 32 && (size_t)2 * nr * (pl.n2 + 1) * sizeof(float2) <= kFsSmemBudget)
      pl.nbr32 = nr;
  }
  pl.mn2 = recip(pl.n2);
  pl.p1 = make_radix(pl.n1);
  pl.p2 = make_radix(pl.n2);
  if (pl.p1.n < 0 || pl.p2.n < 0) return false;
  if ((int64_t)pl.n1 * pl.nb32 < 128) return false;   // partial sums fit the D/128 slots
  *out = pl;
  return true;
}

int cols_nb(const FsPlan& pl, size_t cs) { return cs == sizeof(float2) ? pl.nb32 : pl.nb; }
// two ping-pong buffers, the sub-transform's table and the three W_D tables
size_t cols_smem(const FsPlan& pl, size_t cs) {
  return (2 * (size_t)cols_nb(pl, cs) * (pl.n1 + 1) + pl.n1 + kFsTwSmem) * cs;
}
size_t rows_smem(const FsPlan& pl, size_t cs) {
  const int nbr = cs == sizeof(float2) ? pl.nbr32 : pl.nbr;
  return (2 * (size_t)nbr * (pl.n2 + 1) + pl.n2 + kFsTwSmem) * cs;
}

template <typename CT>
cudaError_t set_attrs(const FsPlan& pl) {
  const int sc = (int)cols_smem(pl, sizeof(CT)), sr = (int)rows_smem(pl, sizeof(CT));
  cudaError_t e = cudaFuncSetAttribute(k_fs_cols_fwd<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sc);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fs_rows<CT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sr);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fs_rows<CT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sr);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fs_cols_inv<CT, kFsOp>, cudaFuncAttributeMaxDynamicSharedMemorySize, sc);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fs_cols_inv<CT, kFsResidual>, cudaFuncAttributeMaxDynamicSharedMemorySize, sc);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fs_cols_inv<CT, kFsB0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sc);
  return e;
}

FsPairs pairs_of(const Ctx* c, int Rc, int jstride) {
  FsPairs pp;
  pp.R = c->R;
  pp.K = c->K;
  pp.C = c->C;
  pp.Dp = c->Dp;
  pp.D = c->D;
  pp.Rc = Rc;
  pp.jstride = jstride;
  pp.npair = (Rc + 1) / 2;
  return pp;
}

// the three passes for the pairs of pp; SPEC: start at the row pass from spec (b0)
template <typename CT, int MODE, bool SPEC>
cudaError_t run_passes(Ctx* c, const FsPairs& pp, const float* X, const CT* spec,
                       const int* flags, const int* task_active, const FsEpi& ep) {
  const FsState* fs = static_cast<const FsState*>(c->fs);
  const FsPlan& pl = fs->pl;
  const bool f64 = sizeof(CT) == sizeof(double2);
  const CT* tab1 = f64 ? reinterpret_cast<const CT*>(fs->tab1_64) : reinterpret_cast<const CT*>(fs->tab1_32);
  const CT* tab2 = f64 ? reinterpret_cast<const CT*>(fs->tab2_64) : reinterpret_cast<const CT*>(fs->tab2_32);
  const CT* tabD = f64 ? reinterpret_cast<const CT*>(fs->tabD_64) : reinterpret_cast<const CT*>(fs->tabD_32);
  CT* Y = static_cast<CT*>(fs->work);
  const unsigned np = (unsigned)((int64_t)c->T * pp.npair);
  const size_t sc = cols_smem(pl, sizeof(CT)), sr = rows_smem(pl, sizeof(CT));
  if (!SPEC) {
    k_fs_cols_fwd<CT><<<dim3(np, pl.n2 / cols_nb(pl, sizeof(CT))), kFsThreads, sc, c->stream>>>(
        X, Y, tab1, tabD, pl, pp, flags, task_active);
    c->launches += 1;
  }
  const int nbr = f64 ? pl.nbr : pl.nbr32;
  k_fs_rows<CT, SPEC><<<dim3(np, (pl.n1 + nbr - 1) / nbr), kFsThreads, sr, c->stream>>>(
      Y, spec, tab2, tabD, fs->mask, pl, pp, flags, task_active);
  k_fs_cols_inv<CT, MODE><<<dim3(np, pl.n2 / cols_nb(pl, sizeof(CT))), kFsThreads, sc, c->stream>>>(
      Y, tab1, pl, pp, flags, task_active, ep);
  c->launches += 2;
  return cudaGetLastError();
}

}  // namespace

bool dft_large_ok(int D) {
  FsPlan pl;
  return make_plan(D, &pl);
}

int fs_create(Ctx* c, const uint8_t* hmask) {
  FsState* fs = new (std::nothrow) FsState();
  if (fs == nullptr) return 2;
  c->fs = fs;
  if (!make_plan(c->D, &fs->pl)) return 6;
  const FsPlan& pl = fs->pl;
  const int T = c->T, D = c->D;
  const double pi = 3.14159265358979323846;
  auto table = [&](int L, std::vector<float2>& t32, std::vector<double2>& t64) {
    t32.resize((size_t)L);
    t64.resize((size_t)L);
    for (int m = 0; m < L; ++m) {
      const double a = -2.0 * pi * (double)m / (double)L;
      t64[(size_t)m] = make_double2(cos(a), sin(a));
      t32[(size_t)m] = make_float2((float)cos(a), (float)sin(a));
    }
  };
  std::vector<float2> a32, b32, d32;
  std::vector<double2> a64, b64, d64;
  table(pl.n1, a32, a64);
  table(pl.n2, b32, b64);
  table(D, d32, d64);
  std::vector<float> mt((size_t)T * D);
  for (int t = 0; t < T; ++t) {
    const uint8_t* m = hmask + (size_t)t * D;
    for (int k = 0; k < D; ++k)
      mt[(size_t)t * D + k] = 0.5f * (float)((m[k] ? 1 : 0) + (m[(D - k) % D] ? 1 : 0));
  }
  const size_t npair = (size_t)(c->R + 1) / 2;
  const size_t nwork = (npair > 2 ? npair : 2) * (size_t)T * D;
  bool ok = cudaMalloc(reinterpret_cast<void**>(&fs->tab1_32), sizeof(float2) * a32.size()) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&fs->tab2_32), sizeof(float2) * b32.size()) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&fs->tabD_32), sizeof(float2) * d32.size()) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&fs->tab1_64), sizeof(double2) * a64.size()) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&fs->tab2_64), sizeof(double2) * b64.size()) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&fs->tabD_64), sizeof(double2) * d64.size()) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&fs->mask), sizeof(float) * mt.size()) == cudaSuccess &&
            cudaMalloc(&fs->work, sizeof(double2) * nwork) == cudaSuccess;
  if (!ok) return 2;
  ok = cudaMemcpy(fs->tab1_32, a32.data(), sizeof(float2) * a32.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(fs->tab2_32, b32.data(), sizeof(float2) * b32.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(fs->tabD_32, d32.data(), sizeof(float2) * d32.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(fs->tab1_64, a64.data(), sizeof(double2) * a64.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(fs->tab2_64, b64.data(), sizeof(double2) * b64.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(fs->tabD_64, d64.data(), sizeof(double2) * d64.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(fs->mask, mt.data(), sizeof(float) * mt.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) return 3;
  if (set_attrs<float2>(pl) != cudaSuccess || set_attrs<double2>(pl) != cudaSuccess) return 4;
  c->dft_ndt = pl.n2 / pl.nb32;
  return 0;
}

void fs_destroy(Ctx* c) {
  FsState* fs = static_cast<FsState*>(c->fs);
  if (fs == nullptr) return;
  void* ptrs[] = {fs->tab1_32, fs->tab2_32, fs->tabD_32, fs->tab1_64, fs->tab2_64, fs->tabD_64,
                  fs->mask, fs->work};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete fs;
  c->fs = nullptr;
}

// Z = A V for every system (with_dots: the CG operator -- only active systems of active tasks,
// and the partial d^T A d per column block into part)
cudaError_t fs_apply(Ctx* c, const float* V, float* Z, int with_dots) {
  FsEpi ep{};
  ep.V = V;
  ep.Z = Z;
  ep.part = with_dots ? c->part : nullptr;
  ep.alpha = c->alpha;
  ep.S = c->S;
  ep.beta = c->beta;
  ep.opcount = c->prof_on ? reinterpret_cast<unsigned long long*>(c->opcount) : nullptr;
  const FsPairs pp = pairs_of(c, c->R, 1);
  return run_passes<float2, kFsOp, false>(c, pp, V, nullptr, with_dots ? c->active : nullptr,
                                          with_dots ? c->task_active : nullptr, ep);
}

cudaError_t fs_residual(Ctx* c, const float* X, const float* Bext, float* Rout, int all_systems,
                        int means_only) {
  FsEpi ep{};
  ep.V = X;
  ep.alpha = c->alpha;
  ep.S = c->S;
  ep.Bext = Bext;
  ep.b0hi = c->b0hi;
  ep.b0lo = c->b0lo;
  ep.Rout = Rout;
  ep.pw = c->precond ? c->pw : nullptr;
  ep.pshare = c->pshare;
  ep.seed = c->seed;
  ep.em_iter = c->em_iter;
  ep.toff = c->toff;
  ep.beta = c->beta;
  const FsPairs pp = means_only ? pairs_of(c, c->C, c->K + 1) : pairs_of(c, c->R, 1);
  const int* flags = (Bext || all_systems) ? nullptr : c->ractive;
  return run_passes<double2, kFsResidual, false>(c, pp, X, nullptr, flags, nullptr, ep);
}

cudaError_t fs_b0(Ctx* c) {
  FsState* fs = static_cast<FsState*>(c->fs);
  const int64_t TD = (int64_t)c->T * c->D;
  // the spectra sit in the second half of the work buffer; the row pass writes the first
  double2* spec = static_cast<double2*>(fs->work) + TD;
  cudaError_t e = cudaMemsetAsync(spec, 0, sizeof(double2) * TD, c->stream);
  if (e != cudaSuccess) return e;
  k_fs_scatter<<<dim3(64, c->T), 256, 0, c->stream>>>(reinterpret_cast<const float2*>(c->dft_y),
                                                     c->dft_freq, c->dft_off, spec, c->D);
  c->launches += 1;
  FsEpi ep{};
  ep.beta = c->beta;
  ep.hi = c->b0hi;
  ep.lo = c->b0lo;
  FsPairs pp = pairs_of(c, 1, 1);     // one vector per task
  pp.R = 1;
  return run_passes<double2, kFsB0, true>(c, pp, nullptr, spec, nullptr, nullptr, ep);
}

}  // namespace cmcs
