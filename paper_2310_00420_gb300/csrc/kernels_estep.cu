// E-step tail and M-step: Lanczos log quadrature (Eqs. 9-11), ell (Eq. 3), responsibilities
// by an FP64 log-sum-exp (Eq. 3), hard assignments (Alg. 2), and the alpha update (Eq. 5).
#include <float.h>
#include <math.h>
#include <stdlib.h>

#include "cmcs_internal.cuh"

namespace cmcs {

namespace {

template <typename Tv>
__device__ __forceinline__ Tv block_sum256(Tv v, Tv* sh) {
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

// Eigenvalues lambda_u and first eigenvector components S_{u,1} of the U x U Lanczos matrix
// of Eq. 9, by implicit-shift symmetric QR steps with the Wilkinson shift on the trailing
// unreduced block (Golub & Van Loan, "Matrix Computations", Sec. 8.3), accumulating only the
// first row of the rotation product (the Golub-Welsch observation).  Returns
// sum_u S_{u,1}^2 log lambda_u; sets *fail if the sweep cap is hit or an eigenvalue is <= 0.
// The diagonal a, the off-diagonal b and the first row z of the rotations live in shared
// memory at stride `st` (the thread's own column of its block's arrays): the QR sweep is a
// chain of dependent FP64 operations, and shared memory keeps each step's loads short where
// per-thread local arrays of this size would fall out of L1.
__device__ double lanczos_log_quad(const float* __restrict__ g, const float* __restrict__ xi,
                                   int U, double* a, double* b, double* z, int st, int* fail) {
  for (int i = 0; i < U; ++i) {
    const double gi = (double)g[i];
    a[i * st] = 1.0 / gi + (i > 0 ? (double)xi[i - 1] / (double)g[i - 1] : 0.0);
    b[i * st] = (i + 1 < U) ? sqrt((double)xi[i]) / gi : 0.0;
    z[i * st] = (i == 0) ? 1.0 : 0.0;
  }
  const double eps = DBL_EPSILON;
  int m = U - 1;
  int iters = 0;
  const int max_iters = 60 * U + 60;
  while (m > 0) {
    if (fabs(b[(m - 1) * st]) <= eps * (fabs(a[(m - 1) * st]) + fabs(a[m * st]))) {
      b[(m - 1) * st] = 0.0;
      --m;
      continue;
    }
    int l = m - 1;
    while (l > 0 && fabs(b[(l - 1) * st]) > eps * (fabs(a[(l - 1) * st]) + fabs(a[l * st]))) --l;
    if (l > 0) b[(l - 1) * st] = 0.0;
    if (++iters > max_iters) {
      *fail = 1;
      break;
    }
    // Wilkinson shift: eigenvalue of the trailing 2x2 block closer to a[m]
    const double dd = 0.5 * (a[(m - 1) * st] - a[m * st]);
    const double bm = b[(m - 1) * st];
    // entries of these matrices lie within about 1e-12 .. 1e12, far from overflow, so the
    // plain square root replaces the (slower) scaled hypot
    const double den = dd + copysign(sqrt(dd * dd + bm * bm), dd);
    const double mu = a[m * st] - bm * bm / den;
    double x = a[l * st] - mu, y = b[l * st];
    // the chase carries a[k], b[k] and z[k] in registers from one rotation to the next
    double ak = a[l * st], bk = b[l * st], zk = z[l * st];
    for (int k = l; k < m; ++k) {
      // r = sqrt(x^2 + y^2) and 1 / r: a single-precision reciprocal square root refined by two
      // Newton-Raphson steps for 1 / sqrt(q) (each y <- y (3 - q y^2) / 2 doubles the correct
      // bits: 24 -> 48 -> beyond double precision), in place of a square root and two
      // divisions per rotation.  The seed needs q inside single precision's normal range;
      // outside it (the last rotations of a converging block can have q far below 1e-38)
      // the square root and division are taken in double precision.
      const double q = x * x + y * y;
      double c = 1.0, s = 0.0, r = 0.0;
      if (q > 1e-30 && q < 1e30) {
        double ir = (double)rsqrtf((float)q);
        ir = ir * (1.5 - 0.5 * q * ir * ir);
        ir = ir * (1.5 - 0.5 * q * ir * ir);
        r = q * ir;
        c = x * ir;
        s = -y * ir;
      } else if (q > 0.0) {
        r = sqrt(q);
        c = x / r;
        s = -y / r;
      }
      if (k > l) b[(k - 1) * st] = r;
      const double ak1 = a[(k + 1) * st];
      const double nak = c * c * ak - 2.0 * c * s * bk + s * s * ak1;
      const double nak1 = s * s * ak + 2.0 * c * s * bk + c * c * ak1;
      const double nbk = c * s * (ak - ak1) + (c * c - s * s) * bk;
      a[k * st] = nak;
      const double zk1 = z[(k + 1) * st];
      z[k * st] = c * zk - s * zk1;
      zk = s * zk + c * zk1;
      ak = nak1;
      bk = nbk;
      if (k + 1 < m) {
        const double bk1 = b[(k + 1) * st];
        const double bulge = -s * bk1;
        x = nbk;
        y = bulge;
        b[k * st] = nbk;
        bk = c * bk1;                      // b[k + 1] for the next rotation
      } else {
        b[k * st] = nbk;
      }
    }
    a[m * st] = ak;
    z[m * st] = zk;
  }
  double sum = 0.0;
  for (int i = 0; i < U; ++i) {
    const double ai = a[i * st], zi = z[i * st];
    if (!(ai > 0.0)) *fail = 1;
    sum += zi * zi * log(ai);
  }
  return sum;
}

}  // namespace

// k_quad: one Lanczos matrix per thread, NT threads per block, arrays of 3 UB doubles per
// thread in shared memory; a grid smaller than the matrix count loops over them
template <int UB, int NT>
__global__ void __launch_bounds__(NT)
k_quad(const float* __restrict__ gam, const float* __restrict__ xi, const int* __restrict__ steps,
       int nsys, int ld, double* out, int* status) {
  extern __shared__ double qsm[];                 // [3][UB][NT]
  double* a = qsm + threadIdx.x;
  double* b = a + UB * NT;
  double* z = b + UB * NT;
  for (int i = blockIdx.x * NT + threadIdx.x; i < nsys; i += gridDim.x * NT) {
    const int U = steps[i];
    if (U <= 0) {
      out[i] = 0.0;
      continue;
    }
    if (U > UB || U > ld) {
      atomicOr(status, 2);
      out[i] = 0.0;
      continue;
    }
    int fail = 0;
    out[i] = lanczos_log_quad(gam + (int64_t)i * ld, xi + (int64_t)i * ld, U, a, b, z, NT, &fail);
    if (fail) atomicOr(status, 1);
  }
}

// the same with the arrays in per-thread local memory (no shared memory: the blocks fit beside
// kernels that hold most of an SM's shared memory)
template <int UB>
__global__ void __launch_bounds__(32)
k_quad_local(const float* __restrict__ gam, const float* __restrict__ xi, const int* __restrict__ steps,
             int nsys, int ld, double* out, int* status) {
  double a[UB], b[UB], z[UB];
  for (int i = blockIdx.x * 32 + threadIdx.x; i < nsys; i += gridDim.x * 32) {
    const int U = steps[i];
    if (U <= 0) {
      out[i] = 0.0;
      continue;
    }
    if (U > UB || U > ld) {
      atomicOr(status, 2);
      out[i] = 0.0;
      continue;
    }
    int fail = 0;
    out[i] = lanczos_log_quad(gam + (int64_t)i * ld, xi + (int64_t)i * ld, U, a, b, z, 1, &fail);
    if (fail) atomicOr(status, 1);
  }
}

template <int UB>
cudaError_t launch_quad_local(const float* gam, const float* xi, const int* steps, int nsys, int ld,
                              double* out, int* status, cudaStream_t st, int max_blocks) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_quad_local<UB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int grid = (nsys + 31) / 32;
  if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
  k_quad_local<UB><<<grid, 32, 0, st>>>(gam, xi, steps, nsys, ld, out, status);
  return cudaGetLastError();
}

template <int UB, int NT>
cudaError_t launch_quad(const float* gam, const float* xi, const int* steps, int nsys, int ld,
                        double* out, int* status, cudaStream_t st, int max_blocks) {
  const size_t smem = sizeof(double) * 3 * UB * NT;
  static bool attr = false;                       // set once per kernel instance
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_quad<UB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    // an SM that takes a block of this kernel keeps its whole shared memory available, so the
    // tensor-core kernels running meanwhile can still be placed beside it
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_quad<UB, NT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int grid = (nsys + NT - 1) / NT;
  if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
  k_quad<UB, NT><<<grid, NT, smem, st>>>(gam, xi, steps, nsys, ld, out, status);
  return cudaGetLastError();
}

template <int NT>
cudaError_t launch_quad_nt(const float* gam, const float* xi, const int* steps, int nsys, int ld,
                           double* out, int* status, cudaStream_t st, int max_blocks = 0) {
  if (ld <= 64) return launch_quad<64, NT>(gam, xi, steps, nsys, ld, out, status, st, max_blocks);
  if (ld <= 128) return launch_quad<128, NT>(gam, xi, steps, nsys, ld, out, status, st, max_blocks);
  if (ld <= 256) return launch_quad<256, NT>(gam, xi, steps, nsys, ld, out, status, st, max_blocks);
  if (ld <= 512)
    return launch_quad<512, (NT < 16 ? NT : 16)>(gam, xi, steps, nsys, ld, out, status, st, max_blocks);
  return cudaErrorInvalidValue;
}

cudaError_t launch_quadrature(const float* gam, const float* xi, const int* steps, int nsys,
                              int ld, double* out, int* status, cudaStream_t st) {
  if (nsys <= 0) return cudaSuccess;
  static int nt = -1;                             // evaluation switch CMCS_QUAD_NT: 4, 8, 16, 32
  if (nt < 0) {
    const char* v = getenv("CMCS_QUAD_NT");
    nt = v ? atoi(v) : 32;
  }
  switch (nt) {
    case 4: return launch_quad_nt<4>(gam, xi, steps, nsys, ld, out, status, st);
    case 16: return launch_quad_nt<16>(gam, xi, steps, nsys, ld, out, status, st);
    case 8: return launch_quad_nt<8>(gam, xi, steps, nsys, ld, out, status, st);
    default: return launch_quad_nt<32>(gam, xi, steps, nsys, ld, out, status, st);
  }
}

// In the E-step the eigen step runs on a side stream beside the refinement, whose tensor-core
// kernels hold most of each SM's shared memory.  There it uses the local-memory kernel, with the
// SMs it lands on kept at their full shared-memory carve-out, so it fits beside them: the
// shared-memory kernel (96 KiB per block) made the first refinement residual wait for it.
// CMCS_QUAD_SIDE=0 (evaluation switch) launches the shared-memory kernel instead.
cudaError_t launch_quadrature_ctx(Ctx* c, cudaStream_t st) {
  c->launches += 1;
  static int side = -1;
  if (side < 0) {
    const char* v = getenv("CMCS_QUAD_SIDE");
    side = v ? atoi(v) != 0 : 1;
  }
  const int nsys = c->T * c->C * c->K;
  if (side && nsys > 0 && c->U <= 64)
    return launch_quad_local<64>(c->gam, c->xi, c->psteps, nsys, c->U, c->quad, &c->counters[2], st, 0);
  if (side && nsys > 0 && c->U <= 128)
    return launch_quad_local<128>(c->gam, c->xi, c->psteps, nsys, c->U, c->quad, &c->counters[2], st, 0);
  return launch_quadrature(c->gam, c->xi, c->psteps, nsys, c->U, c->quad, &c->counters[2], st);
}

// ---- ell_tc = nu + sum_d log alpha_cd + b0^T mu (Eq. 3), nu from Eq. 11 ------------------
__global__ void __launch_bounds__(256)
k_ell(const float* __restrict__ xacc, const float* __restrict__ b0hi,
      const float* __restrict__ b0lo, const double* __restrict__ quad,
      const double* __restrict__ sumlogalpha, const float* __restrict__ rmu, double* logdet,
      double* ell, int R, int K, int C, int Dp, int D, const double* __restrict__ sumlogm) {
  __shared__ double sh[33];
  const int tc = blockIdx.x, t = tc / C, c = tc % C;
  const int64_t off = ((int64_t)t * R + (int64_t)c * (K + 1)) * Dp;
  const float* mu = xacc + off;
  double acc = 0.0;
  for (int d = threadIdx.x; d < D; d += 256) {
    const double m = (double)mu[d];
    acc += ((double)b0hi[(int64_t)t * Dp + d] + (double)b0lo[(int64_t)t * Dp + d]) * m;
    if (rmu != nullptr) acc += m * (double)rmu[off + d];    // + mu^T (b0 - A mu)
  }
  const double b0mu = block_sum256(acc, sh);
  if (threadIdx.x == 0) {
    double qs = 0.0;
    for (int k = 0; k < K; ++k) qs += quad[(int64_t)tc * K + k];
    // Jacobi-preconditioned CG: the quadrature is of M^-1/2 A M^-1/2, and log det A adds
    // log det M = sum_d log m_d
    const double nu = -((double)D / (double)K) * qs - (sumlogm != nullptr ? sumlogm[tc] : 0.0);
    logdet[tc] = nu;
    ell[tc] = nu + sumlogalpha[c] + b0mu;
  }
}

// ---- q_t = softmax_c(ell_tc / 2 + log pi_c), L(theta), a_t = argmax_c q_tc --------------
__global__ void __launch_bounds__(256)
k_softmax(const double* __restrict__ ell, const double* __restrict__ logpi,
          const double* __restrict__ tconst, double* q, int* assign, double* stats,
          double* lltask, int* status, int T, int C) {
  __shared__ double sh[33];
  __shared__ double smin[256];
  double ll = 0.0, mn = 1.0;
  for (int t = threadIdx.x; t < T; t += 256) {
    double mx = -INFINITY;
    int arg = 0;
    for (int c = 0; c < C; ++c) {
      const double z = 0.5 * ell[(int64_t)t * C + c] + logpi[c];
      if (!isfinite(z)) atomicOr(status, 4);
      if (z > mx) {
        mx = z;
        arg = c;
      }
    }
    double se = 0.0;
    for (int c = 0; c < C; ++c) se += exp(0.5 * ell[(int64_t)t * C + c] + logpi[c] - mx);
    double best2 = 0.0;
    for (int c = 0; c < C; ++c) {
      const double qc = exp(0.5 * ell[(int64_t)t * C + c] + logpi[c] - mx) / se;
      q[(int64_t)t * C + c] = qc;
      if (c != arg && qc > best2) best2 = qc;
    }
    assign[t] = arg;
    const double margin = q[(int64_t)t * C + arg] - best2;
    mn = fmin(mn, margin);
    const double lt = mx + log(se) - tconst[t];   // log sum_c pi_c p(y_t | alpha_c)
    lltask[t] = lt;
    ll += lt;
  }
  const double tot = block_sum256(ll, sh);
  smin[threadIdx.x] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 1.0;
    for (int i = 0; i < 256; ++i) m = fmin(m, smin[i]);
    stats[0] = tot / (double)T;
    stats[1] = m;
  }
}

cudaError_t launch_ell_softmax(Ctx* c, const float* rmu) {
  c->launches += 2;
  k_ell<<<c->T * c->C, 256, 0, c->stream>>>(c->xacc, c->b0hi, c->b0lo, c->quad, c->sumlogalpha,
                                            rmu, c->logdet, c->ell, c->R, c->K, c->C, c->Dp, c->D,
                                            c->precond ? c->sumlogm : nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_softmax<<<1, 256, 0, c->stream>>>(c->ell, c->logpi, c->tconst, c->q, c->assign, c->stats,
                                      c->lltask, &c->counters[2], c->T, c->C);
  return cudaGetLastError();
}

// ---- M-step, Eq. 5 with s for diag Sigma, split into per-task terms and their ordered sum ---
// Row t of the term matrix (W = C (D + 1) + 1 doubles): q_tc at c (D + 1), q_tc max(mu_tcd^2 +
// s_tcd, 0) at c (D + 1) + 1 + d, and log sum_c pi_c p(y_t | alpha_c) at C (D + 1).  The
// M-step sums the rows of all tasks of the problem in task order, so contexts that each hold a
// range of tasks (one per GPU) reach the same alpha bit for bit as one context holding them all.
__global__ void __launch_bounds__(256)
k_mstep_terms(const float* __restrict__ xacc, const float* __restrict__ sest,
              const double* __restrict__ q, const double* __restrict__ lltask,
              double* __restrict__ terms, int C, int R, int K, int Dp, int D) {
  const int t = blockIdx.y / C, c = blockIdx.y % C;
  const int64_t W = (int64_t)C * (D + 1) + 1;
  double* row = terms + (int64_t)t * W;
  const double qt = q[(int64_t)t * C + c];
  const float* mu = xacc + ((int64_t)t * R + (int64_t)c * (K + 1)) * Dp;
  const float* sv = sest + ((int64_t)t * C + c) * Dp;
  for (int d = blockIdx.x * 256 + threadIdx.x; d < D; d += gridDim.x * 256) {
    const double m = (double)mu[d];
    const double f = fmax(__fma_rn(m, m, (double)sv[d]), 0.0);
    row[(int64_t)c * (D + 1) + 1 + d] = __dmul_rn(qt, f);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    row[(int64_t)c * (D + 1)] = qt;
    if (c == 0) row[(int64_t)C * (D + 1)] = lltask[t];
  }
}

cudaError_t launch_mstep_terms(Ctx* c) {
  c->launches += 1;
  int bx = (c->D + 255) / 256;
  if (bx > 64) bx = 64;
  dim3 grid(bx, c->T * c->C);
  k_mstep_terms<<<grid, 256, 0, c->stream>>>(c->xacc, c->sest, c->q, c->lltask,
                                             c->mterms + (int64_t)c->toff * c->mterm_w, c->C, c->R,
                                             c->K, c->Dp, c->D);
  return cudaGetLastError();
}

// alpha_cd = sum_t q_tc / sum_t q_tc max(mu^2 + s, 0) over the T_total rows in task order
// (one thread per (c, d): reads of one row are coalesced across d), clamped; an empty cluster
// (sum_t q_tc < 1e-300) keeps its alpha
__global__ void __launch_bounds__(256)
k_mstep_apply(const double* __restrict__ terms, float* alpha, int Ttot, int C, int Dp, int D,
              double amin, double amax) {
  const int c = blockIdx.y;
  const int d = blockIdx.x * 256 + threadIdx.x;
  if (d >= Dp) return;
  if (d >= D) {
    alpha[(int64_t)c * Dp + d] = 1.0f;
    return;
  }
  const int64_t W = (int64_t)C * (D + 1) + 1;
  const double* col = terms + (int64_t)c * (D + 1);
  double num = 0.0, den = 0.0;
  for (int t = 0; t < Ttot; ++t) {
    num = __dadd_rn(num, col[(int64_t)t * W]);
    den = __dadd_rn(den, col[(int64_t)t * W + 1 + d]);
  }
  if (num < 1e-300) return;
  double a = (den <= num / amax) ? amax : num / den;
  a = fmin(fmax(a, amin), amax);
  alpha[(int64_t)c * Dp + d] = (float)a;
}

// L(theta) = (1/T_total) sum_t ll_t in task order, and (learned priors) pi_c = max((1/T_total)
// sum_t q_tc, 1e-300) renormalised: the maximiser of sum_tc q_tc log pi_c over the simplex,
// the floor keeps log pi finite
__global__ void k_mstep_scalars(const double* __restrict__ terms, double* stats, double* pi,
                                double* logpi, int Ttot, int C, int D, int learn_pi) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t W = (int64_t)C * (D + 1) + 1;
  double ll = 0.0;
  for (int t = 0; t < Ttot; ++t) ll = __dadd_rn(ll, terms[(int64_t)t * W + (int64_t)C * (D + 1)]);
  stats[0] = ll / (double)Ttot;
  if (!learn_pi) return;
  double tot = 0.0;
  for (int c = 0; c < C; ++c) {
    double sq = 0.0;
    for (int t = 0; t < Ttot; ++t) sq = __dadd_rn(sq, terms[(int64_t)t * W + (int64_t)c * (D + 1)]);
    pi[c] = fmax(sq / (double)Ttot, 1e-300);
    tot += pi[c];
  }
  for (int c = 0; c < C; ++c) {
    const double v = pi[c] / tot;
    pi[c] = v;
    logpi[c] = log(v);
  }
}

cudaError_t launch_mstep_apply(Ctx* c) {
  c->launches += 2;
  dim3 grid((c->Dp + 255) / 256, c->C);
  k_mstep_apply<<<grid, 256, 0, c->stream>>>(c->mterms, c->alpha, c->T_total, c->C, c->Dp, c->D,
                                             c->alpha_min, c->alpha_max);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mstep_scalars<<<1, 32, 0, c->stream>>>(c->mterms, c->stats, c->pi, c->logpi, c->T_total, c->C,
                                           c->D, c->learn_pi);
  return cudaGetLastError();
}

}  // namespace cmcs
