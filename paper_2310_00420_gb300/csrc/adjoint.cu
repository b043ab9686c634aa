// Gradients of the posterior means mu_tc = A_tc^-1 b_t (Eq. 3) with respect to y_t, alpha_c and
// Phi_t, given lambda_tc = A_tc^-1 g_tc for g = dL/dmu (the adjoint system, same symmetric
// operator).  From d mu = A^-1 (d b - d A mu) with b = beta Phi^T y and
// A = beta Phi^T Phi + diag(alpha):
//   dL/dy_t     = beta sum_c Phi_t lambda_tc
//   dL/dalpha_c = - sum_t lambda_tc * mu_tc
//   dL/dPhi_t   = beta sum_c [ (y_t - Phi_t mu_tc) lambda_tc^T - (Phi_t lambda_tc) mu_tc^T ]
// The paper has no adjoint; these follow from its Eq. 3 by differentiation.
#include "cmcs_internal.cuh"

namespace cmcs {

// dy[orow_t + n] = beta sum_c Phi_t lambda_tc [n], with Phi lambda as a compensated pair
// (Wl + Wl_lo) in the pass-1 layout with C columns per task.  lambda = A^-1 g has large
// components in the null space of Phi_t, which Phi_t cancels: a plain FP32 product would keep
// few correct digits of the (much smaller) result, so both parts are summed in FP64.
__global__ void k_adj_dy(const float* __restrict__ Wl, const float* __restrict__ Wl_lo,
                         const int* __restrict__ tile_task, const int64_t* __restrict__ drow,
                         const int64_t* __restrict__ dN, const int64_t* __restrict__ orow, float* dy,
                         int64_t rows, int C, double beta) {
  const int64_t row = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (row >= rows) return;
  const int t = tile_task[row / 128];
  const int64_t rbeg = drow[t], Np = drow[t + 1] - rbeg, n = row - rbeg;
  if (n >= dN[t]) return;
  double acc = 0.0;
  for (int c = 0; c < C; ++c) {
    const int64_t i = rbeg * C + (int64_t)c * Np + n;
    acc += (double)Wl[i] + (double)Wl_lo[i];
  }
  dy[orow[t] + n] = (float)(beta * acc);
}

// dalpha[c][d] = - sum_t lambda_tc[d] mu_tc[d]
__global__ void k_adj_dalpha(const float* __restrict__ lam, const float* __restrict__ mu,
                             float* dalpha, int T, int C, int R, int K, int Dp, int D) {
  const int c = blockIdx.y;
  const int d = blockIdx.x * 256 + threadIdx.x;
  if (d >= Dp) return;
  float acc = 0.f;
  if (d < D)
    for (int t = 0; t < T; ++t)
      acc = fmaf(lam[((int64_t)t * C + c) * Dp + d],
                 mu[((int64_t)t * R + (int64_t)c * (K + 1)) * Dp + d], acc);
  dalpha[(int64_t)c * Dp + d] = -acc;
}

// dPhi rows of tasks t0..t1-1 in the caller's unpadded layout, row index shifted by out_base
// The row terms y_n - (Phi mu)_n and (Phi lambda)_n come from compensated pairs and are
// rounded to FP32 once, after the cancellation.
__global__ void k_adj_dphi(const float* __restrict__ lam, const float* __restrict__ mu,
                           const float* __restrict__ Wl, const float* __restrict__ Wl_lo,
                           const float* __restrict__ Wm, const float* __restrict__ Wm_lo,
                           const float* __restrict__ y, const int* __restrict__ tile_task,
                           const int64_t* __restrict__ drow, const int64_t* __restrict__ dN,
                           const int64_t* __restrict__ orow, float* out, int64_t row_lo,
                           int64_t row_hi, int64_t out_base, int C, int R, int K, int Dp, int D,
                           float beta) {
  const int d = blockIdx.x * 256 + threadIdx.x;
  for (int64_t row = row_lo + blockIdx.y; row < row_hi; row += gridDim.y) {
    const int t = tile_task[row / 128];
    const int64_t rbeg = drow[t], Np = drow[t + 1] - rbeg, n = row - rbeg;
    if (n >= dN[t] || d >= D) continue;
    const float yn = y[row];
    float acc = 0.f;
    for (int c = 0; c < C; ++c) {
      const int64_t i = rbeg * C + (int64_t)c * Np + n;
      const float res = (float)(((double)yn - (double)Wm[i]) - (double)Wm_lo[i]);
      const float wl = (float)((double)Wl[i] + (double)Wl_lo[i]);
      const float l = lam[((int64_t)t * C + c) * Dp + d];
      const float m = mu[((int64_t)t * R + (int64_t)c * (K + 1)) * Dp + d];
      acc = fmaf(res, l, acc);
      acc = fmaf(-wl, m, acc);
    }
    out[(orow[t] + n - out_base) * D + d] = beta * acc;
  }
}

cudaError_t launch_adj_dy(Ctx* c, const float* Wl, const float* Wl_lo, float* dy) {
  c->launches += 1;
  k_adj_dy<<<(unsigned)((c->rows_total + 255) / 256), 256, 0, c->stream>>>(
      Wl, Wl_lo, c->tile_task, c->drow, c->dN, c->dorow, dy, c->rows_total, c->C, c->beta);
  return cudaGetLastError();
}

cudaError_t launch_adj_dalpha(Ctx* c, const float* lam, float* dalpha) {
  c->launches += 1;
  dim3 grid((c->Dp + 255) / 256, c->C);
  k_adj_dalpha<<<grid, 256, 0, c->stream>>>(lam, c->xacc, dalpha, c->T, c->C, c->R, c->K, c->Dp,
                                            c->D);
  return cudaGetLastError();
}

cudaError_t launch_adj_dphi(Ctx* c, const float* lam, const float* Wl, const float* Wl_lo,
                            const float* Wm, const float* Wm_lo, float* out, int64_t lo,
                            int64_t hi, int64_t out_row_base) {
  c->launches += 1;
  const int64_t nrows = hi - lo;
  if (nrows <= 0) return cudaSuccess;
  dim3 grid((c->D + 255) / 256, (unsigned)(nrows < 65535 ? nrows : 65535));
  k_adj_dphi<<<grid, 256, 0, c->stream>>>(lam, c->xacc, Wl, Wl_lo, Wm, Wm_lo, c->y, c->tile_task,
                                          c->drow, c->dN,
                                          c->dorow, out, lo, hi, out_row_base, c->C, c->R, c->K,
                                          c->Dp, c->D, (float)c->beta);
  return cudaGetLastError();
}

}  // namespace cmcs
