// Internal declarations shared by the translation units of libcmcs.so.
//
// Device memory layout (all owned by the context, sizes for the plain-scale workload
// T=32, C=4, D=8192, N=2048, K=32 in brackets):
//   D_pad  = D rounded up to 128; padded coordinates carry alpha = 1, zero Phi columns, zero
//            right-hand sides and zero probes, so they never enter a Krylov space.
//   Np_t   = N_t rounded up to 128; padded rows of Phi_t and y_t are zero (Phi^T Phi and
//            Phi^T y are unchanged).
//   phi    float [sum_t Np_t][D_pad]              Phi, row-major          [2 GiB]
//   R      = C*(K+1) right-hand sides per task; system sys = t*R + j, j = c*(K+1) + k,
//            k = 0 the posterior-mean system, k >= 1 the probe p_{t,c,k}.
//   S      = T*R systems                                                   [4224]
//   x, r, d, ad, xacc  float [S][D_pad]  CG state of Alg. 1 and the refined solution
//   w, wlo float [sum_t R*Np_t]           Phi V (and its low part for the residual)
//   b0hi, b0lo float [T][D_pad]           beta Phi^T y as an unevaluated sum hi + lo
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cmcs.h"

namespace cmcs {

constexpr int kDAlign = 128;      // padding of D
constexpr int kNAlign = 128;      // padding of N_t
constexpr int kUpdThreads = 256;  // threads of the per-system CG kernels
constexpr int kProfEvents = 8192; // timed operator applications per E-step

// ---- Philox-4x32-10 (Salmon et al., SC'11, Sec. 5) ------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    uint64_t p0 = (uint64_t)M0 * c.x;
    uint64_t p1 = (uint64_t)M1 * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

__host__ __device__ inline uint32_t pick_word(const U4& w, int i) {
  return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
}

// Probe counter: (d >> 7, k, t*C + c, (em_iter << 4) | 1); sign from bit d & 31 of word
// (d >> 5) & 3; bit 0 -> +1.  k is 0-based (probe k+1 of the paper).
constexpr uint32_t kTagProbe = 1u;
constexpr uint32_t kTagAlpha = 2u;

__device__ inline uint32_t probe_bits32(uint64_t seed, int64_t em_iter, int t, int c, int C,
                                        int k, int d_base /* multiple of 32 */) {
  U4 ctr{(uint32_t)(d_base >> 7), (uint32_t)k, (uint32_t)(t * C + c),
         (uint32_t)(((uint64_t)em_iter << 4) | kTagProbe)};
  U4 w = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
  return pick_word(w, (d_base >> 5) & 3);
}

// cluster index the probes of cluster c are drawn for: c, or 0 when probes are shared
__host__ __device__ inline int probe_cluster(int c, int pshare) { return pshare ? 0 : c; }

// ---- context --------------------------------------------------------------------------
struct Ctx {
  // configuration
  int T, C, D, K, R, S, Dp, U;    // U = cg_max_iter
  double beta, cg_tol, refine_tol, alpha_min, alpha_max;
  int precision, refine_max;
  int learn_pi;      // each M-step also sets pi_c = max(mean_t q_tc, 1e-300), renormalised
  int pshare;        // probes shared across clusters: p_{t,c,k} = p_{t,0,k}
  int precond;       // Jacobi-preconditioned CG (buffers colnorm, pminv, pw, sumlogm)
  int warm_start;    // mean systems start from the previous E-step's means
  int have_prev;     // xacc holds the means of an earlier E-step of this problem
  uint64_t seed;
  int64_t em_iter;
  int toff;          // global index of this context's first task (keys its probes)
  int T_total;       // tasks of the whole problem (T unless the tasks are split over contexts)
  int mterm_w;       // doubles per row of the M-step terms, C (D + 1) + 1
  cudaStream_t stream;
  int own_stream;      // the context created its stream (caller passed NULL)
  cudaStream_t side;   // runs the Lanczos eigen step while refinement proceeds on stream
  cudaEvent_t ev_fork, ev_join;
  // captured CG chunks: [record][profiling]
  // captured CG chunks: [record][cap in force][profiling]
  cudaGraphExec_t graph[2][2][2];
  int64_t graph_launches;  // kernels in one captured chunk
  int graph_failed[2][2][2];  // capture of that variant failed: use direct launches
  int refine_steps;        // step cap of the refinement sweeps' CG solves
  int chunk;               // CG steps per host poll (and per captured graph)
  int capsel;              // cap in force: 0 cg_max_iter (first solves), 1 refine_steps
  int capturing;           // a chunk is being captured
  int* stall_flag;         // device int, test hook of the bounded-wait path (cmcs_test_stall)
  int device;
  int sm_count;

  // host copies
  int64_t* hN;       // [T]
  int64_t* hNp;      // [T]
  int64_t* hrow;     // [T+1] padded row offsets
  double* hpi;       // [C]
  int64_t rows_total;

  // device buffers
  float* phi;        // [rows_total][Dp]
  float* y;          // [rows_total]
  int64_t* drow;     // [T+1]
  int64_t* dN;       // [T] unpadded N_t
  int64_t* dorow;    // [T+1] unpadded row offsets (caller's layout)
  int64_t* horow;    // host copy
  // adjoint work buffers: right-hand side and solution [T*C][Dp], Phi lambda and Phi mu
  // [C * rows_total], dy [sum N_t], dalpha [C][Dp]
  float *adj_g, *adj_x, *adj_wl, *adj_wm, *adj_wl_lo, *adj_wm_lo, *adj_dy, *adj_da;
  int* tile_task;    // [rows_total / 128] task owning each 128-row tile of phi
  int tn_plain, tn_ds; // operator tile widths (0: chosen from R)
  int per_task;        // 1: launch the operator once per task (comparison schedule)
  int use_graphs;      // 1: replay the CG step chunks from captured CUDA graphs
  int tuned;           // operator variant the autotuner chose (TN or pipeline stages), 0: none
  float *b0hi, *b0lo;  // [T][Dp]
  float* alpha;        // [C][Dp]
  double* sumlogalpha; // [C]
  double* logpi;       // [C]
  double* pi;          // [C] priors in force
  float* colnorm;      // [T][Dp] beta-free diagonal of Phi_t^T Phi_t (precond only)
  float *pminv, *pw;   // [T*C][Dp] 1/m and sqrt(m), m = beta colnorm + alpha_c (precond only)
  double* sumlogm;     // [T*C] sum_{d<D} log m_d (precond only)
  double* tconst;      // [T]  (N_t log 2pi - N_t log beta + beta ||y_t||^2) / 2
  float *x, *r, *d, *ad, *xacc;  // [S][Dp]
  float *w, *wlo;      // [R * rows_total]
  float* part;         // [Dp/128][S] partial d^T A d per 128-coordinate tile
  float *rr, *bb;      // [S]
  int* steps;          // [S] CG steps of the current solve
  int* steps0;         // [S] CG steps of the first solve (Lanczos)
  int* active;         // [S]
  int* ractive;        // [S] still refining
  int* sweeps;         // [S]
  float* rrel;         // [S] last ||delta|| / ||x||
  float* rres;         // [S] ||b - A x|| / ||b|| of the returned solution
  int* task_active;    // [T]
  int* counters;       // [5]: 0 active systems, 1 refine-active systems, 2 status flags,
                       //      3 systems whose refinement diverged (reverted) in this E-step,
                       //      4 steps of the longest solve of a persistent CG launch
  int last_diverged;   // host copy of counters[3] after the last E-step
  int* hcounters;      // pinned host mirror [5]
  float *gam, *xi;     // [T*C*K][U]
  int* psteps;         // [T*C*K] CG steps of the probe systems' first solve
  float* sest;         // [T][C][Dp]
  double* quad;        // [T*C*K]
  double *logdet, *ell, *q;  // [T][C]
  int* assign;         // [T]
  double* stats;       // [4]: 0 loglik, 1 min margin
  double* lltask;      // [T] log sum_c pi_c p(y_t | alpha_c) of the last E-step
  double* mterms;      // [T_total][mterm_w] M-step terms of every task of the problem
  int64_t op_applies;

  // profiling (cmcs_profile): events around operator applications, per-task application
  // counts (device), launch counter (host)
  int prof_on;
  int prof_nev;                  // events recorded in the current E-step (pairs)
  cudaEvent_t* prof_ev;          // [2 * kProfEvents]
  int64_t* opcount;              // [T] device: operator applications per task
  int64_t prof_calls, res_calls, launches;
  double prof_ms, res_ms;
  int64_t prof_calls1;           // applications with Phi as one BF16 plane, and their time
  double prof_ms1;
  unsigned char* prof_tag;       // [kProfEvents] the recorded application used one plane
  int first_solve;               // the E-step's first solve (Lanczos coefficients) is running
  cudaEvent_t res_ev[2];

  // tensor-core operator (precision 1, 2 and 3); null otherwise
  void* tc;
  // tensor-core refinement residual (digit planes of Phi, kernels_ozaki.cu); null otherwise
  void* oz;
  // structured sensing of Sec. 4 (op == 1): Phi_t = Omega_t F applied by FFT (kernels_dft.cu)
  int op;
  int dft_L;              // log2 D
  float* dft_mask;        // [T][D] symmetrised mask in bit-reversed order
  void* dft_tw32;         // float2 [D/2] twiddles
  void* dft_tw64;         // double2 [D/2] twiddles
  int* dft_freq;          // [sum N_t] sampled frequencies, ascending per task
  int64_t* dft_off;       // [T+1]
  float* dft_y;           // [sum N_t][2] measured coefficients
  int dft_large;          // D beyond one CTA (or not a power of two): four-step transforms
  int dft_ndt;            // partial d^T A d slots per system written by the Fourier operator
  void* fs;               // four-step plan, tables and work buffer (kernels_dft_large.cu)
  void *dhi, *dlo;     // [S][Dp] BF16 hi and lo parts of the CG direction d (tensor-core path)

  char err[512];
};

// ---- kernels launched from the API unit -------------------------------------------------
cudaError_t launch_b0(Ctx* c);
cudaError_t launch_alpha_init(Ctx* c);
cudaError_t launch_sumlogalpha(Ctx* c);
cudaError_t launch_tconst_dev(Ctx* c, const int64_t* dN);
cudaError_t launch_probes_out(const Ctx* c, int64_t em_iter, float* dst);
// CG (kernels_cg.cu)
cudaError_t launch_cg_init(Ctx* c, int mode /*0 first solve, 1 refinement*/, int warm = 0);
// x of the mean systems += xacc of the mean systems (warm start: mu = mu_prev + delta)
cudaError_t launch_add_means(Ctx* c);
cudaError_t launch_cg_update(Ctx* c, int record);
cudaError_t launch_refine_update(Ctx* c);
cudaError_t launch_sest(Ctx* c);
// Jacobi preconditioner of the current alpha: pminv, pw and sumlogm (no-op without precond)
cudaError_t launch_precond(Ctx* c);
// column norms of Phi_t for the preconditioner (dense Phi; Fourier contexts fill N_t / D)
cudaError_t launch_colnorm(Ctx* c);
// operator (kernels_op.cu): AD = A D for all active tasks
cudaError_t launch_operator(Ctx* c, const float* V, float* Z, int with_dots);
// accurate residual: r = B - A xacc, B = b0 (k = 0) or the probe (k >= 1) when Bext == null
cudaError_t launch_residual(Ctx* c, const float* X, const float* Bext, float* Rout,
                            int all_systems = 0, int means_only = 0);
cudaError_t launch_resid_norm(Ctx* c);
// the same residual (all systems, dense Phi) on the tensor cores by error-free digit splitting
int oz_create(Ctx* c);
cudaError_t oz_refresh(Ctx* c);      // Phi changed: its column scales and digit planes
void oz_destroy(Ctx* c);
// columns j' < Rc of every task, systems j = j' jstride (all R, or the C means with K + 1)
cudaError_t oz_residual(Ctx* c, const float* X, const float* Bext, float* Rout, int Rc, int jstride);
// W[t][j'][n] = (Phi_t V_{t, j' * jstride})[n] for j' < Rc (FP32 SIMT pass 1 only)
// W = Phi V for Rc columns (systems j = j' * jstride); with Wlo, as a compensated pair W + Wlo
cudaError_t launch_phi_v(Ctx* c, const float* V, float* W, float* Wlo, int Rc, int jstride);
// structured (Fourier) operator (kernels_dft.cu)
constexpr int kDftMaxD = 8192;     // one pair's FP64 spectrum in shared memory (single CTA)
constexpr int kDftMaxLarge = 1 << 20;   // four-step transforms
bool dft_size_ok(int D);
int dft_create(Ctx* c, const uint8_t* mask, const float* y, int on_device);
void dft_destroy(Ctx* c);
cudaError_t launch_dft_apply(Ctx* c, const float* V, float* Z, int with_dots);
cudaError_t launch_dft_residual(Ctx* c, const float* X, const float* Bext, float* Rout,
                                int all_systems, int means_only);
cudaError_t launch_dft_b0(Ctx* c);
// one whole CG step (operator and update) for every active system of a Fourier context
cudaError_t launch_dft_cg_step(Ctx* c, int record);
// a whole CG solve in one persistent launch (counters[4]: steps of the longest solve)
cudaError_t launch_dft_cg_solve(Ctx* c, int record);
// four-step transforms for D = 2^a 5^b (16 | D, D <= 2^20) beyond one CTA (kernels_dft_large.cu)
bool dft_large_ok(int D);
int fs_create(Ctx* c, const uint8_t* hmask);   // hmask: host [T][D]
void fs_destroy(Ctx* c);
cudaError_t fs_apply(Ctx* c, const float* V, float* Z, int with_dots);
cudaError_t fs_residual(Ctx* c, const float* X, const float* Bext, float* Rout, int all_systems,
                        int means_only);
cudaError_t fs_b0(Ctx* c);
// adjoint gradients (adjoint.cu)
cudaError_t launch_adj_dy(Ctx* c, const float* Wl, const float* Wl_lo, float* dy);
cudaError_t launch_adj_dalpha(Ctx* c, const float* lam, float* dalpha);
// dPhi for the padded rows [row_lo, row_hi) of the packed Phi, written to out at the caller's
// unpadded row index minus out_base
cudaError_t launch_adj_dphi(Ctx* c, const float* lam, const float* Wl, const float* Wl_lo,
                            const float* Wm, const float* Wm_lo, float* out, int64_t row_lo,
                            int64_t row_hi, int64_t out_base);
// E-step tail and M-step (kernels_estep.cu)
cudaError_t launch_quadrature(const float* gam, const float* xi, const int* steps, int nsys,
                              int ld, double* out, int* status, cudaStream_t st);
cudaError_t launch_quadrature_ctx(Ctx* c, cudaStream_t st);
cudaError_t launch_ell_softmax(Ctx* c, const float* rmu /* residuals for the correction, or null */);
// M-step: this context's per-task terms into its rows of mterms, then alpha (and pi, L) from
// all T_total rows summed in task order
cudaError_t launch_mstep_terms(Ctx* c);
cudaError_t launch_mstep_apply(Ctx* c);

// tensor-core operator hooks (kernels_tc.cu)
int tc_create(Ctx* c);      // returns 0 on success
void tc_destroy(Ctx* c);
cudaError_t tc_operator(Ctx* c, const float* V, float* Z, int with_dots);
cudaError_t tc_split_vectors(Ctx* c, const float* V);   // V -> dhi, dlo
cudaError_t tc_refresh(Ctx* c);                         // recompute the BF16 copies of Phi

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
// CG step cap in force: cg_max_iter, or refine_steps during the refinement sweeps
inline int cg_cap(const Ctx* c) { return c->capsel ? c->refine_steps : c->U; }
// the tensor-core operator holds Phi as one BF16 plane now: always with CMCS_BF16_REFINE, in
// the first solve with CMCS_BF16_MIXED
inline int one_plane(const Ctx* c) {
  return c->tc != nullptr && (c->precision == CMCS_BF16_REFINE ||
                              (c->precision == CMCS_BF16_MIXED && c->first_solve));
}
int pick_tn(int R, int max_tn);
int tc_set_stages(Ctx* c, int stages);   // returns the stages in force (0: not a TC context)
int tc_max_stages(Ctx* c);

}  // namespace cmcs
