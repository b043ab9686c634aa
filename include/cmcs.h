/*
 * cmcs.h -- C ABI of libcmcs.so: covariance-free EM (CoFEM) for clustered multi-task
 * compressive sensing on one NVIDIA GB300 (sm_103a).
 *
 * Model (Lin & Ba, "An efficient algorithm for clustered multi-task compressive sensing",
 * Sec. 2, Eq. 1): task t has measurements y_t = Phi_t z_t + noise (noise precision beta),
 * z_t | a_t = c ~ N(0, diag(alpha_c)^-1), a_t ~ Categorical(pi).  The library runs the EM
 * loop of Alg. 2 with the E-step of Sec. 3: for every (task t, cluster c) it solves
 *     (beta Phi_t^T Phi_t + diag(alpha_c)) x = b                                  (Eq. 7)
 * by conjugate gradient (Alg. 1) for b = beta Phi_t^T y_t (posterior mean mu_tc) and for K
 * Rademacher probes (Eq. 4), estimates diag(Sigma_tc) (Eq. 4) and log det Sigma_tc by
 * Lanczos quadrature over the CG coefficients (Eqs. 9-11), forms the responsibilities q_tc
 * (Eq. 3) and updates alpha_c by Eq. 5.
 *
 * Conventions for every call:
 *  - Array layouts are dense row-major with no padding: Phi is [sum_t N_t][D] (task t's
 *    rows follow task t-1's), y is [sum_t N_t], per-(t,c) vectors are [T][C][D], per-(t,c)
 *    scalars [T][C], alpha [C][D].
 *  - A pointer argument is host memory when the accompanying `on_device` is 0 and CUDA device
 *    memory of the context's device when it is 1.  The library never keeps a caller pointer
 *    past the call that received it; it copies what it needs into memory it owns.
 *  - All GPU work is ordered on the CUDA stream given to cmcs_create.  For NULL (the legacy
 *    default stream) the context creates a blocking stream of its own, which orders itself
 *    with the legacy stream and, unlike it, can be captured into CUDA graphs.  Every call
 *    returns only after its work has completed, and reports device errors through its status.
 *  - Errors: a call that fails validation returns CMCS_ERR_INVALID_ARG and changes no state.
 *    cmcs_last_error() returns a description of the most recent failure of that context.
 *  - No call allocates or frees device memory except cmcs_create and cmcs_destroy.
 */
#ifndef CMCS_H
#define CMCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cmcs_ctx cmcs_ctx;

typedef enum {
  CMCS_OK = 0,
  CMCS_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad enum, non-positive beta, ... */
  CMCS_ERR_CUDA = 2,          /* a CUDA runtime call failed; see cmcs_last_error          */
  CMCS_ERR_OOM = 3,           /* device allocation failed in cmcs_create                  */
  CMCS_ERR_NUMERIC = 4,       /* NaN or Inf reached an output (e.g. NaN in y)             */
  CMCS_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up                       */
  CMCS_ERR_UNSUPPORTED = 6    /* a valid request the library does not implement          */
} cmcs_status;

typedef enum {
  /* operator and CG in FP32 (SIMT FMA); refinement residual with compensated FP32 products
     and sums (about twice FP32's precision) */
  CMCS_FP32 = 0,
  /* operator with Phi held in BF16 on the tcgen05 tensor cores (FP32 accumulation in TMEM);
     CG vectors FP32 (entering the MMA as BF16 hi + lo pairs); the refinement residual is the
     tensor-core one of CMCS_BF16X3 */
  CMCS_BF16_REFINE = 1,
  /* operator on the tensor cores with Phi and the vectors both split into BF16 hi + lo pairs
     (three MMAs per step: about 16 significant bits per product, FP32 accumulation); the
     refinement residual on the tensor cores from exact BF16 digit planes of the FP32 Phi and
     of the vectors (Ozaki's error-free splitting): Phi^T W is formed without rounding, W and x
     are rounded at FP32 level (an error refinement sees only through beta Phi^T); the residual
     of the returned means (for ell's data term) is the compensated one of CMCS_FP32 */
  CMCS_BF16X3 = 2,
  /* the first CG solve (the one whose coefficients feed the log-det estimate of Eqs. 9-11)
     with Phi held in BF16 on the tensor cores, as CMCS_BF16_REFINE (half the bytes of Phi per
     application); the refinement sweeps' inner solves with the CMCS_BF16X3 operator and its
     refinement residual, so the returned solutions reach the same accuracy.  cmcs_apply with
     accurate = 0 applies the CMCS_BF16X3 operator */
  CMCS_BF16_MIXED = 3
} cmcs_precision;

typedef struct {
  int T;                  /* tasks, >= 1                                                  */
  int C;                  /* clusters, >= 1                                               */
  int D;                  /* signal dimension, >= 1                                       */
  int K;                  /* Rademacher probes per (t, c), >= 1                           */
  const int64_t *N;       /* host [T]: rows N_t of Phi_t, each >= 1                      */
  double beta;            /* noise precision (known, Sec. 2), > 0                         */
  const double *pi;       /* host [C]: cluster priors (known, Sec. 2), > 0, summing to 1  */
  int cg_max_iter;        /* cap on CG steps per solve (U of Sec. 3), 1..512               */
  double cg_tol;          /* stop a system once ||r_{u+1}|| <= cg_tol * ||b||, >= 0        */
  uint64_t seed;          /* keys the Philox draws: alpha initialisation and probes       */
  int precision;          /* cmcs_precision                                               */
  int refine_max;         /* refinement sweeps after the first CG solve, 0..64            */
  double refine_tol;      /* stop refining a system once its estimated relative error is
                             <= refine_tol: after sweep 1 ||delta_1|| / ||x||, after sweep k
                             rho ||delta_k|| / ((1 - rho) ||x||), rho = ||delta_k|| / ||delta_k-1|| */
  double alpha_min;       /* M-step clamp, > 0                                            */
  double alpha_max;       /* M-step clamp, > alpha_min                                    */
  int schedule;           /* 0: every task in one operator launch per pass (default);
                             1: one launch per task (the per-task loop, for comparison)   */
  int graphs;             /* 1: capture chunks of CG steps in CUDA graphs and replay them  */
  int autotune;           /* 1: at create, time the operator variants (SIMT tile width or
                             tensor-core pipeline depth) and keep the fastest              */
  /* Variants of the method, all 0 (off) by default. */
  int learn_pi;           /* 1: every M-step also learns the priors (Sec. 2 allows it):
                             pi_c = max((1/T) sum_t q_tc, 1e-300), renormalised to sum 1   */
  int probe_share;        /* 1: every cluster of task t uses the same probes,
                             p_{t,c,k} = p_{t,0,k} (common random numbers across c)         */
  int precond;            /* 1: Jacobi-preconditioned CG, M = diag(A), m_d = beta ||Phi_t e_d||^2
                             + alpha_cd: probe systems A x_k = sqrt(m) * p_k, stopping test
                             r^T M^-1 r <= cg_tol^2 b^T M^-1 b, s = (1/K) sum_k p_k x_k /
                             sqrt(m) and log det Sigma = Eq. 11's estimate - sum_d log m_d  */
  int warm_start;         /* 1: from the second E-step on, each mean system starts from the
                             previous E-step's mean (x_1 = mu_prev: CG on b0 - A mu_prev, with
                             the compensated residual, stopped at ||r|| <= cg_tol ||b0||); the
                             probe systems keep x_1 = 0, which the Lanczos estimate needs.
                             cmcs_set_alpha keeps the previous means as the start (any start
                             is valid); cmcs_set_data and a failed E-step drop them          */
  /* Tasks split across contexts, one per GPU (Sec. 3.3: the E-step of task t needs only Phi_t,
     y_t and every alpha_c; the M-step of Eq. 5 sums over tasks).  0 and 0 for a whole problem. */
  int task_offset;        /* global index of this context's first task, >= 0: the probes of its
                             task t are those of task task_offset + t of the whole problem     */
  int T_total;            /* tasks of the whole problem (0: T); task_offset + T <= T_total.
                             With T_total > T, cmcs_em_iter is refused: the M-step goes through
                             cmcs_mstep_terms and cmcs_mstep_apply                            */
  int refine_steps;       /* step cap of the CG solves inside the refinement sweeps, 0..cg_max_iter
                             (0: cg_max_iter).  Only the first solve feeds the Lanczos estimate
                             (Eqs. 9-11); a sweep only has to shrink the error, and refine_tol
                             still decides when the sweeps stop                               */
} cmcs_config;

/* Summary of the most recent E-step and the EM state. */
typedef struct {
  int64_t em_iters_done;   /* M-steps applied since create (plus the offset of set_alpha) */
  double loglik;           /* L(theta) = (1/T) sum_t log sum_c pi_c p(y_t|alpha_c) (Sec. 2)
                              of the last E-step, with log det from the estimator of Eq. 11 */
  int cg_steps_max;        /* largest CG step count U_i of the first solve                  */
  double cg_steps_mean;    /* mean U_i over all T*C*(K+1) systems of the first solve        */
  int64_t cg_capped;       /* systems of the first solve that stopped at cg_max_iter        */
  int refine_sweeps_max;   /* largest number of refinement sweeps any system took           */
  double refine_rel_max;   /* largest final ||delta|| / ||x|| over refined systems (0: none) */
  double min_margin;       /* smallest gap q_{t,a_t} - max_{c != a_t} q_tc over tasks        */
  int64_t operator_applies;/* batched operator applications (all systems) in the last E-step */
  double resid_rel_max;    /* largest ||b0 - A mu|| / ||b0|| of the returned means, from the
                              compensated residual after refinement (0 when refine_max = 0)  */
  int64_t refine_diverged; /* systems whose refinement stopped because a correction grew (the
                              inner solves did not contract); their last correction is undone */
  int operator_variant;    /* operator variant in use: SIMT tile width (columns per thread)
                              or tensor-core pipeline stages                                */
} cmcs_summary;

/* What cmcs_read copies out.  Element types and shapes: */
typedef enum {
  CMCS_OUT_MU = 0,       /* float  [T][C][D]  posterior means mu_tc (Eq. 3), refined       */
  CMCS_OUT_S = 1,        /* float  [T][C][D]  diagonal estimates s_tc (Eq. 4)              */
  CMCS_OUT_Q = 2,        /* double [T][C]     responsibilities q_tc (Eq. 3)                */
  CMCS_OUT_LOGDET = 3,   /* double [T][C]     log det Sigma_tc estimate nu (Eq. 11)        */
  CMCS_OUT_ELL = 4,      /* double [T][C]     ell_tc (Eq. 3)                               */
  CMCS_OUT_ALPHA = 5,    /* float  [C][D]     current alpha_c (after the last M-step)      */
  CMCS_OUT_ASSIGN = 6,   /* int32  [T]        a_t = argmax_c q_tc, lowest c on ties (Alg. 2)*/
  CMCS_OUT_RECON = 7,    /* float  [T][D]     reconstructions mu_{t, a_t} (Alg. 2)         */
  CMCS_OUT_STEPS = 8,    /* int32  [T][C][K+1] CG steps U of the first solve; index 0 is the
                                              mean system, 1..K the probes                  */
  CMCS_OUT_GAMMA = 9,    /* float  [T][C][K][cg_max_iter] CG step sizes gamma_u of the probe
                                              systems (Alg. 1), zero past U               */
  CMCS_OUT_XI = 10,      /* float  [T][C][K][cg_max_iter] CG coefficients xi_u, zero past U */
  CMCS_OUT_B0 = 11,      /* float  [T][D]     beta Phi_t^T y_t (Eq. 7)                      */
  CMCS_OUT_SWEEPS = 12,  /* int32  [T][C][K+1] refinement sweeps taken per system           */
  CMCS_OUT_RESID = 13,   /* float  [T][C][K+1] ||b - A x|| / ||b|| of the returned means
                                              (index 0; other entries and refine_max = 0: 0) */
  CMCS_OUT_PI = 14       /* double [C]        cluster priors in force (learned: after the
                                              last M-step; else the configured ones)        */
} cmcs_output;

/* Create a context: validates cfg, copies Phi and y into library-owned device memory (padded
 * and, for CMCS_BF16_REFINE, also converted to BF16), computes b0_t = beta Phi_t^T y_t, and
 * draws alpha_c ~ Uniform(0,1) (Alg. 2, first step) from Philox-4x32-10 keyed by cfg->seed.
 * Phi: float [sum N_t][D]; y: float [sum N_t]; host or device per on_device.
 * stream: a cudaStream_t (or NULL).  On success *out owns all its memory; free it with
 * cmcs_destroy.  Returns CMCS_ERR_OOM if device memory runs out (nothing is leaked). */
cmcs_status cmcs_create(const cmcs_config *cfg, const float *Phi, const float *y, int on_device,
                        void *stream, cmcs_ctx **out);

/* Create a context for the structured sensing matrices of Sec. 4, Phi_t = Omega_t F: F the
 * unitary D x D DFT (F_kd = e^{-2 pi i k d / D} / sqrt(D)) and Omega_t the rows selected by
 * mask (uint8 [T][D], nonzero = frequency k sampled for task t; cfg->N[t] must equal the
 * count).  y: float [sum N_t][2], the complex measurements (real, imaginary) of each task in
 * ascending frequency order.  The signals z_t are real; reading the real and imaginary parts
 * of y_t as 2 N_t real measurements of noise precision beta gives
 *     A_tc = beta Re(Phi_t^H Phi_t) + diag(alpha_c),   b0_t = beta Re(Phi_t^H y_t),
 * applied by FFT in O(D log D) per system (Sec. 3.3) instead of O(N_t D).  Requires
 * cfg->precision == CMCS_FP32 and D either a power of two in [128, 8192] (one CTA transforms
 * a pair of systems in shared memory, fused with the CG update) or D = 2^a 5^b with 16 | D,
 * 128 <= D <= 2^20, e.g. 100,000 (four-step transforms, D = n1 n2 with n1, n2 <= 1024, in
 * three launches per application); else CMCS_ERR_UNSUPPORTED.  The CG operator runs FP32
 * FFTs; the refinement residual and b0 run FP64 FFTs.  Every call below works on such a
 * context except cmcs_set_data and cmcs_adjoint (CMCS_ERR_UNSUPPORTED).  mask and y are host
 * or device per on_device. */
cmcs_status cmcs_create_dft(const cmcs_config *cfg, const uint8_t *mask, const float *y,
                            int on_device, void *stream, cmcs_ctx **out);

/* Replace alpha (float [C][D], every entry > 0) and set the EM iteration counter, which keys
 * the probes of the next E-step (Alg. 2 draws fresh probes every iteration). */
cmcs_status cmcs_set_alpha(cmcs_ctx *ctx, const float *alpha, int on_device, int64_t em_iter);

/* One E-step (Eq. 3 via Sec. 3) with the current alpha: fills mu, s, logdet, ell, q, the
 * assignments and the CG statistics.  alpha and the iteration counter are unchanged.
 * With refine_max > 0 the data term beta y^T Phi mu of ell (= b0^T A^-1 b0) is evaluated as
 * b0^T mu + mu^T (b0 - A mu) with the compensated residual, so its error is quadratic in the
 * error of mu. */
cmcs_status cmcs_estep(cmcs_ctx *ctx);

/* n EM iterations of Alg. 2: each is an E-step followed by the M-step of Eq. 5 and an
 * increment of the iteration counter.  After the call, mu/q/assign are those of the last
 * E-step and alpha is the result of the last M-step. */
cmcs_status cmcs_em_iter(cmcs_ctx *ctx, int n);

/* Per-task terms of the M-step (Eq. 5) and of L(theta) (Sec. 2) from the last E-step, for EM
 * with the tasks split across contexts (Sec. 3.3).  terms: double [T][W] with W = C (D + 1) + 1,
 * host or device per on_device; row t (this context's task t) holds
 *   [c (D + 1)]         q_tc                                   (Eq. 3)
 *   [c (D + 1) + 1 + d] q_tc max(mu_tcd^2 + s_tcd, 0)           (Eq. 5 with s for diag Sigma)
 *   [C (D + 1)]         log sum_c pi_c p(y_t | alpha_c)          (the task's term of L(theta))
 * The rows of every context, stacked in global task order, are what cmcs_mstep_apply takes. */
cmcs_status cmcs_mstep_terms(cmcs_ctx *ctx, double *terms, int on_device);

/* The M-step from the terms of all T_total tasks of the problem (double [T_total][W] in global
 * task order, host or device per on_device): alpha_cd = sum_t q_tc / sum_t q_tc max(mu^2 + s, 0)
 * with the sums taken over t in order (then the clamps of cmcs_config; a cluster with
 * sum_t q_tc < 1e-300 keeps its alpha), pi_c = max((1/T_total) sum_t q_tc, 1e-300) renormalised
 * when learned, L(theta) = (1/T_total) sum_t of the last column; then the iteration counter is
 * incremented.  Because the sums run over the same rows in the same order, contexts holding
 * any split of the tasks reach the same alpha bit for bit as one context holding them all
 * (cmcs_em_iter goes through the same two steps). */
cmcs_status cmcs_mstep_apply(cmcs_ctx *ctx, const double *terms, int on_device);

/* Replace Phi and y (same shapes as at create; host or device per on_device) and recompute
 * b0 = beta Phi^T y.  alpha, the iteration counter and the settings are kept; outputs of earlier
 * E-steps are stale until the next cmcs_estep. */
cmcs_status cmcs_set_data(cmcs_ctx *ctx, const float *Phi, const float *y, int on_device);

/* Reverse-mode derivative of the posterior means of the last E-step.  The paper has no adjoint;
 * this follows from Eq. 3 by differentiating mu_tc = A_tc^-1 (beta Phi_t^T y_t) with
 * A_tc = beta Phi_t^T Phi_t + diag(alpha_c).  Given g = dL/dmu (float [T][C][D]) it solves the
 * adjoint systems A_tc lambda_tc = g_tc with the same symmetric operator (CG of Alg. 1 with the
 * context's tol and step cap, then compensated refinement as in the E-step; nothing from the
 * forward CG is stored) and writes
 *   dy     float [sum N_t]     = beta sum_c Phi_t lambda_tc
 *   dalpha float [C][D]        = - sum_t lambda_tc * mu_tc
 *   dPhi   float [sum N_t][D]  = beta sum_c ((y_t - Phi_t mu_tc) lambda_tc^T - (Phi_t lambda_tc) mu_tc^T)
 * (dPhi may be NULL).  Responsibilities, s and the log-det estimate are treated as constants.
 * All pointers host or device per on_device.  The E-step's work buffers and refinement
 * statistics (CMCS_OUT_SWEEPS, refine fields of cmcs_summary) are overwritten; mu, s, q and
 * alpha are not. */
cmcs_status cmcs_adjoint(cmcs_ctx *ctx, const float *g, float *dy, float *dalpha, float *dPhi,
                         int on_device);

/* Copy an output (see cmcs_output) into dst, host or device per on_device. */
cmcs_status cmcs_read(const cmcs_ctx *ctx, int what, void *dst, int on_device);

/* Scalar summary of the last E-step. */
cmcs_status cmcs_result(const cmcs_ctx *ctx, cmcs_summary *out);

/* Apply A_tc = beta Phi_t^T Phi_t + diag(alpha_c) (Eq. 7) to V, float [T][C*(K+1)][D] (vector
 * j of task t uses cluster c = j / (K+1)), writing Z of the same shape.  accurate = 0 uses
 * the E-step's batched operator (FP32 or BF16 per precision); accurate = 1 computes
 * B - A V as the refinement residual of the context's precision (compensated SIMT products
 * for CMCS_FP32, the tensor-core digit-plane residual for the BF16 precisions) for B given in
 * Z on entry.  V and Z are host or device per on_device.  The E-step's work buffers are reused,
 * so results of a previous E-step other than alpha, b0 and the counter are invalidated. */
cmcs_status cmcs_apply(cmcs_ctx *ctx, const float *V, float *Z, int on_device, int accurate);

/* Write the probes p_{t,c,k} of EM iteration em_iter (Eq. 4, Alg. 2) as float +-1 into
 * dst [T][C][K][D], host or device per on_device. */
cmcs_status cmcs_probes(const cmcs_ctx *ctx, int64_t em_iter, float *dst, int on_device);

/* Stand-alone Lanczos log quadrature (Eqs. 9-10): for each of nsys systems, build the
 * U_i x U_i matrix of Eq. 9 from gamma[i*ld .. i*ld+U_i-1] and xi[i*ld .. i*ld+U_i-2]
 * (float, device), eigendecompose it (implicit-shift QR in FP64, first eigenvector
 * components only) and write out[i] = sum_u S_{u,1}^2 log lambda_u (double, device), i.e.
 * Eq. 10 divided by ||p||^2.  steps: int32 [nsys] device, 0 <= U_i <= ld <= 512; U_i = 0
 * gives 0.  status: int32 device scalar, set to nonzero if an eigen iteration cap was hit.
 * stream: cudaStream_t or NULL. */
cmcs_status cmcs_lanczos_quadrature(const float *gamma, const float *xi, const int32_t *steps,
                                    int nsys, int ld, double *out, int32_t *status,
                                    void *stream);

/* Test hook for failure detection (tensor-core precisions only).  With enable = 1 every
 * operator launch makes its MMA warp wait on a barrier that nothing arrives at; the wait gives
 * up after its 2-second wall-time limit, the kernel takes its abort path (stops issuing, waits
 * for its copies and MMAs in flight, frees its tensor memory) and the E-step returns
 * CMCS_ERR_TIMEOUT.  enable = 0 restores normal operation; the context stays usable. */
cmcs_status cmcs_test_stall(cmcs_ctx *ctx, int enable);

/* Operator profile accumulated since profiling was last enabled on a context. */
typedef struct {
  int64_t operator_calls;    /* batched operator applications (each: Phi pass + Phi^T pass) */
  double operator_ms;        /* their summed device time, CUDA events on the context stream  */
  double operator_flops;     /* algorithmic FLOPs: sum over applied tasks of 4 N_t D R        */
  double operator_bytes;     /* algorithmic bytes: per applied task s_Phi N_t D (Phi read once,
                                s_Phi = 4 for FP32, 2 for BF16) + 4 R (2 D + 2 N_t) (V, W, Z)  */
  int64_t residual_calls;    /* refinement residual applications                             */
  double residual_ms;        /* their summed device time                                     */
  int64_t kernel_launches;   /* all kernels the library launched                             */
  int64_t operator_calls_bf16; /* of the operator applications, those with Phi held as one
                                  BF16 plane (CMCS_BF16_REFINE; the first solve of
                                  CMCS_BF16_MIXED)                                            */
  double operator_ms_bf16;   /* their summed device time                                     */
} cmcs_profile_data;

/* enable = 1 resets and starts the profile (events bracket every operator application, which
 * adds a few microseconds per application); enable = 0 stops it.  Events are created here, not
 * during the E-step; at most 8192 operator applications per E-step are timed. */
cmcs_status cmcs_profile(cmcs_ctx *ctx, int enable);

/* Read the profile (synchronises the context stream). */
cmcs_status cmcs_profile_read(const cmcs_ctx *ctx, cmcs_profile_data *out);

/* Operator without device allocation: Z = beta Phi^T (Phi V) + diag(alpha) V for m vectors
 * of one task.  The paper has no counterpart; this entry point exists for callers that cannot
 * call cudaMalloc while they run (their device memory is owned by their own pool allocator,
 * or they cannot afford cudaMalloc's implicit synchronisation).  It allocates nothing and calls
 * no allocating routine: the intermediate Phi V is kept in a fixed 16 MiB device array inside
 * the library, so m * N must not exceed 4,194,304 (larger requests return
 * CMCS_ERR_INVALID_ARG with a message for cmcs_last_error(NULL)).
 * Phi: float [N][D] row-major, alpha: float [D], V and Z: float [m][D]; all device memory of
 * the current device (a host pointer or another device's memory returns CMCS_ERR_INVALID_ARG
 * before anything is launched); beta > 0.  stream: cudaStream_t or NULL; the call synchronises
 * that stream before it returns, so the host waits for its two kernels.  Every call shares that
 * one array (per device), which keeps the previous call's contents; calls whose GPU work
 * overlaps (other host threads, other streams) race on it.  The first call on each device looks
 * up the array's device address with that device current and keeps it; make that first call
 * before any stream capture.  The kept address does not survive cudaDeviceReset: do not call
 * this entry point on a device after resetting it. */
cmcs_status cmcs_apply_noalloc(const float *Phi, int N, int D, const float *alpha, double beta,
                               const float *V, int m, float *Z, void *stream);

/* Description of the last failure on ctx (or, when ctx is NULL, of the last failed
 * cmcs_create or context-free call).  Valid until the next call on the same context. */
const char *cmcs_last_error(const cmcs_ctx *ctx);

/* Release everything the context owns.  NULL is accepted. */
void cmcs_destroy(cmcs_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* CMCS_H */
