// C ABI of libcmcs.so (declared in include/cmcs.h): context management and the host driver of
// the E-step (Alg. 2, inner loop) and M-step (Eq. 5).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <utility>
#include <vector>

#include "cmcs_internal.cuh"

using namespace cmcs;

struct cmcs_ctx {
  Ctx c;
};

namespace {

thread_local char g_create_err[512] = "";

void set_err(Ctx* c, const char* fmt, ...) {
  char* dst = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
}

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess) {                                                        \
      set_err(c, "%s failed: %s", #call, cudaGetErrorString(_e));                   \
      return _e == cudaErrorMemoryAllocation ? CMCS_ERR_OOM : CMCS_ERR_CUDA;         \
    }                                                                               \
  } while (0)

template <typename Tp>
cudaError_t dalloc(Tp** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(Tp));
}

void free_ctx(Ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->phi, c->y, c->drow, c->tile_task, c->b0hi, c->b0lo, c->alpha,
                  c->sumlogalpha, c->logpi, c->tconst, c->x, c->r, c->d, c->ad, c->xacc,
                  c->w, c->wlo, c->part, c->rr, c->bb, c->steps, c->steps0, c->active,
                  c->ractive, c->sweeps, c->rrel, c->rres, c->task_active, c->counters, c->gam, c->xi,
                  c->psteps, c->sest, c->quad, c->logdet, c->ell, c->q, c->assign, c->stats, c->lltask, c->mterms,
                  c->dN, c->opcount, c->dorow, c->stall_flag, c->adj_g, c->adj_x, c->adj_wl, c->adj_wm,
                  c->adj_wl_lo, c->adj_wm_lo, c->adj_dy, c->adj_da, c->pi, c->colnorm, c->pminv,
                  c->pw, c->sumlogm};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->prof_ev) {
    for (int i = 0; i < 2 * kProfEvents; ++i) cudaEventDestroy(c->prof_ev[i]);
    cudaEventDestroy(c->res_ev[0]);
    cudaEventDestroy(c->res_ev[1]);
    free(c->prof_ev);
    free(c->prof_tag);
  }
  if (c->hcounters) cudaFreeHost(c->hcounters);
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 2; ++k)
      for (int q = 0; q < 2; ++q)
        if (c->graph[r][k][q]) cudaGraphExecDestroy(c->graph[r][k][q]);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->tc) tc_destroy(c);
  if (c->oz) oz_destroy(c);
  dft_destroy(c);
  free(c->hN);
  free(c->hNp);
  free(c->hrow);
  free(c->hpi);
  free(c->horow);
}

cudaMemcpyKind kind_in(int on_device) {
  return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_out(int on_device) {
  return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

cmcs_status sync_check(Ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(c, "CUDA error: %s", cudaGetErrorString(e));
    return CMCS_ERR_CUDA;
  }
  return CMCS_OK;
}

cmcs_status read_counters(Ctx* c) {
  CK(cudaMemcpyAsync(c->hcounters, c->counters, 5 * sizeof(int), cudaMemcpyDeviceToHost,
                     c->stream));
  return sync_check(c);
}

// CG steps between host polls of the active-system count (evaluation switch CMCS_CG_CHUNK)
constexpr int kCheckEvery = 8;
static_assert(kCheckEvery <= kProfEvents, "events of one chunk");

// operator application, bracketed by profiling events when enabled (pair prof_nev of the
// current chunk of CG steps)
cudaError_t timed_operator(Ctx* c, int record) {
  const bool ev = c->prof_on && c->prof_nev < kProfEvents;
  // while capturing, external records become event-record nodes of the graph
  const unsigned flags = c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (ev) {
    cudaError_t er = cudaEventRecordWithFlags(c->prof_ev[2 * c->prof_nev], c->stream, flags);
    if (er != cudaSuccess) return er;
    c->prof_tag[c->prof_nev] = (unsigned char)one_plane(c);
  }
  // Fourier with D in one CTA: the operator and the CG update are one kernel
  cudaError_t e = (c->op == 1 && !c->dft_large) ? launch_dft_cg_step(c, record)
                                                : launch_operator(c, c->d, c->ad, 1);
  if (ev && e == cudaSuccess) {
    e = cudaEventRecordWithFlags(c->prof_ev[2 * c->prof_nev + 1], c->stream, flags);
    c->prof_nev++;
  }
  if (c->prof_on) {
    c->prof_calls++;
    if (one_plane(c)) c->prof_calls1++;
  }
  return e;
}

// fold the recorded event pairs into the profile (the stream must have been synchronised)
void fold_events(Ctx* c) {
  for (int i = 0; i < c->prof_nev; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]) == cudaSuccess) {
      c->prof_ms += ms;
      if (c->prof_tag[i]) c->prof_ms1 += ms;
    }
    else
      cudaGetLastError();     // a missing timing must not surface as a failure of the E-step
  }
  c->prof_nev = 0;
}

// n CG steps (operator + update) launched directly
cmcs_status cg_steps_direct(Ctx* c, int record, int n) {
  for (int i = 0; i < n; ++i) {
    CK(timed_operator(c, record));
    if (c->op != 1 || c->dft_large) CK(launch_cg_update(c, record));
    c->op_applies++;
  }
  return CMCS_OK;
}

// the graph replaying c->chunk CG steps, captured on first use
cudaGraphExec_t chunk_graph(Ctx* c, int record) {
  cudaGraphExec_t& g = c->graph[record][c->capsel][c->prof_on];
  if (g != nullptr || c->graph_failed[record][c->capsel][c->prof_on]) return g;
  const int64_t l0 = c->launches, a0 = c->op_applies, p0 = c->prof_calls;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return nullptr;
  c->prof_nev = 0;
  c->capturing = 1;
  cmcs_status s = cg_steps_direct(c, record, c->chunk);
  c->capturing = 0;
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  c->graph_launches = c->launches - l0;
  c->launches = l0;
  c->op_applies = a0;
  c->prof_calls = p0;
  c->prof_nev = 0;
  if (s != CMCS_OK || e != cudaSuccess || graph == nullptr) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    c->graph_failed[record][c->capsel][c->prof_on] = 1;   // run this variant directly
    c->err[0] = 0;
    return nullptr;
  }
  e = cudaGraphInstantiate(&g, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g = nullptr;
    c->graph_failed[record][c->capsel][c->prof_on] = 1;
  }
  return g;
}

// Alg. 1 for every active system until all have stopped (or the step cap in force), in
// chunks of c->chunk steps between host polls of the number of active systems
// Fourier operator within one CTA: the whole solve as one persistent launch (each CTA loops its
// pair's CG steps); CMCS_DFT_PERSIST=0 (evaluation switch) keeps one launch per step
cmcs_status run_cg_persistent(Ctx* c, int record) {
  CK(cudaMemsetAsync(c->counters + 4, 0, sizeof(int), c->stream));
  const bool ev = c->prof_on;
  if (ev) CK(cudaEventRecord(c->prof_ev[0], c->stream));
  CK(launch_dft_cg_solve(c, record));
  if (ev) CK(cudaEventRecord(c->prof_ev[1], c->stream));
  cmcs_status s = read_counters(c);
  if (s != CMCS_OK) return s;
  const int n = c->hcounters[4];        // steps of the longest solve: operator applications
  c->op_applies += n;
  if (ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[0], c->prof_ev[1]) == cudaSuccess) c->prof_ms += ms;
    else cudaGetLastError();
    c->prof_calls += n;
  }
  return CMCS_OK;
}

cmcs_status run_cg(Ctx* c, int record) {
  static int persist = -1;
  if (persist < 0) {
    const char* v = getenv("CMCS_DFT_PERSIST");
    persist = v ? atoi(v) != 0 : 1;
  }
  if (persist && c->op == 1 && !c->dft_large) return run_cg_persistent(c, record);
  const int cap = cg_cap(c);
  for (int u = 0; u < cap; u += c->chunk) {
    const int n = cap - u < c->chunk ? cap - u : c->chunk;
    cudaGraphExec_t g = (c->use_graphs && n == c->chunk) ? chunk_graph(c, record) : nullptr;
    if (g != nullptr) {
      CK(cudaGraphLaunch(g, c->stream));
      c->launches += c->graph_launches;
      c->op_applies += n;
      if (c->prof_on) {
        c->prof_calls += n;
        c->prof_nev = n;
        const int op1 = one_plane(c);
        if (op1) c->prof_calls1 += n;
        for (int i = 0; i < n; ++i) c->prof_tag[i] = (unsigned char)op1;
      }
    } else {
      c->prof_nev = 0;
      cmcs_status s = cg_steps_direct(c, record, n);
      if (s != CMCS_OK) return s;
    }
    cmcs_status s = read_counters(c);
    if (s != CMCS_OK) return s;
    fold_events(c);
    if (c->hcounters[2] & 8) {
      set_err(c, "a bounded device-side wait expired in the tensor-core operator");
      return CMCS_ERR_TIMEOUT;
    }
    if (c->hcounters[0] == 0) break;
  }
  return CMCS_OK;
}

// Iterative refinement of the solutions in xacc: each sweep forms the residual B - A xacc with
// compensated products (B = b0 and the probes, or Bext), solves for the correction with
// Alg. 1 and adds it; a system stops once its correction is small or stops shrinking.
cmcs_status refine_sweeps(Ctx* c, const float* Bext) {
  for (int sw = 0; sw < c->refine_max; ++sw) {
    if (c->prof_on) cudaEventRecord(c->res_ev[0], c->stream);
    CK(launch_residual(c, c->xacc, Bext, c->r));
    if (c->prof_on) {
      cudaEventRecord(c->res_ev[1], c->stream);
      c->res_calls++;
    }
    c->op_applies++;
    CK(cudaMemsetAsync(c->task_active, 0, sizeof(int) * c->T, c->stream));
    CK(cudaMemsetAsync(c->counters, 0, sizeof(int) * 2, c->stream));
    CK(launch_cg_init(c, 1));
    c->capsel = 1;                     // the sweeps' own step cap
    cmcs_status s = run_cg(c, 0);
    c->capsel = 0;
    if (s != CMCS_OK) return s;
    CK(cudaMemsetAsync(c->counters + 1, 0, sizeof(int), c->stream));
    CK(launch_refine_update(c));
    s = read_counters(c);
    if (s != CMCS_OK) return s;
    if (c->prof_on) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->res_ev[0], c->res_ev[1]) == cudaSuccess) c->res_ms += ms;
      else cudaGetLastError();
    }
    if (c->hcounters[1] == 0) break;
  }
  return CMCS_OK;
}

cmcs_status estep(Ctx* c) {
  CK(cudaMemsetAsync(c->task_active, 0, sizeof(int) * c->T, c->stream));
  CK(cudaMemsetAsync(c->counters, 0, sizeof(int) * 4, c->stream));
  CK(cudaMemsetAsync(c->psteps, 0, sizeof(int) * (size_t)c->T * c->C * c->K, c->stream));
  c->op_applies = 0;
  CK(launch_precond(c));              // Jacobi preconditioner of the current alpha
  // warm start: the mean systems solve for a correction to the previous means, from the
  // compensated residual b0 - A mu_prev
  const int warm = c->warm_start && c->have_prev;
  c->have_prev = 0;                   // set again once this E-step has completed
  if (warm) {
    CK(launch_residual(c, c->xacc, nullptr, c->r, 1, 1));
    c->op_applies++;
  }
  // first solve: Alg. 1 from x = 0 on b0 and the probes, recording gamma and xi (with
  // CMCS_BF16_MIXED, Phi held as one BF16 plane)
  CK(launch_cg_init(c, 0, warm));
  c->first_solve = 1;
  cmcs_status s = run_cg(c, 1);
  c->first_solve = 0;
  if (s != CMCS_OK) return s;
  if (warm) CK(launch_add_means(c));  // mu = mu_prev + delta
  CK(cudaMemcpyAsync(c->steps0, c->steps, sizeof(int) * c->S, cudaMemcpyDeviceToDevice, c->stream));
  // the Lanczos coefficients are final: their eigen step (Eqs. 9-11) runs on the side stream,
  // overlapping the refinement sweeps
  CK(cudaEventRecord(c->ev_fork, c->stream));
  CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
  CK(launch_quadrature_ctx(c, c->side));
  CK(cudaEventRecord(c->ev_join, c->side));
  // the solution moves to xacc by copy, so captured graphs keep valid buffer addresses
  CK(cudaMemcpyAsync(c->xacc, c->x, sizeof(float) * (size_t)c->S * c->Dp, cudaMemcpyDeviceToDevice,
                     c->stream));
  // refinement sweeps: residual with compensated products (FP64 combine), CG on it, add
  s = refine_sweeps(c, nullptr);
  if (s != CMCS_OK) return s;
  const float* rmu = nullptr;
  if (c->refine_max > 0) {
    // residual of the returned means: verified accuracy and the correction of ell
    CK(cudaMemsetAsync(c->rres, 0, sizeof(float) * c->S, c->stream));
    CK(launch_residual(c, c->xacc, nullptr, c->r, 1, 1));
    CK(launch_resid_norm(c));
    rmu = c->r;
  } else {
    CK(cudaMemsetAsync(c->rres, 0, sizeof(float) * c->S, c->stream));
  }
  CK(launch_sest(c));
  CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  CK(launch_ell_softmax(c, rmu));
  s = read_counters(c);
  if (s != CMCS_OK) return s;
  c->last_diverged = c->hcounters[3];
  fold_events(c);
  if (c->hcounters[2] != 0) {
    set_err(c, "non-finite value or eigen failure in the E-step (flags 0x%x)", c->hcounters[2]);
    c->have_prev = 0;
    return CMCS_ERR_NUMERIC;
  }
  c->have_prev = 1;
  return CMCS_OK;
}

// time one operator application of every variant (after one warm-up) on the context's own
// buffers and keep the fastest: SIMT tile width TN, or tensor-core pipeline depth
cmcs_status autotune(Ctx* c) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<int> cands;
  if (c->tc) {
    for (int st = 2; st <= tc_max_stages(c); ++st) cands.push_back(st);
  } else {
    for (int tn : {3, 4, 6, 8, 9}) cands.push_back(tn);
  }
  float best = 1e30f;
  int best_v = cands.empty() ? 0 : cands.back();
  for (int v : cands) {
    if (c->tc) tc_set_stages(c, v);
    else c->tn_plain = v;
    cudaError_t e = launch_operator(c, c->d, c->ad, 0);
    cudaEventRecord(e0, c->stream);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = launch_operator(c, c->d, c->ad, 0);
    cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      set_err(c, "autotune: %s", cudaGetErrorString(e));
      return CMCS_ERR_CUDA;
    }
    if (ms < best) {
      best = ms;
      best_v = v;
    }
  }
  if (c->tc) tc_set_stages(c, best_v);
  else c->tn_plain = best_v;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return CMCS_OK;
}

cmcs_status validate(const cmcs_config* cfg) {
  if (!cfg) return CMCS_ERR_INVALID_ARG;
  if (cfg->T < 1 || cfg->C < 1 || cfg->D < 1 || cfg->K < 1) return CMCS_ERR_INVALID_ARG;
  if (!cfg->N || !cfg->pi) return CMCS_ERR_INVALID_ARG;
  if (!(cfg->beta > 0.0) || !isfinite(cfg->beta)) return CMCS_ERR_INVALID_ARG;
  if (cfg->cg_max_iter < 1 || cfg->cg_max_iter > 512) return CMCS_ERR_INVALID_ARG;
  if (!(cfg->cg_tol >= 0.0)) return CMCS_ERR_INVALID_ARG;
  if (cfg->precision != CMCS_FP32 && cfg->precision != CMCS_BF16_REFINE &&
      cfg->precision != CMCS_BF16X3 && cfg->precision != CMCS_BF16_MIXED)
    return CMCS_ERR_INVALID_ARG;
  if (cfg->refine_max < 0 || cfg->refine_max > 64) return CMCS_ERR_INVALID_ARG;
  if (!(cfg->refine_tol >= 0.0)) return CMCS_ERR_INVALID_ARG;
  if (!(cfg->alpha_min > 0.0) || !(cfg->alpha_max > cfg->alpha_min) || !isfinite(cfg->alpha_max))
    return CMCS_ERR_INVALID_ARG;
  double ps = 0.0;
  for (int c = 0; c < cfg->C; ++c) {
    if (!(cfg->pi[c] > 0.0)) return CMCS_ERR_INVALID_ARG;
    ps += cfg->pi[c];
  }
  if (fabs(ps - 1.0) > 1e-6) return CMCS_ERR_INVALID_ARG;
  for (int t = 0; t < cfg->T; ++t)
    if (cfg->N[t] < 1 || cfg->N[t] > (1 << 24)) return CMCS_ERR_INVALID_ARG;
  if ((int64_t)cfg->C * (cfg->K + 1) > 4096) return CMCS_ERR_INVALID_ARG;
  if (cfg->schedule != 0 && cfg->schedule != 1) return CMCS_ERR_INVALID_ARG;
  if (cfg->graphs != 0 && cfg->graphs != 1) return CMCS_ERR_INVALID_ARG;
  if (cfg->autotune != 0 && cfg->autotune != 1) return CMCS_ERR_INVALID_ARG;
  if (cfg->learn_pi != 0 && cfg->learn_pi != 1) return CMCS_ERR_INVALID_ARG;
  if (cfg->probe_share != 0 && cfg->probe_share != 1) return CMCS_ERR_INVALID_ARG;
  if (cfg->precond != 0 && cfg->precond != 1) return CMCS_ERR_INVALID_ARG;
  if (cfg->warm_start != 0 && cfg->warm_start != 1) return CMCS_ERR_INVALID_ARG;
  if (cfg->task_offset < 0 || cfg->T_total < 0) return CMCS_ERR_INVALID_ARG;
  if (cfg->refine_steps < 0 || cfg->refine_steps > cfg->cg_max_iter) return CMCS_ERR_INVALID_ARG;
  const int64_t ttot = cfg->T_total == 0 ? cfg->T : cfg->T_total;
  if ((int64_t)cfg->task_offset + cfg->T > ttot) return CMCS_ERR_INVALID_ARG;
  if (ttot * cfg->C >= ((int64_t)1 << 31)) return CMCS_ERR_INVALID_ARG;   // probe counter word
  return CMCS_OK;
}

}  // namespace

namespace cmcs {
// error text reported by cmcs_last_error(NULL) for calls that have no context
void set_global_error(const char* msg) { snprintf(g_create_err, sizeof(g_create_err), "%s", msg); }
}  // namespace cmcs

extern "C" {

namespace {

// one context for dense Phi (mask == NULL) or for the structured Phi_t = Omega_t F (Phi == NULL)
cmcs_status create_ctx(const cmcs_config* cfg, const float* Phi, const float* y,
                       const uint8_t* mask, int on_device, void* stream, cmcs_ctx** out) {
  Ctx* c = nullptr;
  if (!out) {
    set_err(nullptr, "out is NULL");
    return CMCS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (validate(cfg) != CMCS_OK || (!Phi && !mask) || !y || (on_device != 0 && on_device != 1)) {
    set_err(nullptr, "invalid configuration or null input");
    return CMCS_ERR_INVALID_ARG;
  }
  if (mask && (cfg->precision != CMCS_FP32 || !dft_size_ok(cfg->D))) {
    set_err(nullptr, "the Fourier operator needs precision CMCS_FP32 and D either a power of two "
                     "in [128, %d] or D = 2^a 5^b with 16 | D, up to %d", kDftMaxD, kDftMaxLarge);
    return CMCS_ERR_UNSUPPORTED;
  }
  cmcs_ctx* h = static_cast<cmcs_ctx*>(calloc(1, sizeof(cmcs_ctx)));
  if (!h) {
    set_err(nullptr, "host allocation failed");
    return CMCS_ERR_OOM;
  }
  c = &h->c;
  c->T = cfg->T;
  c->C = cfg->C;
  c->D = cfg->D;
  c->K = cfg->K;
  c->R = cfg->C * (cfg->K + 1);
  c->S = cfg->T * c->R;
  c->Dp = (int)round_up(cfg->D, kDAlign);
  c->U = cfg->cg_max_iter;
  {
    const char* cv = getenv("CMCS_CG_CHUNK");
    const int ch = cv ? atoi(cv) : kCheckEvery;
    c->chunk = (ch >= 1 && ch <= 64) ? ch : kCheckEvery;
  }
  c->refine_steps = cfg->refine_steps == 0 ? cfg->cg_max_iter : cfg->refine_steps;
  c->beta = cfg->beta;
  c->cg_tol = cfg->cg_tol;
  c->refine_tol = cfg->refine_tol;
  c->refine_max = cfg->refine_max;
  c->alpha_min = cfg->alpha_min;
  c->alpha_max = cfg->alpha_max;
  c->precision = cfg->precision;
  c->learn_pi = cfg->learn_pi;
  c->pshare = cfg->probe_share;
  c->precond = cfg->precond;
  c->warm_start = cfg->warm_start;
  c->seed = cfg->seed;
  c->toff = cfg->task_offset;
  c->T_total = cfg->T_total == 0 ? cfg->T : cfg->T_total;
  c->mterm_w = cfg->C * (cfg->D + 1) + 1;
  c->op = mask ? 1 : 0;
  c->em_iter = 0;
  c->stream = static_cast<cudaStream_t>(stream);
  c->per_task = cfg->schedule;
  c->use_graphs = cfg->graphs;
  c->hN = static_cast<int64_t*>(malloc(sizeof(int64_t) * c->T));
  c->hNp = static_cast<int64_t*>(malloc(sizeof(int64_t) * c->T));
  c->hrow = static_cast<int64_t*>(malloc(sizeof(int64_t) * (c->T + 1)));
  c->hpi = static_cast<double*>(malloc(sizeof(double) * c->C));
  if (!c->hN || !c->hNp || !c->hrow || !c->hpi) {
    free_ctx(c);
    free(h);
    set_err(nullptr, "host allocation failed");
    return CMCS_ERR_OOM;
  }
  c->horow = static_cast<int64_t*>(malloc(sizeof(int64_t) * (c->T + 1)));
  if (!c->horow) {
    free_ctx(c);
    free(h);
    set_err(nullptr, "host allocation failed");
    return CMCS_ERR_OOM;
  }
  c->hrow[0] = 0;
  c->horow[0] = 0;
  // rows of the measurement vector: N_t, or 2 N_t real values [Re y_t; Im y_t] for Fourier
  const int64_t rowmul = mask ? 2 : 1;
  for (int t = 0; t < c->T; ++t) {
    c->horow[t + 1] = c->horow[t] + rowmul * cfg->N[t];
    c->hN[t] = rowmul * cfg->N[t];
    c->hNp[t] = round_up(c->hN[t], kNAlign);
    c->hrow[t + 1] = c->hrow[t] + c->hNp[t];
  }
  for (int k = 0; k < c->C; ++k) c->hpi[k] = cfg->pi[k];
  c->rows_total = c->hrow[c->T];

  cmcs_status st = CMCS_OK;
  auto fail = [&](cmcs_status s) {
    char msg[512];
    memcpy(msg, c->err, sizeof(msg));
    free_ctx(c);
    free(h);
    snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
    return s;
  };
#define CKC(call)                                                                  \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess) {                                                       \
      set_err(c, "%s failed: %s", #call, cudaGetErrorString(_e));                  \
      return fail(_e == cudaErrorMemoryAllocation ? CMCS_ERR_OOM : CMCS_ERR_CUDA);  \
    }                                                                              \
  } while (0)

  CKC(cudaGetDevice(&c->device));
  if (c->stream == nullptr) {
    // a blocking stream of our own: ordered with the legacy stream, and capturable
    CKC(cudaStreamCreate(&c->stream));
    c->own_stream = 1;
  }
  CKC(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CKC(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CKC(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CKC(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
  const int64_t Dp = c->Dp, S = c->S, T = c->T, C = c->C, K = c->K;
  const int64_t ntiles = c->rows_total / 128;
  if (!mask) CKC(dalloc(&c->phi, (size_t)(c->rows_total * Dp)));
  CKC(dalloc(&c->y, (size_t)c->rows_total));
  CKC(dalloc(&c->drow, (size_t)(T + 1)));
  CKC(dalloc(&c->dN, (size_t)T));
  CKC(dalloc(&c->tile_task, (size_t)ntiles));
  CKC(dalloc(&c->b0hi, (size_t)(T * Dp)));
  CKC(dalloc(&c->b0lo, (size_t)(T * Dp)));
  CKC(dalloc(&c->alpha, (size_t)(C * Dp)));
  CKC(dalloc(&c->sumlogalpha, (size_t)C));
  CKC(dalloc(&c->logpi, (size_t)C));
  CKC(dalloc(&c->pi, (size_t)C));
  if (c->precond) {
    CKC(dalloc(&c->colnorm, (size_t)(T * Dp)));
    CKC(dalloc(&c->pminv, (size_t)(T * C * Dp)));
    CKC(dalloc(&c->pw, (size_t)(T * C * Dp)));
    CKC(dalloc(&c->sumlogm, (size_t)(T * C)));
    CKC(cudaMemsetAsync(c->colnorm, 0, sizeof(float) * T * Dp, c->stream));
  }
  CKC(dalloc(&c->tconst, (size_t)T));
  CKC(dalloc(&c->x, (size_t)(S * Dp)));
  CKC(dalloc(&c->r, (size_t)(S * Dp)));
  CKC(dalloc(&c->d, (size_t)(S * Dp)));
  CKC(dalloc(&c->ad, (size_t)(S * Dp)));
  CKC(dalloc(&c->xacc, (size_t)(S * Dp)));
  CKC(dalloc(&c->w, (size_t)(c->R * c->rows_total)));
  CKC(dalloc(&c->wlo, (size_t)(c->R * c->rows_total)));
  CKC(dalloc(&c->part, (size_t)((Dp / 128) * S)));
  CKC(dalloc(&c->rr, (size_t)S));
  CKC(dalloc(&c->bb, (size_t)S));
  CKC(dalloc(&c->steps, (size_t)S));
  CKC(dalloc(&c->steps0, (size_t)S));
  CKC(dalloc(&c->active, (size_t)S));
  CKC(dalloc(&c->ractive, (size_t)S));
  CKC(dalloc(&c->sweeps, (size_t)S));
  CKC(dalloc(&c->rrel, (size_t)S));
  CKC(dalloc(&c->rres, (size_t)S));
  CKC(cudaMemsetAsync(c->rres, 0, sizeof(float) * S, c->stream));
  CKC(dalloc(&c->task_active, (size_t)T));
  CKC(dalloc(&c->counters, 5));
  CKC(cudaMallocHost(reinterpret_cast<void**>(&c->hcounters), 5 * sizeof(int)));
  CKC(dalloc(&c->gam, (size_t)(T * C * K * c->U)));
  CKC(dalloc(&c->xi, (size_t)(T * C * K * c->U)));
  CKC(dalloc(&c->psteps, (size_t)(T * C * K)));
  CKC(dalloc(&c->sest, (size_t)(T * C * Dp)));
  CKC(dalloc(&c->quad, (size_t)(T * C * K)));
  CKC(dalloc(&c->logdet, (size_t)(T * C)));
  CKC(dalloc(&c->ell, (size_t)(T * C)));
  CKC(dalloc(&c->q, (size_t)(T * C)));
  CKC(dalloc(&c->assign, (size_t)T));
  CKC(dalloc(&c->stats, 4));
  CKC(dalloc(&c->lltask, (size_t)T));
  CKC(dalloc(&c->mterms, (size_t)c->T_total * (size_t)c->mterm_w));
  CKC(dalloc(&c->opcount, (size_t)(2 * T)));   // [all-plane applications][one-plane ones]
  CKC(dalloc(&c->dorow, (size_t)(T + 1)));
  CKC(dalloc(&c->stall_flag, 1));
  CKC(cudaMemsetAsync(c->stall_flag, 0, sizeof(int), c->stream));
  CKC(dalloc(&c->adj_g, (size_t)(T * C * Dp)));
  CKC(dalloc(&c->adj_x, (size_t)(T * C * Dp)));
  CKC(dalloc(&c->adj_wl, (size_t)(C * c->rows_total)));
  CKC(dalloc(&c->adj_wm, (size_t)(C * c->rows_total)));
  CKC(dalloc(&c->adj_wl_lo, (size_t)(C * c->rows_total)));
  CKC(dalloc(&c->adj_wm_lo, (size_t)(C * c->rows_total)));
  CKC(dalloc(&c->adj_dy, (size_t)c->hrow[c->T]));
  CKC(dalloc(&c->adj_da, (size_t)(C * Dp)));
  CKC(cudaMemsetAsync(c->opcount, 0, sizeof(int64_t) * 2 * T, c->stream));

  // zero everything that padding relies on
  if (!mask) CKC(cudaMemsetAsync(c->phi, 0, sizeof(float) * c->rows_total * Dp, c->stream));
  CKC(cudaMemsetAsync(c->y, 0, sizeof(float) * c->rows_total, c->stream));
  for (void* p : {(void*)c->x, (void*)c->r, (void*)c->d, (void*)c->ad, (void*)c->xacc})
    CKC(cudaMemsetAsync(p, 0, sizeof(float) * S * Dp, c->stream));
  CKC(cudaMemsetAsync(c->sest, 0, sizeof(float) * T * C * Dp, c->stream));
  CKC(cudaMemsetAsync(c->gam, 0, sizeof(float) * T * C * K * c->U, c->stream));
  CKC(cudaMemsetAsync(c->xi, 0, sizeof(float) * T * C * K * c->U, c->stream));
  CKC(cudaMemsetAsync(c->steps0, 0, sizeof(int) * S, c->stream));
  CKC(cudaMemsetAsync(c->sweeps, 0, sizeof(int) * S, c->stream));
  CKC(cudaMemsetAsync(c->rrel, 0, sizeof(float) * S, c->stream));
  CKC(cudaMemsetAsync(c->q, 0, sizeof(double) * T * C, c->stream));
  CKC(cudaMemsetAsync(c->stats, 0, sizeof(double) * 4, c->stream));

  // Phi and y into the padded layout (Fourier: the mask, spectra and stacked y)
  const cudaMemcpyKind kin = kind_in(on_device);
  if (mask) {
    CKC(cudaStreamSynchronize(c->stream));
    const int e = dft_create(c, mask, y, on_device);
    if (e == 5) {
      set_err(c, "the mask's sampled frequencies per task differ from N");
      return fail(CMCS_ERR_INVALID_ARG);
    }
    if (e != 0) {
      set_err(c, "Fourier operator set-up failed (%d): %s", e, cudaGetErrorString(cudaGetLastError()));
      return fail(CMCS_ERR_CUDA);
    }
  }
  int64_t src_row = 0;
  for (int t = 0; !mask && t < c->T; ++t) {
    CKC(cudaMemcpy2DAsync(c->phi + c->hrow[t] * Dp, sizeof(float) * Dp, Phi + src_row * c->D,
                          sizeof(float) * c->D, sizeof(float) * c->D, (size_t)c->hN[t], kin,
                          c->stream));
    CKC(cudaMemcpyAsync(c->y + c->hrow[t], y + src_row, sizeof(float) * c->hN[t], kin, c->stream));
    src_row += c->hN[t];
  }
  std::vector<int> ttask((size_t)ntiles);
  for (int t = 0; t < c->T; ++t)
    for (int64_t g = c->hrow[t] / 128; g < c->hrow[t + 1] / 128; ++g) ttask[(size_t)g] = t;
  std::vector<double> lpi((size_t)C);
  for (int k = 0; k < C; ++k) lpi[(size_t)k] = log(c->hpi[k]);
  CKC(cudaMemcpyAsync(c->drow, c->hrow, sizeof(int64_t) * (T + 1), cudaMemcpyHostToDevice, c->stream));
  CKC(cudaMemcpyAsync(c->dN, c->hN, sizeof(int64_t) * T, cudaMemcpyHostToDevice, c->stream));
  CKC(cudaMemcpyAsync(c->dorow, c->horow, sizeof(int64_t) * (T + 1), cudaMemcpyHostToDevice, c->stream));
  CKC(cudaMemcpyAsync(c->tile_task, ttask.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice, c->stream));
  CKC(cudaMemcpyAsync(c->logpi, lpi.data(), sizeof(double) * C, cudaMemcpyHostToDevice, c->stream));
  CKC(cudaMemcpyAsync(c->pi, c->hpi, sizeof(double) * C, cudaMemcpyHostToDevice, c->stream));
  CKC(launch_b0(c));
  CKC(launch_colnorm(c));
  CKC(launch_alpha_init(c));
  CKC(launch_sumlogalpha(c));
  CKC(launch_tconst_dev(c, c->dN));
  if (c->precision == CMCS_BF16_REFINE || c->precision == CMCS_BF16X3 ||
      c->precision == CMCS_BF16_MIXED) {
    if (tc_create(c) != 0) {
      if (c->err[0] == 0) set_err(c, "BF16 tensor-core operator unavailable");
      return fail(CMCS_ERR_UNSUPPORTED);
    }
    // the refinement residual on the tensor cores (digit planes of Phi); CMCS_OZ=0 keeps the
    // double-single SIMT residual (evaluation switch)
    const char* ov = getenv("CMCS_OZ");
    if ((ov == nullptr || atoi(ov) != 0) && oz_create(c) != 0) {
      if (c->err[0] == 0) set_err(c, "tensor-core residual unavailable");
      return fail(CMCS_ERR_UNSUPPORTED);
    }
  }
  CKC(cudaStreamSynchronize(c->stream));
  CKC(cudaGetLastError());
  if (cfg->autotune && !mask) {
    st = autotune(c);
    if (st != CMCS_OK) return fail(st);
  }
  c->tuned = c->tc ? tc_set_stages(c, 0) : (c->tn_plain > 0 ? c->tn_plain : pick_tn(c->R, 9));
#undef CKC
  *out = h;
  return CMCS_OK;
}

}  // namespace

cmcs_status cmcs_create(const cmcs_config* cfg, const float* Phi, const float* y, int on_device,
                        void* stream, cmcs_ctx** out) {
  if (!Phi) {
    if (out) *out = nullptr;
    set_err(nullptr, "invalid configuration or null input");
    return CMCS_ERR_INVALID_ARG;
  }
  return create_ctx(cfg, Phi, y, nullptr, on_device, stream, out);
}

cmcs_status cmcs_create_dft(const cmcs_config* cfg, const uint8_t* mask, const float* y,
                            int on_device, void* stream, cmcs_ctx** out) {
  if (!mask) {
    if (out) *out = nullptr;
    set_err(nullptr, "invalid configuration or null input");
    return CMCS_ERR_INVALID_ARG;
  }
  return create_ctx(cfg, nullptr, y, mask, on_device, stream, out);
}

void cmcs_destroy(cmcs_ctx* h) {
  if (!h) return;
  cudaStreamSynchronize(h->c.stream);
  free_ctx(&h->c);
  free(h);
}

const char* cmcs_last_error(const cmcs_ctx* h) { return h ? h->c.err : g_create_err; }

cmcs_status cmcs_test_stall(cmcs_ctx* h, int enable) {
  if (!h || (enable != 0 && enable != 1)) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  if (c->tc == nullptr) {
    set_err(c, "cmcs_test_stall: only the tensor-core operator has device-side waits");
    return CMCS_ERR_UNSUPPORTED;
  }
  CK(cudaMemcpyAsync(c->stall_flag, &enable, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  return sync_check(c);
}

cmcs_status cmcs_profile(cmcs_ctx* h, int enable) {
  if (!h || (enable != 0 && enable != 1)) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  if (enable) {
    if (!c->prof_ev) {
      c->prof_ev = static_cast<cudaEvent_t*>(calloc(2 * kProfEvents, sizeof(cudaEvent_t)));
      c->prof_tag = static_cast<unsigned char*>(calloc(kProfEvents, 1));
      if (!c->prof_tag) {
        set_err(c, "host allocation failed");
        return CMCS_ERR_OOM;
      }
      if (!c->prof_ev) return CMCS_ERR_OOM;
      for (int i = 0; i < 2 * kProfEvents; ++i) CK(cudaEventCreate(&c->prof_ev[i]));
      CK(cudaEventCreate(&c->res_ev[0]));
      CK(cudaEventCreate(&c->res_ev[1]));
    }
    CK(cudaMemsetAsync(c->opcount, 0, sizeof(int64_t) * 2 * c->T, c->stream));
    c->prof_nev = 0;
    c->prof_calls = c->res_calls = c->launches = c->prof_calls1 = 0;
    c->prof_ms = c->res_ms = c->prof_ms1 = 0.0;
  }
  c->prof_on = enable;
  return sync_check(c);
}

cmcs_status cmcs_profile_read(const cmcs_ctx* hc, cmcs_profile_data* out) {
  if (!hc || !out) return CMCS_ERR_INVALID_ARG;
  Ctx* c = const_cast<Ctx*>(&hc->c);
  std::vector<int64_t> cnt(2 * (size_t)c->T);
  CK(cudaMemcpyAsync(cnt.data(), c->opcount, sizeof(int64_t) * 2 * c->T, cudaMemcpyDeviceToHost,
                     c->stream));
  cmcs_status s = sync_check(c);
  if (s != CMCS_OK) return s;
  fold_events(c);
  double fl = 0.0, by = 0.0;
  for (int t = 0; t < c->T; ++t) {
    const double n = (double)c->hN[t], D = (double)c->D, R = (double)c->R;
    if (c->op == 1 && c->dft_large) {
      // the operator alone (three four-step launches): a forward and an inverse complex
      // transform (5 D log2 D each) per two systems, mask and scaling; d read, A d written,
      // the mask
      fl += (double)cnt[t] * R * (5.0 * D * log2(D) + 4.0 * D);
      by += (double)cnt[t] * (8.0 * R * D + 4.0 * D);
    } else if (c->op == 1) {
      // one CG step fused with the operator: one complex FFT pair (5 D log2 D each) per two
      // systems plus the update; d, x, r read, x, r, d written, the mask
      fl += (double)cnt[t] * R * (5.0 * D * (double)c->dft_L + 12.0 * D);
      by += (double)cnt[t] * (24.0 * R * D + 4.0 * D);
    } else {
      // Phi counted once per application: 4 bytes per element as FP32 or a BF16 pair (first
      // T counters), 2 as one BF16 plane (second T counters)
      const double a4 = (double)cnt[(size_t)t], a2 = (double)cnt[(size_t)c->T + t];
      fl += (a4 + a2) * 4.0 * n * D * R;
      by += a4 * 4.0 * n * D + a2 * 2.0 * n * D + (a4 + a2) * 4.0 * R * (2.0 * D + 2.0 * n);
    }
  }
  out->operator_calls = c->prof_calls;
  out->operator_ms = c->prof_ms;
  out->operator_flops = fl;
  out->operator_bytes = by;
  out->residual_calls = c->res_calls;
  out->residual_ms = c->res_ms;
  out->kernel_launches = c->launches;
  out->operator_calls_bf16 = c->prof_calls1;
  out->operator_ms_bf16 = c->prof_ms1;
  return CMCS_OK;
}

cmcs_status cmcs_set_alpha(cmcs_ctx* h, const float* alpha, int on_device, int64_t em_iter) {
  if (!h || !alpha || (on_device != 0 && on_device != 1) || em_iter < 0) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  std::vector<float> tmp((size_t)c->C * c->D);
  if (on_device) {
    CK(cudaMemcpy(tmp.data(), alpha, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost));
  } else {
    memcpy(tmp.data(), alpha, sizeof(float) * tmp.size());
  }
  for (float v : tmp)
    if (!(v > 0.f) || !isfinite(v)) {
      set_err(c, "alpha must be positive and finite");
      return CMCS_ERR_INVALID_ARG;
    }
  CK(cudaMemcpy2DAsync(c->alpha, sizeof(float) * c->Dp, tmp.data(), sizeof(float) * c->D,
                       sizeof(float) * c->D, (size_t)c->C, cudaMemcpyHostToDevice, c->stream));
  CK(launch_sumlogalpha(c));
  c->em_iter = em_iter;
  return sync_check(c);
}

cmcs_status cmcs_set_data(cmcs_ctx* h, const float* Phi, const float* y, int on_device) {
  if (!h || !Phi || !y || (on_device != 0 && on_device != 1)) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  if (c->op == 1) {
    set_err(c, "cmcs_set_data: not available for the Fourier operator");
    return CMCS_ERR_UNSUPPORTED;
  }
  const cudaMemcpyKind kin = kind_in(on_device);
  int64_t src_row = 0;
  for (int t = 0; t < c->T;) {
    if (c->D == c->Dp) {
      // unpadded rows: consecutive tasks without padding rows are one contiguous block on both
      // sides, copied in one piece
      int t1 = t + 1;
      int64_t rows = c->hN[t];
      while (c->hN[t1 - 1] == c->hNp[t1 - 1] && t1 < c->T) rows += c->hN[t1++];
      CK(cudaMemcpyAsync(c->phi + c->hrow[t] * c->Dp, Phi + src_row * c->D, sizeof(float) * rows * c->D,
                         kin, c->stream));
      for (int u = t; u < t1; ++u) {
        CK(cudaMemcpyAsync(c->y + c->hrow[u], y + src_row, sizeof(float) * c->hN[u], kin, c->stream));
        src_row += c->hN[u];
      }
      t = t1;
      continue;
    }
    CK(cudaMemcpy2DAsync(c->phi + c->hrow[t] * c->Dp, sizeof(float) * c->Dp, Phi + src_row * c->D,
                         sizeof(float) * c->D, sizeof(float) * c->D, (size_t)c->hN[t], kin, c->stream));
    CK(cudaMemcpyAsync(c->y + c->hrow[t], y + src_row, sizeof(float) * c->hN[t], kin, c->stream));
    src_row += c->hN[t];
    ++t;
  }
  CK(launch_b0(c));
  CK(launch_tconst_dev(c, c->dN));
  CK(launch_colnorm(c));
  c->have_prev = 0;                   // the previous means belong to the old data
  if (c->tc != nullptr) CK(tc_refresh(c));
  if (c->oz != nullptr) CK(oz_refresh(c));
  return sync_check(c);
}

cmcs_status cmcs_adjoint(cmcs_ctx* h, const float* g, float* dy, float* dalpha, float* dPhi,
                         int on_device) {
  if (!h || !g || !dy || !dalpha || (on_device != 0 && on_device != 1)) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  if (c->op == 1) {
    set_err(c, "cmcs_adjoint: not available for the Fourier operator");
    return CMCS_ERR_UNSUPPORTED;
  }
  const size_t D = c->D, Dp = c->Dp, T = c->T, C = c->C;
  // the adjoint systems A_tc lambda_tc = g_tc as a narrow problem: R = C columns per task, K = 0,
  // FP32 operator and compensated refinement; its solution goes to adj_x, not to the means
  const int64_t launches0 = c->launches;
  Ctx a = *c;
  a.R = c->C;
  a.K = 0;
  a.S = c->T * c->C;
  a.tc = nullptr;
  a.oz = nullptr;                     // the tensor-core residual's buffers are sized for R systems
  a.dhi = a.dlo = nullptr;
  a.prof_on = 0;
  a.xacc = c->adj_x;
  a.tn_plain = a.tn_ds = 0;
  a.use_graphs = 0;
  CK(cudaMemsetAsync(c->adj_g, 0, sizeof(float) * T * C * Dp, c->stream));
  CK(cudaMemcpy2DAsync(c->adj_g, sizeof(float) * Dp, g, sizeof(float) * D, sizeof(float) * D, T * C,
                       kind_in(on_device), c->stream));
  CK(cudaMemcpyAsync(a.r, c->adj_g, sizeof(float) * T * C * Dp, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemsetAsync(c->task_active, 0, sizeof(int) * T, c->stream));
  CK(cudaMemsetAsync(c->counters, 0, sizeof(int) * 4, c->stream));
  CK(launch_precond(c));              // the adjoint systems (t, c) share A_tc's preconditioner
  CK(launch_cg_init(&a, 2));
  cmcs_status s = run_cg(&a, 0);
  if (s != CMCS_OK) return s;
  CK(cudaMemcpyAsync(a.xacc, a.x, sizeof(float) * T * C * Dp, cudaMemcpyDeviceToDevice, c->stream));
  s = refine_sweeps(&a, c->adj_g);
  if (s != CMCS_OK) return s;
  // gradients
  // Phi lambda and Phi mu as compensated pairs (see k_adj_dy)
  CK(launch_phi_v(&a, c->adj_x, c->adj_wl, c->adj_wl_lo, (int)C, 1));
  CK(launch_phi_v(c, c->xacc, c->adj_wm, c->adj_wm_lo, (int)C, c->K + 1));
  CK(launch_adj_dy(c, c->adj_wl, c->adj_wl_lo, c->adj_dy));
  CK(launch_adj_dalpha(c, c->adj_x, c->adj_da));
  const cudaMemcpyKind kout = kind_out(on_device);
  CK(cudaMemcpyAsync(dy, c->adj_dy, sizeof(float) * c->horow[c->T], kout, c->stream));
  CK(cudaMemcpy2DAsync(dalpha, sizeof(float) * D, c->adj_da, sizeof(float) * Dp, sizeof(float) * D,
                       C, kout, c->stream));
  if (dPhi != nullptr) {
    if (on_device) {
      CK(launch_adj_dphi(c, c->adj_x, c->adj_wl, c->adj_wl_lo, c->adj_wm, c->adj_wm_lo, dPhi, 0,
                         c->rows_total, 0));
    } else {
      // stage row blocks in the work buffer ad (S * Dp floats) and copy each out
      const int64_t m = (int64_t)(((size_t)c->S * Dp) / D);
      for (int t = 0; t < c->T; ++t) {
        for (int64_t i = 0; i < c->hN[t]; i += m) {
          const int64_t nr = c->hN[t] - i < m ? c->hN[t] - i : m;
          CK(launch_adj_dphi(c, c->adj_x, c->adj_wl, c->adj_wl_lo, c->adj_wm, c->adj_wm_lo, c->ad,
                             c->hrow[t] + i, c->hrow[t] + i + nr, c->horow[t] + i));
          CK(cudaMemcpyAsync(dPhi + (c->horow[t] + i) * D, c->ad, sizeof(float) * nr * D,
                             cudaMemcpyDeviceToHost, c->stream));
        }
      }
    }
  }
  c->launches += a.launches - launches0;
  s = read_counters(c);
  if (s != CMCS_OK) return s;
  if (c->hcounters[2] != 0) {
    set_err(c, "non-finite value in the adjoint solve (flags 0x%x)", c->hcounters[2]);
    return CMCS_ERR_NUMERIC;
  }
  return CMCS_OK;
}

cmcs_status cmcs_estep(cmcs_ctx* h) {
  if (!h) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  cmcs_status s = estep(c);
  if (s != CMCS_OK) return s;
  return sync_check(c);
}

cmcs_status cmcs_em_iter(cmcs_ctx* h, int n) {
  if (!h || n < 0) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  if (c->T_total != c->T) {
    set_err(c, "the context holds tasks %d..%d of %d: its M-step needs every task's terms "
               "(cmcs_mstep_terms, then cmcs_mstep_apply with all rows)", c->toff,
            c->toff + c->T - 1, c->T_total);
    return CMCS_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) {
    cmcs_status s = estep(c);
    if (s != CMCS_OK) return s;
    CK(launch_mstep_terms(c));
    CK(launch_mstep_apply(c));
    CK(launch_sumlogalpha(c));
    c->em_iter++;
  }
  return sync_check(c);
}

cmcs_status cmcs_mstep_terms(cmcs_ctx* h, double* terms, int on_device) {
  if (!h || !terms || (on_device != 0 && on_device != 1)) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  CK(launch_mstep_terms(c));
  const size_t w = (size_t)c->mterm_w;
  CK(cudaMemcpyAsync(terms, c->mterms + (size_t)c->toff * w, sizeof(double) * w * c->T,
                     kind_out(on_device), c->stream));
  return sync_check(c);
}

cmcs_status cmcs_mstep_apply(cmcs_ctx* h, const double* terms, int on_device) {
  if (!h || !terms || (on_device != 0 && on_device != 1)) return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  CK(cudaMemcpyAsync(c->mterms, terms, sizeof(double) * (size_t)c->mterm_w * c->T_total,
                     kind_in(on_device), c->stream));
  CK(launch_mstep_apply(c));
  CK(launch_sumlogalpha(c));
  c->em_iter++;
  return sync_check(c);
}

cmcs_status cmcs_read(const cmcs_ctx* hc, int what, void* dst, int on_device) {
  if (!hc || !dst || (on_device != 0 && on_device != 1)) return CMCS_ERR_INVALID_ARG;
  Ctx* c = const_cast<Ctx*>(&hc->c);
  const cudaMemcpyKind k = kind_out(on_device);
  const size_t D = c->D, Dp = c->Dp, T = c->T, C = c->C, K = c->K;
  switch (what) {
    case CMCS_OUT_MU:
      CK(cudaMemcpy2DAsync(dst, sizeof(float) * D, c->xacc, sizeof(float) * Dp * (K + 1),
                           sizeof(float) * D, T * C, k, c->stream));
      break;
    case CMCS_OUT_S:
      CK(cudaMemcpy2DAsync(dst, sizeof(float) * D, c->sest, sizeof(float) * Dp, sizeof(float) * D,
                           T * C, k, c->stream));
      break;
    case CMCS_OUT_Q:
      CK(cudaMemcpyAsync(dst, c->q, sizeof(double) * T * C, k, c->stream));
      break;
    case CMCS_OUT_LOGDET:
      CK(cudaMemcpyAsync(dst, c->logdet, sizeof(double) * T * C, k, c->stream));
      break;
    case CMCS_OUT_ELL:
      CK(cudaMemcpyAsync(dst, c->ell, sizeof(double) * T * C, k, c->stream));
      break;
    case CMCS_OUT_ALPHA:
      CK(cudaMemcpy2DAsync(dst, sizeof(float) * D, c->alpha, sizeof(float) * Dp, sizeof(float) * D,
                           C, k, c->stream));
      break;
    case CMCS_OUT_ASSIGN:
      CK(cudaMemcpyAsync(dst, c->assign, sizeof(int) * T, k, c->stream));
      break;
    case CMCS_OUT_RECON: {
      std::vector<int> a(T);
      CK(cudaMemcpyAsync(a.data(), c->assign, sizeof(int) * T, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      for (size_t t = 0; t < T; ++t)
        CK(cudaMemcpyAsync(static_cast<float*>(dst) + t * D,
                           c->xacc + (t * c->R + (size_t)a[t] * (K + 1)) * Dp, sizeof(float) * D,
                           k, c->stream));
      break;
    }
    case CMCS_OUT_STEPS:
      CK(cudaMemcpyAsync(dst, c->steps0, sizeof(int) * c->S, k, c->stream));
      break;
    case CMCS_OUT_GAMMA:
      CK(cudaMemcpyAsync(dst, c->gam, sizeof(float) * T * C * K * c->U, k, c->stream));
      break;
    case CMCS_OUT_XI:
      CK(cudaMemcpyAsync(dst, c->xi, sizeof(float) * T * C * K * c->U, k, c->stream));
      break;
    case CMCS_OUT_B0:
      CK(cudaMemcpy2DAsync(dst, sizeof(float) * D, c->b0hi, sizeof(float) * Dp, sizeof(float) * D,
                           T, k, c->stream));
      break;
    case CMCS_OUT_SWEEPS:
      CK(cudaMemcpyAsync(dst, c->sweeps, sizeof(int) * c->S, k, c->stream));
      break;
    case CMCS_OUT_RESID:
      CK(cudaMemcpyAsync(dst, c->rres, sizeof(float) * c->S, k, c->stream));
      break;
    case CMCS_OUT_PI:
      CK(cudaMemcpyAsync(dst, c->pi, sizeof(double) * C, k, c->stream));
      break;
    default:
      set_err(c, "unknown output %d", what);
      return CMCS_ERR_INVALID_ARG;
  }
  return sync_check(c);
}

cmcs_status cmcs_result(const cmcs_ctx* hc, cmcs_summary* out) {
  if (!hc || !out) return CMCS_ERR_INVALID_ARG;
  Ctx* c = const_cast<Ctx*>(&hc->c);
  std::vector<int> st(c->S), sw(c->S);
  std::vector<float> rel(c->S), res(c->S);
  double stats[4];
  CK(cudaMemcpyAsync(res.data(), c->rres, sizeof(float) * c->S, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(st.data(), c->steps0, sizeof(int) * c->S, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(sw.data(), c->sweeps, sizeof(int) * c->S, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(rel.data(), c->rrel, sizeof(float) * c->S, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(stats, c->stats, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream));
  cmcs_status s = sync_check(c);
  if (s != CMCS_OK) return s;
  memset(out, 0, sizeof(*out));
  out->em_iters_done = c->em_iter;
  out->loglik = stats[0];
  out->min_margin = stats[1];
  double sum = 0.0;
  for (int i = 0; i < c->S; ++i) {
    out->cg_steps_max = st[i] > out->cg_steps_max ? st[i] : out->cg_steps_max;
    sum += st[i];
    if (st[i] >= c->U) out->cg_capped++;
    out->refine_sweeps_max = sw[i] > out->refine_sweeps_max ? sw[i] : out->refine_sweeps_max;
    out->refine_rel_max = rel[i] > out->refine_rel_max ? rel[i] : out->refine_rel_max;
    out->resid_rel_max = res[i] > out->resid_rel_max ? res[i] : out->resid_rel_max;
  }
  out->cg_steps_mean = sum / c->S;
  out->operator_applies = c->op_applies;
  out->refine_diverged = c->last_diverged;
  out->operator_variant = c->tuned;
  return CMCS_OK;
}

cmcs_status cmcs_apply(cmcs_ctx* h, const float* V, float* Z, int on_device, int accurate) {
  if (!h || !V || !Z || (on_device != 0 && on_device != 1) || (accurate != 0 && accurate != 1))
    return CMCS_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  const size_t D = c->D, Dp = c->Dp, S = c->S;
  const cudaMemcpyKind kin = kind_in(on_device), kout = kind_out(on_device);
  CK(cudaMemsetAsync(c->x, 0, sizeof(float) * S * Dp, c->stream));
  CK(cudaMemcpy2DAsync(c->x, sizeof(float) * Dp, V, sizeof(float) * D, sizeof(float) * D, S, kin,
                       c->stream));
  if (!accurate) {
    if (c->tc != nullptr) CK(tc_split_vectors(c, c->x));
    CK(launch_operator(c, c->x, c->ad, 0));
  } else {
    CK(cudaMemsetAsync(c->d, 0, sizeof(float) * S * Dp, c->stream));
    CK(cudaMemcpy2DAsync(c->d, sizeof(float) * Dp, Z, sizeof(float) * D, sizeof(float) * D, S, kin,
                         c->stream));
    CK(launch_residual(c, c->x, c->d, c->ad));
  }
  CK(cudaMemcpy2DAsync(Z, sizeof(float) * D, c->ad, sizeof(float) * Dp, sizeof(float) * D, S, kout,
                       c->stream));
  return sync_check(c);
}

cmcs_status cmcs_probes(const cmcs_ctx* hc, int64_t em_iter, float* dst, int on_device) {
  if (!hc || !dst || (on_device != 0 && on_device != 1) || em_iter < 0) return CMCS_ERR_INVALID_ARG;
  Ctx* c = const_cast<Ctx*>(&hc->c);
  const size_t n = (size_t)c->T * c->C * c->K * c->D;
  if (on_device) {
    CK(launch_probes_out(c, em_iter, dst));
  } else {
    CK(launch_probes_out(c, em_iter, c->ad));
    CK(cudaMemcpyAsync(dst, c->ad, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
  }
  return sync_check(c);
}

cmcs_status cmcs_lanczos_quadrature(const float* gamma, const float* xi, const int32_t* steps,
                                    int nsys, int ld, double* out, int32_t* status,
                                    void* stream) {
  if (!gamma || !xi || !steps || !out || !status || nsys < 0 || ld < 1 || ld > 512) {
    set_err(nullptr, "invalid argument to cmcs_lanczos_quadrature");
    return CMCS_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_quadrature(gamma, xi, steps, nsys, ld, out, status, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_err(nullptr, "CUDA error: %s", cudaGetErrorString(e));
    return CMCS_ERR_CUDA;
  }
  return CMCS_OK;
}

}  // extern "C"
