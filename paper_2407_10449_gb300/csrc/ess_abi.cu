// ess_abi.cu -- the extern "C" entry points declared in include/ess.h.
//
// Host-side orchestration only: validation, device buffers owned by the
// state, and the per-step launch sequence
//   [refresh p = A x]  ->  draw nu  ->  q = A nu  ->  chain step
// on the caller's stream.  All arithmetic of the step runs in the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "ess.h"
#include "ess_kernels.cuh"
#include "ess_gemm_tc.cuh"

using ess::DevStats;

namespace {

thread_local std::string g_err;

ess_status fail(ess_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

ess_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? ESS_ERR_OOM : ESS_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define ESS_CUDA(expr)                                 \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

template <typename T>
cudaError_t dev_alloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

template <typename T>
void dev_free(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

bool all_finite(const double* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

}  // namespace

// Lets the other entry-point files of the library report through ess_last_error.
void ess_internal_set_error(const std::string& msg) { g_err = msg; }

struct ess_state {
  int d = 0, m = 0;
  ess_config cfg{};
  int device = 0;
  int ld16 = 0;           // row stride of the 16-bit operands (d rounded up to 8)
  int chain_threads = 0;  // threads per chain of the step kernel
  int min_chain_threads = 0;  // the narrowest CTA width that holds m arcs
  // m beyond the CTA kernel's 8192 arcs: the wide-row kernel takes the chains
  // the warp kernel leaves (or every chain when sort_threads > 0)
  bool wide = false;
  // some b_i <= 0: the warp step drops arcs inside the union of those rows'
  // (long) arcs (ChainParams::long_arcs)
  int long_arcs = 0;
  void* wide_scratch = nullptr;  // wide_slots x 4 x wide_cap elements of T
  long long wide_cap = 0;
  int wide_slots = 0;
  int tuned_n = 0;            // chain count the autotuner last tuned for
  int sms = 0;                // SM count of the device
  // constants (device)
  double* A64 = nullptr;
  double* b64 = nullptr;
  double* anorm = nullptr;
  float* b32 = nullptr;
  double* bm_tab = nullptr;  // FP64 Box-Muller tables (ess::bm_table_fill)
  void* slack = nullptr;   // m thresholds b_i - margin ||a_i|| (T, rounded down)
  // work buffers (device), sized for `cap` chains
  int cap = 0;
  void* P = nullptr;       // n x m, T: p = A x of the current states
  void* P2 = nullptr;      // n x m, T: next p (double buffer; swapped after each step)
  int* ovf = nullptr;      // n + 2 ints: [0] count, [1] chain tickets of the streamed
                           // kernel, [2..] chains left to the CTA kernel
  int chain_kernel = ESS_CHAIN_AUTO;  // the float chain-step kernel (ess_set_chain_kernel)
  void* Q = nullptr;       // n x m, T
  void* NU = nullptr;      // n x d, T
  float* Xw = nullptr;     // n x d, mixed-form working states (the loaded chains)
  double* Xd = nullptr;    // n x d, FP64-form working states (the loaded chains)
  int n_loaded = 0;        // chains loaded by ess_chains_init
  int t_next = 0;          // global index of the next step of the loaded chains
  int p_fresh_t = -1;      // step index at which p was last recomputed from x
  long long host_steps = 0;  // chain-steps enqueued since the last stats reset
  __half* NU_h[2] = {nullptr, nullptr};  // scaled fp16 split of nu (tensor-core q)
  // second nu buffers: in a replayed refresh period the draw of step j + 1
  // runs on a low-priority side stream while step j's GEMM runs
  void* NU_alt = nullptr;
  __half* NU_h_alt[2] = {nullptr, nullptr};
  float* nu_unscale = nullptr;           // 1 / t_c of caller-supplied nu (scanned per chain)
  __nv_bfloat16* x_slices = nullptr;  // refresh: fixed-point slices of the states
  float* row_scale = nullptr;         // refresh: per-chain power-of-two scales
  double* P64 = nullptr;              // refresh: FP64 product for the start check
  DevStats* dstats = nullptr;
  int* dstatus = nullptr;
  ess::TcGemmPlan* tc_plan = nullptr;  // tensor-core GEMMs (q = A nu, exact refresh)
  // CUDA graphs of one refresh period (refresh + refresh_k steps), keyed by
  // chain count, seed and the p buffer the period starts from
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;   // graph capture: the steps (highest priority)
  cudaStream_t work_stream = nullptr;  // plain launches: the steps (highest priority)
  cudaStream_t side_stream = nullptr;  // the draws one step ahead (lowest priority)
  cudaEvent_t ev_drawn = nullptr, ev_done = nullptr, ev_fork = nullptr, ev_join = nullptr;
  unsigned* t_dev = nullptr;  // step index base of a replayed period
  struct GraphEntry {
    int n;
    uint64_t seed;
    void* p_first;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  long long graph_launches = 0;
  // optional per-phase device timing (CUDA events on the run's stream)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<int, int>>> ev_pending;  // phase, (start, stop) indices
  int ev_used = 0;
  double phase_ms[ESS_N_PHASES] = {0};
  long long phase_launches[ESS_N_PHASES] = {0};
  // ess_run_host: device copy of X, two sample slots whose copies to the host
  // overlap the next steps (on their own stream), kept across calls
  int host_cap = 0;
  double* host_x = nullptr;
  void* host_slot[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t slot_ready[2] = {nullptr, nullptr}, slot_free[2] = {nullptr, nullptr};
  // ess_run_few: buffers of the persistent few-chain kernel (kMaxFew chains)
  double* few_x = nullptr;    // 2 x kMaxFew x d
  double* few_nu = nullptr;   // 2 x kMaxFew x d
  double* few_p = nullptr;    // 2 x kMaxFew x m
  double* few_q = nullptr;    // kMaxFew x m
  double* few_short = nullptr; // 2 parities x kMaxFew x m x 2
  double* few_th = nullptr;   // 3 x kMaxFew: theta, cos, sin
  unsigned long long* few_bkt = nullptr;  // 2 parities x (min alpha, max beta) x kMaxFew x kFewBuckets
  int* few_int = nullptr;     // 9 x kMaxFew: rej[2], cur[2], nshort[2], bad[2], bad_prev
  unsigned* few_bar = nullptr;   // barrier (2) and abort flag (1)
};

namespace {

bool mixed(const ess_state* s) { return s->cfg.precision == ESS_PREC_MIXED; }
// FP64 form with its products from exact splits on the tensor cores
bool split64(const ess_state* s) {
  return s->cfg.precision == ESS_PREC_FP64 && s->cfg.fp64_products == ESS_PRODUCTS_SPLIT;
}
// bits of the fixed-point splits of the FP64 form's operands (a double's 53
// plus room for the per-row power-of-two scaling)
constexpr int kSplit64Bits = 56;

// Records an event for phase timing; returns its pool index or -1.
int timing_mark(ess_state* s, cudaStream_t st) {
  if (!s->timing) return -1;
  if (s->ev_used == (int)s->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    s->ev_pool.push_back(e);
  }
  const int i = s->ev_used++;
  if (cudaEventRecord(s->ev_pool[i], st) != cudaSuccess) return -1;
  return i;
}

// Phase timing scope: events around the launches of one phase.
struct PhaseScope {
  ess_state* s;
  cudaStream_t st;
  int phase, start;
  int launches;
  PhaseScope(ess_state* s_, cudaStream_t st_, int phase_, int launches_ = 1)
      : s(s_), st(st_), phase(phase_), start(timing_mark(s_, st_)), launches(launches_) {}
  ~PhaseScope() {
    s->phase_launches[phase] += launches;
    if (start < 0) return;
    const int stop = timing_mark(s, st);
    if (stop >= 0) s->ev_pending.push_back({phase, {start, stop}});
  }
};

// Folds the elapsed times of all recorded phases (call after a sync).
void timing_collect(ess_state* s) {
  for (auto& pe : s->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ev_pool[pe.second.first], s->ev_pool[pe.second.second]) ==
        cudaSuccess)
      s->phase_ms[pe.first] += ms;
  }
  s->ev_pending.clear();
  s->ev_used = 0;
}
size_t elem(const ess_state* s) { return mixed(s) ? sizeof(float) : sizeof(double); }

void drop_graphs(ess_state* s) {
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

void free_work(ess_state* s) {
  drop_graphs(s);
  if (s->P) cudaFree(s->P);
  if (s->P2) cudaFree(s->P2);
  s->P2 = nullptr;
  dev_free(s->ovf);
  if (s->Q) cudaFree(s->Q);
  if (s->NU) cudaFree(s->NU);
  if (s->NU_alt) cudaFree(s->NU_alt);
  s->P = s->Q = s->NU = s->NU_alt = nullptr;
  dev_free(s->Xw);
  dev_free(s->Xd);
  for (auto& p : s->NU_h) dev_free(p);
  for (auto& p : s->NU_h_alt) dev_free(p);
  dev_free(s->nu_unscale);
  dev_free(s->x_slices);
  dev_free(s->row_scale);
  dev_free(s->P64);
  s->cap = 0;
  s->n_loaded = 0;
}

ess_status ensure_capacity(ess_state* s, int n) {
  if (n <= s->cap) return ESS_OK;
  free_work(s);
  const size_t e = elem(s);
  ESS_CUDA(cudaMalloc(&s->P, (size_t)n * s->m * e));
  ESS_CUDA(cudaMalloc(&s->P2, (size_t)n * s->m * e));
  ESS_CUDA(dev_alloc(&s->ovf, (size_t)n + 2));
  ESS_CUDA(cudaMalloc(&s->Q, (size_t)n * s->m * e));
  ESS_CUDA(cudaMalloc(&s->NU, (size_t)n * s->d * e));
  ESS_CUDA(cudaMalloc(&s->NU_alt, (size_t)n * s->d * e));
  if (mixed(s)) {
    ESS_CUDA(dev_alloc(&s->Xw, (size_t)n * s->d));
    for (int k = 0; k < 4; ++k) {
      __half*& p = k < 2 ? s->NU_h[k] : s->NU_h_alt[k - 2];
      ESS_CUDA(dev_alloc(&p, (size_t)n * s->ld16));
      // the padding columns d .. ld16 - 1 stay zero
      ESS_CUDA(cudaMemset(p, 0, (size_t)n * s->ld16 * sizeof(__half)));
    }
    ESS_CUDA(dev_alloc(&s->nu_unscale, (size_t)n));
    if (s->cfg.refresh_mode == ESS_REFRESH_SPLIT) {
      const int K = ess::tc_refresh_num_slices(s->tc_plan);
      ESS_CUDA(dev_alloc(&s->x_slices, (size_t)K * n * s->ld16));
      ESS_CUDA(cudaMemset(s->x_slices, 0, (size_t)K * n * s->ld16 * sizeof(__nv_bfloat16)));
      ESS_CUDA(dev_alloc(&s->row_scale, (size_t)n));
      ESS_CUDA(dev_alloc(&s->P64, (size_t)n * s->m));
    }
  } else {
    ESS_CUDA(dev_alloc(&s->Xd, (size_t)n * s->d));
    if (split64(s)) {
      // slices of x (refresh) or nu (q), one at a time
      const int K = ess::tc_refresh_num_slices(s->tc_plan);
      ESS_CUDA(dev_alloc(&s->x_slices, (size_t)K * n * s->ld16));
      ESS_CUDA(cudaMemset(s->x_slices, 0, (size_t)K * n * s->ld16 * sizeof(__nv_bfloat16)));
      ESS_CUDA(dev_alloc(&s->row_scale, (size_t)n));
    }
  }
  s->cap = n;
  return ESS_OK;
}

// p = A x for all chains (refresh), with optional drift statistics and the
// FP64 feasibility check of the rounded states.
ess_status refresh_p(ess_state* s, int n, const void* Xcur, bool with_drift, bool check,
                     cudaStream_t st) {
  DevStats* drift = with_drift ? s->dstats : nullptr;
  if (mixed(s) && s->cfg.refresh_mode == ESS_REFRESH_SPLIT) {
    // exact products on the tensor cores (fixed-point split), rounded once
    const float* Xf = static_cast<const float*>(Xcur);
    ESS_CUDA(ess::tc_refresh(s->tc_plan, Xf, s->d, n, s->x_slices, (size_t)n * s->ld16,
                             s->row_scale, static_cast<float*>(s->P), check ? s->P64 : nullptr,
                             s->m, with_drift ? &s->dstats->max_drift_bits : nullptr,
                             s->dstatus, st));
    if (check) {
      ESS_CUDA(ess::launch_check_feasible_bounded(
          s->P64, s->m, s->b64, n, s->m, s->row_scale, ess::tc_refresh_col_scale(s->tc_plan),
          ess::tc_refresh_bound_factor(s->tc_plan), Xf, s->d, s->A64, s->d, s->dstatus, st));
    }
  } else if (mixed(s)) {
    ESS_CUDA((ess::launch_gemm_nt_f64<float, float>(static_cast<const float*>(Xcur), s->d, s->A64,
                                                     s->d, static_cast<float*>(s->P), s->m, n,
                                                     s->m, s->d, s->anorm, drift, st)));
    if (check) {
      // feasibility of the float-rounded states, decided in FP64
      double* P64 = nullptr;
      ESS_CUDA(dev_alloc(&P64, (size_t)n * s->m));
      cudaError_t e = ess::launch_gemm_nt_f64<float, double>(static_cast<const float*>(Xcur), s->d,
                                                             s->A64, s->d, P64, s->m, n, s->m,
                                                             s->d, s->anorm, nullptr, st);
      if (e == cudaSuccess) e = ess::launch_check_feasible(P64, s->m, s->b64, n, s->m, s->dstatus, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      cudaFree(P64);
      if (e != cudaSuccess) return cuda_fail(e, "feasibility check");
    }
  } else if (split64(s)) {
    // FP64 products from exact 56-bit splits on the tensor cores
    const double* Xd = static_cast<const double*>(Xcur);
    ESS_CUDA(ess::tc_exact_f64(s->tc_plan, Xd, s->d, n, s->x_slices, (size_t)n * s->ld16,
                               s->row_scale, static_cast<double*>(s->P), s->m,
                               with_drift ? &s->dstats->max_drift_bits : nullptr, s->dstatus, st));
    if (check) {
      // entries within the split's bound of b_i are decided by FP64 FMAs
      ESS_CUDA(ess::launch_check_feasible_bounded(
          static_cast<const double*>(s->P), s->m, s->b64, n, s->m, s->row_scale,
          ess::tc_refresh_col_scale(s->tc_plan), ess::tc_refresh_bound_factor(s->tc_plan), Xd,
          s->d, s->A64, s->d, s->dstatus, st));
    }
  } else {
    ESS_CUDA((ess::launch_gemm_nt_f64<double, double>(static_cast<const double*>(Xcur), s->d,
                                                       s->A64, s->d, static_cast<double*>(s->P),
                                                       s->m, n, s->m, s->d, s->anorm, drift, st)));
    if (check)
      ESS_CUDA(ess::launch_check_feasible(static_cast<const double*>(s->P), s->m, s->b64, n, s->m,
                                          s->dstatus, st));
  }
  return ESS_OK;
}

// q = A nu for all chains.  drawn: nu came from the draw kernel (fixed fp16
// split scale); otherwise the caller's nu was split with per-chain scales.
ess_status compute_q(ess_state* s, int n, cudaStream_t st, bool drawn = true) {
  if (mixed(s)) {
    cudaError_t e = ess::tc_gemm_q(s->tc_plan, s->NU_h, drawn ? nullptr : s->nu_unscale, s->ld16,
                                   n, static_cast<float*>(s->Q), s->m, s->dstatus, st);
    if (e != cudaSuccess) return cuda_fail(e, "FP16x3 tensor-core GEMM");
  } else if (split64(s)) {
    ESS_CUDA(ess::tc_exact_f64(s->tc_plan, static_cast<const double*>(s->NU), s->d, n,
                               s->x_slices, (size_t)n * s->ld16, s->row_scale,
                               static_cast<double*>(s->Q), s->m, nullptr, s->dstatus, st));
  } else {
    ESS_CUDA((ess::launch_gemm_nt_f64<double, double>(static_cast<const double*>(s->NU), s->d,
                                                       s->A64, s->d, static_cast<double*>(s->Q),
                                                       s->m, n, s->m, s->d, nullptr, nullptr, st)));
  }
  return ESS_OK;
}

const void* chain_states(const ess_state* s) {
  return mixed(s) ? static_cast<const void*>(s->Xw) : static_cast<const void*>(s->Xd);
}

template <typename T>
ess::ChainParams<T> base_params(ess_state* s, int n) {
  ess::ChainParams<T> p{};
  p.d = s->d;
  p.m = s->m;
  p.n_chains = n;
  p.ldx = s->d;
  p.ldp = s->m;
  p.P_in = static_cast<const T*>(s->P);
  p.P_out = static_cast<T*>(s->P);
  p.Q = static_cast<const T*>(s->Q);
  if constexpr (sizeof(T) == 4) p.b = reinterpret_cast<const T*>(s->b32);
  else p.b = reinterpret_cast<const T*>(s->b64);
  p.b64 = s->b64;
  p.A64 = s->A64;
  p.anorm = s->anorm;
  p.slack = static_cast<const T*>(s->slack);
  p.NU = static_cast<const T*>(s->NU);
  p.trim_eps = s->cfg.trim_eps;
  p.tangent_thresh = s->cfg.tangent_thresh;
  p.margin = s->cfg.residual_margin;
  p.long_arcs = s->long_arcs;
  p.stats = s->dstats;
  p.status = s->dstatus;
  return p;
}

// m > 8192: the warp kernel first (the wide-row kernel behind it for the
// chains it leaves) with ESS_CHAIN_WARP, and by default when some b_i <= 0
// (the long arcs' union leaves such chains few arcs: the probit-style
// orthant at m = 16384, d = 256 went from 0.71 to 0.1x ms per step); else the
// wide-row kernel for every chain.
bool wide_warp_first(const ess_state* s) {
  if (s->cfg.sort_threads > 0) return false;
  return s->chain_kernel == ESS_CHAIN_WARP ||
         (s->chain_kernel == ESS_CHAIN_AUTO && s->long_arcs != 0);
}

// Fewer chains than SMs (ESS_CHAIN_AUTO, m above 256 so that the CTA-per-
// chain kernel gives a chain 64 or more threads): one CTA per chain.  A warp
// per chain wins on throughput once the chains fill the GPU; with fewer
// chains than SMs the step is the latency of one chain, and one warp
// streaming all m rows took 81 us per step at m = 2000 (1 chain) against 33
// us for a CTA of 256 threads, 246 against 54 at m = 4000.
bool few_chains_cta(const ess_state* s, int n) {
  if (s->wide || s->chain_kernel != ESS_CHAIN_AUTO || s->chain_threads < 64 || s->sms <= 0)
    return false;
  return n < s->sms;
}

// Kernel launches of one chain step (per-phase accounting).
int chain_launches_per_step(const ess_state* s) {
  if (s->cfg.sort_threads > 0 || few_chains_cta(s, s->n_loaded)) return 1;
  if (s->wide) return wide_warp_first(s) ? 2 : 1;
  const bool streamed = mixed(s) && s->chain_kernel == ESS_CHAIN_STREAM &&
                        ess::chain_stream_supported(s->m, s->d);
  const bool local = !streamed && mixed(s) && ess::chain_warp_local_fallback<float>(s->m, s->d);
  return local ? 1 : 2;
}

// One chain step of all chains: the warp-per-chain kernel, then the
// CTA-per-chain kernel for the chains it left (too many arcs after the prune),
// reading P and writing P2; the buffers are swapped afterwards.
template <typename T>
ess_status launch_step(ess_state* s, ess::ChainParams<T> p, cudaStream_t st) {
  p.P_in = static_cast<const T*>(s->P);
  p.P_out = static_cast<T*>(s->P2);
  if (s->wide) {
    // m beyond the CTA kernel: the wide-row kernel for every chain (measured
    // faster at m = 12000 and 16384, where most chains keep more arcs than a
    // warp sorts), or with ESS_CHAIN_WARP the warp kernel first and the
    // wide-row kernel for the chains it leaves
    p.wide_scratch = static_cast<T*>(s->wide_scratch);
    p.wide_cap = s->wide_cap;
    if (!wide_warp_first(s)) {
      ESS_CUDA(ess::launch_chain_step_wide<T>(p, s->wide_slots, st));
    } else {
      ESS_CUDA(cudaMemsetAsync(s->ovf, 0, 2 * sizeof(int), st));
      p.overflow_count = s->ovf;
      p.overflow_list = s->ovf + 2;
      ESS_CUDA(ess::launch_chain_step_warp<T>(p, st));
      p.chain_list = s->ovf + 2;
      p.list_count = s->ovf;
      ESS_CUDA(ess::launch_chain_step_wide<T>(p, s->wide_slots, st));
    }
    std::swap(s->P, s->P2);
    return ESS_OK;
  }
  if (s->cfg.sort_threads > 0 || few_chains_cta(s, p.n_chains)) {
    ESS_CUDA(ess::launch_chain_step<T>(p, s->chain_threads, st));
  } else {
    bool streamed = false;
    if constexpr (sizeof(T) == 4)
      streamed = s->chain_kernel == ESS_CHAIN_STREAM && ess::chain_stream_supported(s->m, s->d) &&
                 ess::chain_stream_aligned(p);
    if (!streamed && ess::chain_warp_local_fallback<T>(s->m, s->d)) {
      // the warp kernel steps the chains it leaves itself: one launch, no
      // list to reset (measured 0.2755 -> 0.2654 ms per step at d = 1000,
      // m = 2000, 8192 chains)
      p.overflow_count = nullptr;
      p.overflow_list = nullptr;
      ESS_CUDA(ess::launch_chain_step_warp<T>(p, st));
    } else {
      ESS_CUDA(cudaMemsetAsync(s->ovf, 0, 2 * sizeof(int), st));
      p.overflow_count = s->ovf;
      p.overflow_list = s->ovf + 2;
      if constexpr (sizeof(T) == 4) {
        if (streamed) {
          p.work_counter = s->ovf + 1;
          ESS_CUDA(ess::launch_chain_step_stream(p, st));
        }
      }
      if (!streamed) ESS_CUDA(ess::launch_chain_step_warp<T>(p, st));
      p.chain_list = s->ovf + 2;
      p.list_count = s->ovf;
      ESS_CUDA(ess::launch_chain_step<T>(p, s->chain_threads, st));
    }
  }
  std::swap(s->P, s->P2);
  return ESS_OK;
}

ess_status read_status(ess_state* s, cudaStream_t st) {
  int h = 0;
  ESS_CUDA(cudaMemcpyAsync(&h, s->dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
  ESS_CUDA(cudaStreamSynchronize(st));
  if (h & ess::kStatusInfeasible)
    return fail(ESS_ERR_INFEASIBLE_X0, "a chain state violates A x <= b (checked in FP64)");
  if (h & ess::kStatusNumeric)
    return fail(ESS_ERR_NUMERIC, "NaN or Inf in theta or x; affected chains kept their state");
  if (h & ess::kStatusTimeout) return fail(ESS_ERR_TIMEOUT, "a bounded device wait gave up");
  return ESS_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

namespace {

// Times the candidate q GEMM widths and chain-step paths on the loaded chains
// (their first draw), writing x' to scratch so that no chain moves, and keeps
// the fastest.
ess_status autotune(ess_state* s, int t0, cudaStream_t st) {
  const int n = s->n_loaded, d = s->d;
  cudaEvent_t e0, e1;
  ESS_CUDA(cudaEventCreate(&e0));
  ESS_CUDA(cudaEventCreate(&e1));
  auto timed = [&](auto&& launch, float* ms) -> ess_status {
    ess_status rc = launch();  // warm-up
    if (rc != ESS_OK) return rc;
    ESS_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < 3 && rc == ESS_OK; ++r) rc = launch();
    ESS_CUDA(cudaEventRecord(e1, st));
    ESS_CUDA(cudaEventSynchronize(e1));
    if (rc != ESS_OK) return rc;
    ESS_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return ESS_OK;
  };
  const bool timing = s->timing;
  s->timing = false;
  ess_status rc = ESS_OK;
  // the trial steps must not count in the statistics
  DevStats saved{};
  ESS_CUDA(cudaMemcpyAsync(&saved, s->dstats, sizeof(saved), cudaMemcpyDeviceToHost, st));
  ESS_CUDA(cudaStreamSynchronize(st));
  // the first draw of the loaded chains (nu and, in the mixed form, its splits)
  if (mixed(s))
    ESS_CUDA(ess::launch_draw_nu_f32(static_cast<float*>(s->NU), d, s->NU_h, s->ld16, n, d, 0,
                                     (uint32_t)t0, 0u, 0u, st));
  else
    ESS_CUDA(ess::launch_draw_nu_f64(static_cast<double*>(s->NU), n, d, d, 0, (uint32_t)t0, 0u,
                                     0u, s->bm_tab, st));
  if (mixed(s)) {
    int best = 0;
    float best_ms = 0.f;
    for (int w : ess::kTcWidths) {
      ESS_CUDA(ess::tc_gemm_set_width(s->tc_plan, w));
      float ms = 0.f;
      rc = timed([&]() { return compute_q(s, n, st); }, &ms);
      if (rc != ESS_OK) break;
      if (best == 0 || ms < best_ms) {
        best = w;
        best_ms = ms;
      }
    }
    if (rc == ESS_OK) ESS_CUDA(ess::tc_gemm_set_width(s->tc_plan, best));
  }
  if (rc == ESS_OK) rc = compute_q(s, n, st);
  // chain step: x' to scratch, p' to the second buffer (P is left intact)
  void* scratch = nullptr;
  if (rc == ESS_OK) ESS_CUDA(cudaMalloc(&scratch, (size_t)n * d * elem(s)));
  const int saved_sort = s->cfg.sort_threads, saved_threads = s->chain_threads;
  const int saved_kernel = s->chain_kernel;
  // (sort_threads, CTA width of the fallback or of every chain, float kernel)
  int cands[4][3] = {{0, s->min_chain_threads, ESS_CHAIN_STREAM},
                     {0, s->min_chain_threads, ESS_CHAIN_WARP},
                     {s->min_chain_threads, s->min_chain_threads, ESS_CHAIN_AUTO},
                     {2 * s->min_chain_threads, 2 * s->min_chain_threads, ESS_CHAIN_AUTO}};
  int best = -1;
  float best_ms = 0.f;
  for (int c = 0; c < 4 && rc == ESS_OK; ++c) {
    if (cands[c][1] > ess::kChainMaxThreads) continue;
    // wide rows: the wide-row kernel for every chain, or the warp kernel
    // with the wide-row kernel behind it
    if (s->wide && c != 1 && c != 2) continue;
    // the streamed kernel exists for float chains with supported shapes
    if (c == 0 && !(mixed(s) && ess::chain_stream_supported(s->m, s->d))) continue;
    s->chain_kernel = cands[c][2];
    const size_t smem = mixed(s) ? ess::chain_smem_bytes<float>(cands[c][1], d)
                                 : ess::chain_smem_bytes<double>(cands[c][1], d);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    if (!s->wide && smem + 1024 > (size_t)optin) continue;
    s->cfg.sort_threads = cands[c][0];
    s->chain_threads = cands[c][1];
    float ms = 0.f;
    void* P_keep = s->P;
    void* P2_keep = s->P2;
    auto launch = [&]() -> ess_status {
      s->P = P_keep;
      s->P2 = P2_keep;
      ess_status r;
      if (mixed(s)) {
        ess::ChainParams<float> p = base_params<float>(s, n);
        p.X = s->Xw;
        p.X_out = static_cast<float*>(scratch);
        p.t = (uint32_t)t0;
        r = launch_step<float>(s, p, st);
      } else {
        ess::ChainParams<double> p = base_params<double>(s, n);
        p.X = s->Xd;
        p.X_out = static_cast<double*>(scratch);
        p.t = (uint32_t)t0;
        r = launch_step<double>(s, p, st);
      }
      s->P = P_keep;
      s->P2 = P2_keep;
      return r;
    };
    rc = timed(launch, &ms);
    if (rc == ESS_OK && (best < 0 || ms < best_ms)) {
      best = c;
      best_ms = ms;
    }
  }
  if (scratch) {
    cudaStreamSynchronize(st);
    cudaFree(scratch);
  }
  ESS_CUDA(cudaMemcpyAsync(s->dstats, &saved, sizeof(saved), cudaMemcpyHostToDevice, st));
  ESS_CUDA(cudaStreamSynchronize(st));
  if (best >= 0) {
    s->cfg.sort_threads = cands[best][0];
    s->chain_threads = cands[best][1];
    s->chain_kernel = cands[best][2];
  } else {
    s->cfg.sort_threads = saved_sort;
    s->chain_threads = saved_threads;
    s->chain_kernel = saved_kernel;
  }
  s->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graphs(s);  // captured with the previous choices
  if (rc == ESS_OK) s->tuned_n = n;
  return rc;
}

}  // namespace

namespace {

// nu of step t (+ *t_dev when t_dev is set) for every loaded chain into nu
// (and its fp16 split nu_h, mixed form).
template <typename T>
ess_status draw_step_nu(ess_state* s, uint64_t seed, uint32_t t, const unsigned* t_dev, void* nu,
                        __half* const nu_h[2], cudaStream_t st) {
  const int n = s->n_loaded, d = s->d;
  if constexpr (sizeof(T) == 4)
    ESS_CUDA(ess::launch_draw_nu_f32(static_cast<float*>(nu), d, nu_h, s->ld16, n, d, seed, t,
                                     0u, 0u, st, t_dev));
  else
    ESS_CUDA(ess::launch_draw_nu_f64(static_cast<double*>(nu), n, d, d, seed, t, 0u, 0u,
                                     s->bm_tab, st, t_dev));
  return ESS_OK;
}

// One step of every loaded chain at step index t (+ *t_dev when t_dev is
// set): draw nu (unless it is already in s->NU), q = A nu, chain step (p
// buffers swapped).
template <typename T>
ess_status step_one(ess_state* s, uint64_t seed, uint32_t t, const unsigned* t_dev, T* samples,
                    long long sample_stride, cudaStream_t st, bool draw = true) {
  const int n = s->n_loaded;
  if (draw) {
    PhaseScope ps(s, st, ESS_PHASE_DRAW);
    ess_status rc = draw_step_nu<T>(s, seed, t, t_dev, s->NU, s->NU_h, st);
    if (rc != ESS_OK) return rc;
  }
  {
    PhaseScope ps(s, st, ESS_PHASE_GEMM);
    ess_status rc = compute_q(s, n, st);
    if (rc != ESS_OK) return rc;
  }
  ess::ChainParams<T> p = base_params<T>(s, n);
  p.X = static_cast<const T*>(chain_states(s));
  p.X_out = static_cast<T*>(const_cast<void*>(chain_states(s)));
  p.seed = seed;
  p.t = t;
  p.t_dev = t_dev;
  p.samples = samples;
  p.sample_stride = sample_stride;
  PhaseScope ps(s, st, ESS_PHASE_CHAIN, chain_launches_per_step(s));
  return launch_step<T>(s, p, st);
}

// The internal streams and events of the draws made one step ahead: the steps
// at the highest priority, the draws at the lowest, so that a draw fills the
// SMs' room beside the q GEMM instead of delaying it.
ess_status ensure_streams(ess_state* s) {
  if (s->cap_stream) return ESS_OK;
  int least = 0, greatest = 0;
  ESS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  ESS_CUDA(cudaStreamCreateWithPriority(&s->cap_stream, cudaStreamNonBlocking, greatest));
  ESS_CUDA(cudaStreamCreateWithPriority(&s->work_stream, cudaStreamNonBlocking, greatest));
  ESS_CUDA(cudaStreamCreateWithPriority(&s->side_stream, cudaStreamNonBlocking, least));
  for (cudaEvent_t* e : {&s->ev_drawn, &s->ev_done, &s->ev_fork, &s->ev_join})
    ESS_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return ESS_OK;
}

// Replays (capturing on first use) one refresh period -- refresh, then
// refresh_k steps -- starting at the step index held in *t_dev.
template <typename T>
ess_status graph_period(ess_state* s, uint64_t seed, cudaStream_t st) {
  const int k = s->cfg.refresh_k;
  ess_state::GraphEntry* hit = nullptr;
  for (auto& g : s->graphs)
    if (g.n == s->n_loaded && g.seed == seed && g.p_first == s->P) hit = &g;
  if (!hit) {
    ess_status rs = ensure_streams(s);
    if (rs != ESS_OK) return rs;
    void* p_first = s->P;
    const bool timing = s->timing;
    s->timing = false;
    cudaStream_t cs = s->cap_stream, ss = s->side_stream;
    ESS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    // Step j's nu is drawn on the side stream into the buffer pair that step
    // j - 1 does not use: draw 0 beside the refresh, draw j + 1 beside step j
    // once step j - 1 (the last reader of that pair) is done.  Every side
    // operation is joined back before the step that reads it, and refresh_k
    // is even, so the period leaves the nu buffers where it found them.
    ess_status rc = ESS_OK;
    auto cap_ok = [&](cudaError_t e, const char* what) {
      if (rc == ESS_OK && e != cudaSuccess) rc = cuda_fail(e, what);
      return rc == ESS_OK;
    };
    if (cap_ok(cudaEventRecord(s->ev_done, cs), "graph fork") &&
        cap_ok(cudaStreamWaitEvent(ss, s->ev_done, 0), "graph fork")) {
      rc = draw_step_nu<T>(s, seed, 0u, s->t_dev, s->NU, s->NU_h, ss);
      if (rc == ESS_OK) cap_ok(cudaEventRecord(s->ev_drawn, ss), "graph draw");
    }
    if (rc == ESS_OK) rc = refresh_p(s, s->n_loaded, chain_states(s), true, false, cs);
    for (int j = 0; j < k && rc == ESS_OK; ++j) {
      if (!cap_ok(cudaStreamWaitEvent(cs, s->ev_drawn, 0), "graph join")) break;
      if (j + 1 < k) {
        if (j > 0 && !cap_ok(cudaStreamWaitEvent(ss, s->ev_done, 0), "graph fork")) break;
        rc = draw_step_nu<T>(s, seed, (uint32_t)(j + 1), s->t_dev, s->NU_alt, s->NU_h_alt, ss);
        if (rc != ESS_OK || !cap_ok(cudaEventRecord(s->ev_drawn, ss), "graph draw")) break;
      }
      rc = step_one<T>(s, seed, (uint32_t)j, s->t_dev, nullptr, 0, cs, false);
      if (rc != ESS_OK || !cap_ok(cudaEventRecord(s->ev_done, cs), "graph step")) break;
      std::swap(s->NU, s->NU_alt);
      std::swap(s->NU_h[0], s->NU_h_alt[0]);
      std::swap(s->NU_h[1], s->NU_h_alt[1]);
    }
    if (rc == ESS_OK) {
      cudaError_t e = ess::launch_advance_t(s->t_dev, (unsigned)k, cs);
      if (e != cudaSuccess) rc = cuda_fail(e, "advance step index");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    s->timing = timing;
    if (rc != ESS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return cuda_fail(ec, "graph capture");
    cudaGraphExec_t exec = nullptr;
    ec = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return cuda_fail(ec, "graph instantiate");
    // refresh_k is even, so the period leaves the p buffers where it found them
    if (s->P != p_first) std::swap(s->P, s->P2);
    s->graphs.push_back({s->n_loaded, seed, p_first, exec});
    hit = &s->graphs.back();
  }
  ESS_CUDA(cudaGraphLaunch(hit->exec, st));
  ++s->graph_launches;
  s->phase_launches[ESS_PHASE_REFRESH] += 1;
  s->phase_launches[ESS_PHASE_DRAW] += k;
  s->phase_launches[ESS_PHASE_GEMM] += k;
  s->phase_launches[ESS_PHASE_CHAIN] += (long long)k * chain_launches_per_step(s);
  return ESS_OK;
}

}  // namespace

extern "C" {

ess_status ess_default_config(int precision, ess_config* cfg) {
  if (!cfg) return fail(ESS_ERR_ARG, "cfg is NULL");
  if (precision != ESS_PREC_FP64 && precision != ESS_PREC_MIXED)
    return fail(ESS_ERR_ARG, "unknown precision");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->precision = precision;
  cfg->refresh_k = 32;
  cfg->refresh_mode = precision == ESS_PREC_MIXED ? ESS_REFRESH_SPLIT : ESS_REFRESH_FP64;
  cfg->tangent_thresh = 1e-4;
  cfg->trim_eps = 0.0;
  cfg->residual_margin = precision == ESS_PREC_MIXED ? 2e-4 : 1e-8;
  cfg->sort_threads = 0;
  return ESS_OK;
}

ess_status ess_create(const double* A, const double* b, int d, int m, const ess_config* cfg,
                      ess_state** out) {
  g_err.clear();
  if (!out) return fail(ESS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!A || !b) return fail(ESS_ERR_ARG, "A or b is NULL");
  if (d < 1 || m < 1) return fail(ESS_ERR_ARG, "need d >= 1 and m >= 1");
  if (!all_finite(A, (size_t)m * d) || !all_finite(b, (size_t)m))
    return fail(ESS_ERR_ARG, "A or b has NaN/Inf entries");
  ess_config c;
  if (cfg) c = *cfg;
  else ess_default_config(ESS_PREC_FP64, &c);
  if (c.precision != ESS_PREC_FP64 && c.precision != ESS_PREC_MIXED)
    return fail(ESS_ERR_ARG, "unknown precision");
  if (c.refresh_k < 1) return fail(ESS_ERR_ARG, "refresh_k must be >= 1");
  if (c.refresh_mode != ESS_REFRESH_FP64 && c.refresh_mode != ESS_REFRESH_SPLIT)
    return fail(ESS_ERR_ARG, "unknown refresh_mode");
  if (c.precision == ESS_PREC_FP64) c.refresh_mode = ESS_REFRESH_FP64;  // FP64 form: FP64 products
  if (!(c.tangent_thresh >= 0.0 && c.tangent_thresh < 1.0) || !(c.trim_eps >= 0.0) ||
      !(c.residual_margin >= 0.0))
    return fail(ESS_ERR_ARG, "tangent_thresh in [0, 1), trim_eps >= 0, residual_margin >= 0");
  if (c.fp64_products != ESS_PRODUCTS_DFMA && c.fp64_products != ESS_PRODUCTS_SPLIT)
    return fail(ESS_ERR_ARG, "unknown fp64_products");
  if (c.wait_limit_us < 0) return fail(ESS_ERR_ARG, "wait_limit_us must be >= 0");
  if (c.precision == ESS_PREC_MIXED && !ess::rows_fit_float_scales(A, b, m, d, true, 30))
    return fail(ESS_ERR_ARG,
                "a row of A or an entry of b is outside the mixed form's float scaling range "
                "(nonzero row maxima in [2^-30, 2^30], |b| <= 2^30); the FP64 form takes any "
                "finite values");
  if (c.precision == ESS_PREC_FP64 && c.fp64_products == ESS_PRODUCTS_SPLIT &&
      !ess::rows_fit_float_scales(A, b, m, d, false, 100))
    return fail(ESS_ERR_ARG,
                "a row of A is outside the float scaling range of split products (nonzero row "
                "maxima in [2^-100, 2^100]); DFMA products take any finite values");
  if (c.q_tile != 0 &&
      std::find(ess::kTcWidths, ess::kTcWidths + 16, c.q_tile) == ess::kTcWidths + 16)
    return fail(ESS_ERR_ARG,
                "q_tile: 0, 64/128/160/192/224/256, or 2000/3000 + 128/160/192/224/256");

  if (m > ess::kMaxRows)
    return fail(ESS_ERR_UNSUPPORTED, "m exceeds the chain step's row limit (2^22)");
  // m beyond the CTA kernel's shared-memory sort (8192 arcs): wide rows
  const int min_threads = ess::chain_threads_for(m);
  const bool wide = min_threads == 0;
  // a CTA per chain: at least the minimum width, wider if sort_threads asks
  int threads = min_threads;
  while (!wide && threads < c.sort_threads && threads < ess::kChainMaxThreads) threads <<= 1;
  const size_t smem =
      wide ? (c.precision == ESS_PREC_MIXED ? ess::chain_wide_smem_bytes<float>(d)
                                            : ess::chain_wide_smem_bytes<double>(d))
           : (c.precision == ESS_PREC_MIXED ? ess::chain_smem_bytes<float>(threads, d)
                                            : ess::chain_smem_bytes<double>(threads, d));
  int dev = 0;
  ESS_CUDA(cudaGetDevice(&dev));
  int smem_optin = 0;
  ESS_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + 1024 > (size_t)smem_optin)
    return fail(ESS_ERR_UNSUPPORTED, "d too large for the chain-step kernel's shared memory");

  ess_state* s = new ess_state();
  s->d = d;
  s->m = m;
  s->cfg = c;
  s->device = dev;
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
  s->ld16 = (d + 7) & ~7;
  s->chain_threads = threads;
  s->min_chain_threads = min_threads;
  s->wide = wide;

  auto cleanup = [&](ess_status st) {
    ess_destroy(s);
    return st;
  };
  std::vector<double> norms(m);
  for (int i = 0; i < m; ++i) {
    double acc = 0.0;
    for (int j = 0; j < d; ++j) acc += A[(size_t)i * d + j] * A[(size_t)i * d + j];
    norms[i] = std::sqrt(acc);
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dev_alloc(&s->A64, (size_t)m * d);
  if (e == cudaSuccess) e = dev_alloc(&s->b64, (size_t)m);
  if (e == cudaSuccess) e = dev_alloc(&s->anorm, (size_t)m);
  if (e == cudaSuccess) e = cudaMemcpy(s->A64, A, sizeof(double) * m * d, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->b64, b, sizeof(double) * m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->anorm, norms.data(), sizeof(double) * m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    // residual-recheck thresholds, rounded towards -inf in the step's precision
    const size_t esz = c.precision == ESS_PREC_MIXED ? sizeof(float) : sizeof(double);
    std::vector<unsigned char> buf(esz * m);
    for (int i = 0; i < m; ++i) {
      const double v = b[i] - c.residual_margin * norms[i];
      if (c.precision == ESS_PREC_MIXED) {
        float f = (float)v;
        if ((double)f > v) f = std::nextafter(f, -INFINITY);
        std::memcpy(&buf[esz * i], &f, esz);
      } else {
        std::memcpy(&buf[esz * i], &v, esz);
      }
    }
    e = cudaMalloc(&s->slack, esz * m);
    if (e == cudaSuccess) e = cudaMemcpy(s->slack, buf.data(), esz * m, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = dev_alloc(&s->dstats, 1);
  if (e == cudaSuccess) e = dev_alloc(&s->dstatus, 1);
  if (e == cudaSuccess) e = dev_alloc(&s->t_dev, 1);
  if (e == cudaSuccess && wide) {
    // scratch slots of the wide-row kernel (one per CTA of its launch)
    s->wide_slots = ess::chain_wide_slots(dev);
    s->wide_cap = c.precision == ESS_PREC_MIXED ? ess::chain_wide_cap<float>(m)
                                                : ess::chain_wide_cap<double>(m);
    const size_t esz = c.precision == ESS_PREC_MIXED ? sizeof(float) : sizeof(double);
    e = cudaMalloc(&s->wide_scratch, (size_t)s->wide_slots * 4 * (size_t)s->wide_cap * esz);
  }
  if (e == cudaSuccess) {
    std::vector<double> tab(ess::kBmTableSize);
    ess::bm_table_fill(tab.data());
    e = dev_alloc(&s->bm_tab, tab.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(s->bm_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(s->dstats, 0, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(s->dstatus, 0, sizeof(int));
  for (int i = 0; i < m; ++i)
    if (b[i] <= 0.0) s->long_arcs = 1;
  if (e == cudaSuccess && c.precision == ESS_PREC_MIXED) {
    std::vector<float> bf(m);
    for (int i = 0; i < m; ++i) bf[i] = (float)b[i];
    e = dev_alloc(&s->b32, (size_t)m);
    if (e == cudaSuccess) e = cudaMemcpy(s->b32, bf.data(), sizeof(float) * m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = ess::tc_gemm_create(&s->tc_plan, A, m, d);
    if (e == cudaSuccess && c.q_tile) e = ess::tc_gemm_set_width(s->tc_plan, c.q_tile);
  }
  if (e == cudaSuccess && c.precision == ESS_PREC_FP64 && c.fp64_products == ESS_PRODUCTS_SPLIT)
    e = ess::tc_gemm_create(&s->tc_plan, A, m, d, kSplit64Bits, false);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "ess_create device setup"));
  *out = s;
  return ESS_OK;
}

void ess_destroy(ess_state* s) {
  if (!s) return;
  DeviceGuard g(s->device);
  free_work(s);
  dev_free(s->A64);
  dev_free(s->b64);
  dev_free(s->anorm);
  if (s->slack) cudaFree(s->slack);
  s->slack = nullptr;
  dev_free(s->b32);
  dev_free(s->bm_tab);
  dev_free(s->dstats);
  dev_free(s->dstatus);
  ess::tc_gemm_destroy(s->tc_plan);
  s->tc_plan = nullptr;
  dev_free(s->t_dev);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->side_stream) cudaStreamDestroy(s->side_stream);
  if (s->work_stream) cudaStreamDestroy(s->work_stream);
  for (cudaEvent_t e : {s->ev_drawn, s->ev_done, s->ev_fork, s->ev_join})
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  dev_free(s->host_x);
  for (int k = 0; k < 2; ++k) {
    if (s->host_slot[k]) cudaFree(s->host_slot[k]);
    if (s->slot_ready[k]) cudaEventDestroy(s->slot_ready[k]);
    if (s->slot_free[k]) cudaEventDestroy(s->slot_free[k]);
  }
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->wide_scratch) cudaFree(s->wide_scratch);
  s->wide_scratch = nullptr;
  dev_free(s->few_x);
  dev_free(s->few_nu);
  dev_free(s->few_p);
  dev_free(s->few_q);
  dev_free(s->few_short);
  dev_free(s->few_th);
  dev_free(s->few_bkt);
  dev_free(s->few_int);
  dev_free(s->few_bar);
  delete s;
}

ess_status ess_limits(const ess_state* s, int* max_m, int* max_d) {
  if (!s || !max_m || !max_d) return fail(ESS_ERR_ARG, "NULL argument");
  *max_m = ess::kMaxRows;
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
  const size_t esz = mixed(s) ? sizeof(float) : sizeof(double);
  // d is bounded by the shared memory of the kernel that takes this state's m
  const size_t base =
      s->wide ? (mixed(s) ? ess::chain_wide_smem_bytes<float>(0)
                          : ess::chain_wide_smem_bytes<double>(0))
              : (mixed(s) ? ess::chain_smem_bytes<float>(s->chain_threads, 0)
                          : ess::chain_smem_bytes<double>(s->chain_threads, 0));
  long long room = (long long)smem_optin - 1024 - (long long)base;
  *max_d = room > 0 ? (int)(room / (long long)esz) - 1 : 0;
  return ESS_OK;
}

ess_status ess_chains_init(ess_state* s, const double* X, int n_chains, int t0,
                           void* cuda_stream) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (n_chains < 1 || t0 < 0) return fail(ESS_ERR_ARG, "need n_chains >= 1 and t0 >= 0");
  if (!X) return fail(ESS_ERR_ARG, "X is NULL");
  DeviceGuard g(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  s->n_loaded = 0;
  ess_status rc = ensure_capacity(s, n_chains);
  if (rc != ESS_OK) return rc;
  ESS_CUDA(cudaMemsetAsync(s->dstatus, 0, sizeof(int), st));
  const int n = n_chains, d = s->d;
  if (mixed(s)) ESS_CUDA((ess::launch_convert<double, float>(X, d, s->Xw, d, n, d, st)));
  else ESS_CUDA((ess::launch_convert<double, double>(X, d, s->Xd, d, n, d, st)));
  rc = refresh_p(s, n, chain_states(s), false, true, st);
  if (rc != ESS_OK) return rc;
  rc = read_status(s, st);
  if (rc != ESS_OK) return rc;
  s->n_loaded = n;
  s->t_next = t0;
  s->p_fresh_t = t0;
  if (s->cfg.autotune && s->tuned_n != n) {
    rc = autotune(s, t0, st);
    if (rc != ESS_OK) return rc;
  }
  return ESS_OK;
}

ess_status ess_get_tuning(const ess_state* s, int* q_width, int* sort_threads) {
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (q_width) *q_width = mixed(s) ? ess::tc_gemm_width(s->tc_plan, std::max(1, s->n_loaded)) : 0;
  if (sort_threads) *sort_threads = s->cfg.sort_threads;
  return ESS_OK;
}

namespace {

// The steps of ess_chains_step on stream st.  With `ahead`, each plain step
// t that another plain step follows draws nu of step t + 1 on the side
// stream into the second nu buffers, once step t - 1 (their last reader) is
// done, so that the draw runs beside step t; graph-replayed periods do the
// same inside the graph.
ess_status chains_step_on(ess_state* s, int n_iter, uint64_t seed, void* samples,
                          int record_every, cudaStream_t st, bool ahead) {
  const int n = s->n_loaded, d = s->d;
  const int n_rec = record_every > 0 ? n_iter / record_every : 0;
  const int k = s->cfg.refresh_k;
  // whole refresh periods replay from a CUDA graph (not with sample recording
  // or per-phase timing, whose pointers and events change from step to step)
  const bool graphs_ok = s->use_graphs && !s->timing && record_every == 0 && k % 2 == 0;
  auto graph_at = [&](int it_) {
    const int t_ = s->t_next + it_;
    return graphs_ok && t_ % k == 0 && t_ != s->p_fresh_t && n_iter - it_ >= k;
  };
  bool drawn = false;  // s->NU holds nu of step t, drawn on the side stream
  int it = 0;
  while (it < n_iter) {
    const int t = s->t_next + it;
    if (graph_at(it)) {
      ESS_CUDA(ess::launch_set_t(s->t_dev, (unsigned)t, st));
      while (n_iter - it >= k) {
        ess_status rc = mixed(s) ? graph_period<float>(s, seed, st) : graph_period<double>(s, seed, st);
        if (rc != ESS_OK) return rc;
        it += k;
      }
      s->p_fresh_t = s->t_next + it - k;
      continue;
    }
    const bool next = ahead && it + 1 < n_iter && !graph_at(it + 1);
    if (next) {
      ESS_CUDA(cudaEventRecord(s->ev_done, st));  // step t - 1 is done here
      ESS_CUDA(cudaStreamWaitEvent(s->side_stream, s->ev_done, 0));
      ess_status rc = mixed(s)
          ? draw_step_nu<float>(s, seed, (uint32_t)(t + 1), nullptr, s->NU_alt, s->NU_h_alt,
                                s->side_stream)
          : draw_step_nu<double>(s, seed, (uint32_t)(t + 1), nullptr, s->NU_alt, s->NU_h_alt,
                                 s->side_stream);
      if (rc != ESS_OK) return rc;
      s->phase_launches[ESS_PHASE_DRAW] += 1;
      ESS_CUDA(cudaEventRecord(s->ev_drawn, s->side_stream));
    }
    if (t % k == 0 && t != s->p_fresh_t) {
      PhaseScope ps(s, st, ESS_PHASE_REFRESH);
      ess_status rc = refresh_p(s, n, chain_states(s), true, false, st);
      if (rc != ESS_OK) return rc;
      s->p_fresh_t = t;
    }
    const bool rec = record_every > 0 && (it + 1) % record_every == 0 &&
                     (it + 1) / record_every <= n_rec;
    const long long rec_off = rec ? (long long)((it + 1) / record_every - 1) * d : 0;
    const long long stride = (long long)n_rec * d;
    ess_status rc = mixed(s)
        ? step_one<float>(s, seed, (uint32_t)t, nullptr,
                          rec ? static_cast<float*>(samples) + rec_off : nullptr, stride, st,
                          !drawn)
        : step_one<double>(s, seed, (uint32_t)t, nullptr,
                           rec ? static_cast<double*>(samples) + rec_off : nullptr, stride, st,
                           !drawn);
    if (rc != ESS_OK) return rc;
    if (next) {
      // step t + 1 reads the buffers just drawn, after the draw
      std::swap(s->NU, s->NU_alt);
      std::swap(s->NU_h[0], s->NU_h_alt[0]);
      std::swap(s->NU_h[1], s->NU_h_alt[1]);
      ESS_CUDA(cudaStreamWaitEvent(st, s->ev_drawn, 0));
    }
    drawn = next;
    ++it;
  }
  s->t_next += n_iter;
  s->host_steps += (long long)n * n_iter;
  return ESS_OK;
}

}  // namespace

ess_status ess_chains_step(ess_state* s, int n_iter, uint64_t seed, void* samples,
                           int record_every, void* cuda_stream) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (n_iter < 0 || record_every < 0) return fail(ESS_ERR_ARG, "negative size");
  if (s->n_loaded < 1) return fail(ESS_ERR_ARG, "no chains loaded (call ess_chains_init)");
  if (record_every > 0 && !samples) return fail(ESS_ERR_ARG, "samples is NULL");
  if ((long long)s->t_next + n_iter > 0x7fffffffLL) return fail(ESS_ERR_ARG, "step index overflow");
  DeviceGuard g(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // Without per-phase timing the steps run on the internal high-priority
  // stream, forked from and joined back into the caller's stream (the join
  // also covers every draw on the side stream, each of which a later step
  // waited for).
  const bool ahead = !s->timing && n_iter > 1;
  if (!ahead) return chains_step_on(s, n_iter, seed, samples, record_every, st, false);
  ess_status rc = ensure_streams(s);
  if (rc != ESS_OK) return rc;
  ESS_CUDA(cudaEventRecord(s->ev_fork, st));
  ESS_CUDA(cudaStreamWaitEvent(s->work_stream, s->ev_fork, 0));
  rc = chains_step_on(s, n_iter, seed, samples, record_every, s->work_stream, true);
  // join even after an error: no internal work may outlive the call's stream order
  cudaError_t e = cudaEventRecord(s->ev_join, s->work_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->ev_join, 0);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_join, s->side_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->ev_join, 0);
  if (e != cudaSuccess && rc == ESS_OK) rc = cuda_fail(e, "join internal streams");
  return rc;
}

ess_status ess_set_chain_kernel(ess_state* s, int kind) {
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (kind != ESS_CHAIN_AUTO && kind != ESS_CHAIN_WARP && kind != ESS_CHAIN_STREAM)
    return fail(ESS_ERR_ARG, "kind: ESS_CHAIN_AUTO, ESS_CHAIN_WARP or ESS_CHAIN_STREAM");
  if (kind != s->chain_kernel) drop_graphs(s);  // captured periods hold the old kernel
  s->chain_kernel = kind;
  return ESS_OK;
}

ess_status ess_get_chain_kernel(const ess_state* s, int* kind) {
  if (!s || !kind) return fail(ESS_ERR_ARG, "NULL argument");
  if (s->cfg.sort_threads > 0 || (s->wide && !wide_warp_first(s)) ||
      few_chains_cta(s, s->n_loaded))
    *kind = ESS_CHAIN_CTA;
  else if (mixed(s) && s->chain_kernel == ESS_CHAIN_STREAM && ess::chain_stream_supported(s->m, s->d))
    *kind = ESS_CHAIN_STREAM;
  else *kind = ESS_CHAIN_WARP;
  return ESS_OK;
}

ess_status ess_set_graphs(ess_state* s, int enable) {
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  s->use_graphs = enable != 0;
  return ESS_OK;
}

ess_status ess_graph_launches(const ess_state* s, long long* launches) {
  if (!s || !launches) return fail(ESS_ERR_ARG, "NULL argument");
  *launches = s->graph_launches;
  return ESS_OK;
}

ess_status ess_chains_get(ess_state* s, double* X, void* cuda_stream) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (s->n_loaded < 1) return fail(ESS_ERR_ARG, "no chains loaded (call ess_chains_init)");
  DeviceGuard g(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int n = s->n_loaded, d = s->d;
  if (X) {
    if (mixed(s)) ESS_CUDA((ess::launch_convert<float, double>(s->Xw, d, X, d, n, d, st)));
    else ESS_CUDA((ess::launch_convert<double, double>(s->Xd, d, X, d, n, d, st)));
  }
  ess_status rc = read_status(s, st);
  timing_collect(s);
  return rc;
}

ess_status ess_set_timing(ess_state* s, int enable) {
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  s->timing = enable != 0;
  return ESS_OK;
}

ess_status ess_get_timing(ess_state* s, double* ms, long long* launches, int n_phases) {
  if (!s || n_phases < 0) return fail(ESS_ERR_ARG, "bad argument");
  DeviceGuard g(s->device);
  ESS_CUDA(cudaDeviceSynchronize());
  timing_collect(s);
  for (int i = 0; i < n_phases && i < ESS_N_PHASES; ++i) {
    if (ms) ms[i] = s->phase_ms[i];
    if (launches) launches[i] = s->phase_launches[i];
  }
  return ESS_OK;
}

ess_status ess_reset_timing(ess_state* s) {
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  DeviceGuard g(s->device);
  ESS_CUDA(cudaDeviceSynchronize());
  timing_collect(s);
  for (int i = 0; i < ESS_N_PHASES; ++i) {
    s->phase_ms[i] = 0.0;
    s->phase_launches[i] = 0;
  }
  return ESS_OK;
}

ess_status ess_run(ess_state* s, double* X, int n_chains, int t0, int n_iter, uint64_t seed,
                   void* samples, int record_every, void* cuda_stream) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (n_chains < 0 || n_iter < 0 || t0 < 0 || record_every < 0)
    return fail(ESS_ERR_ARG, "negative size");
  if (n_chains == 0) return ESS_OK;
  if (!X) return fail(ESS_ERR_ARG, "X is NULL");
  if (record_every > 0 && !samples) return fail(ESS_ERR_ARG, "samples is NULL");
  ess_status rc = ess_chains_init(s, X, n_chains, t0, cuda_stream);
  if (rc == ESS_OK) rc = ess_chains_step(s, n_iter, seed, samples, record_every, cuda_stream);
  if (rc == ESS_OK) rc = ess_chains_get(s, X, cuda_stream);
  return rc;
}

namespace {
ess_status run_few_impl(ess_state* s, double* X, int n_chains, int t0, int n_iter, uint64_t seed,
                        double* samples, int record_every, void* cuda_stream, bool hold);
}  // namespace

ess_status ess_run_few(ess_state* s, double* X, int n_chains, int t0, int n_iter, uint64_t seed,
                       double* samples, int record_every, void* cuda_stream) {
  return run_few_impl(s, X, n_chains, t0, n_iter, seed, samples, record_every, cuda_stream, false);
}

ess_status ess_selftest_wait(ess_state* s) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (s->cfg.precision != ESS_PREC_FP64)
    return fail(ESS_ERR_UNSUPPORTED, "the self-test runs the FP64 few-chain kernel");
  DeviceGuard g(s->device);
  double* X = nullptr;
  ESS_CUDA(dev_alloc(&X, (size_t)s->d));
  ESS_CUDA(cudaMemset(X, 0, sizeof(double) * s->d));
  const ess_status rc = run_few_impl(s, X, 1, 0, 1, 0, nullptr, 0, nullptr, true);
  cudaFree(X);
  return rc;
}

namespace {
ess_status run_few_impl(ess_state* s, double* X, int n_chains, int t0, int n_iter, uint64_t seed,
                        double* samples, int record_every, void* cuda_stream, bool hold) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (s->cfg.precision != ESS_PREC_FP64)
    return fail(ESS_ERR_UNSUPPORTED, "ess_run_few runs the FP64 form");
  if (n_chains < 1 || n_chains > ess::kMaxFew)
    return fail(ESS_ERR_ARG, "ess_run_few takes 1 to 16 chains");
  if (n_iter < 0 || t0 < 0 || record_every < 0) return fail(ESS_ERR_ARG, "negative size");
  if (!X) return fail(ESS_ERR_ARG, "X is NULL");
  if (record_every > 0 && !samples) return fail(ESS_ERR_ARG, "samples is NULL");
  if (s->m > ess::kFewMaxM) return fail(ESS_ERR_UNSUPPORTED, "ess_run_few takes m <= 6144");
  if ((long long)t0 + n_iter > 0x7fffffffLL) return fail(ESS_ERR_ARG, "step index overflow");
  if (n_iter == 0) return ESS_OK;
  DeviceGuard g(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int d = s->d, m = s->m, F = ess::kMaxFew;
  if (!s->few_x) {
    ESS_CUDA(dev_alloc(&s->few_x, (size_t)2 * F * d));
    ESS_CUDA(dev_alloc(&s->few_nu, (size_t)2 * F * d));
    ESS_CUDA(dev_alloc(&s->few_p, (size_t)2 * F * m));
    ESS_CUDA(dev_alloc(&s->few_q, (size_t)F * m));
    ESS_CUDA(dev_alloc(&s->few_short, (size_t)4 * F * m));
    ESS_CUDA(dev_alloc(&s->few_th, (size_t)3 * F));
    ESS_CUDA(dev_alloc(&s->few_bkt, (size_t)4 * F * ess::kFewBuckets));
    ESS_CUDA(dev_alloc(&s->few_int, (size_t)9 * F));
    ESS_CUDA(dev_alloc(&s->few_bar, (size_t)4));
  }
  // rej[(t0 - 1) & 1] = 1 and cur = 0: step t0 starts from buffer 0
  int init[9 * ess::kMaxFew] = {0};
  for (int c = 0; c < F; ++c) init[((t0 + 1) & 1) * F + c] = 1;
  ESS_CUDA(cudaMemcpyAsync(s->few_int, init, sizeof(init), cudaMemcpyHostToDevice, st));
  ESS_CUDA(cudaMemsetAsync(s->few_bar, 0, sizeof(unsigned) * 4, st));
  ESS_CUDA(cudaMemsetAsync(s->dstatus, 0, sizeof(int), st));
  ess::FewArgs a{};
  a.A = s->A64;
  a.b = s->b64;
  a.anorm = s->anorm;
  a.bm_tab = s->bm_tab;
  a.d = d;
  a.m = m;
  a.C = n_chains;
  a.chunk = ess::few_chains_chunk(n_chains, d);
  for (int k = 0; k < 2; ++k) {
    a.X[k] = s->few_x + (size_t)k * F * d;
    a.NU[k] = s->few_nu + (size_t)k * F * d;
    a.P[k] = s->few_p + (size_t)k * F * m;
    a.rej[k] = s->few_int + (size_t)k * F;
    a.cur[k] = s->few_int + (size_t)(2 + k) * F;
  }
  a.Q = s->few_q;
  for (int k = 0; k < 2; ++k) {
    a.bmin[k] = s->few_bkt + (size_t)(2 * k) * F * ess::kFewBuckets;
    a.bmax[k] = s->few_bkt + (size_t)(2 * k + 1) * F * ess::kFewBuckets;
    a.shorts[k] = s->few_short + (size_t)k * 2 * F * m;
    a.nshort[k] = s->few_int + (size_t)(4 + k) * F;
    a.bad[k] = s->few_int + (size_t)(6 + k) * F;
  }
  a.bad_prev = s->few_int + (size_t)8 * F;
  a.theta = s->few_th;
  a.cth = s->few_th + F;
  a.sth = s->few_th + 2 * F;
  a.bar = s->few_bar;
  a.abort_flag = reinterpret_cast<int*>(s->few_bar + 2);
  a.X_user = X;
  a.samples = record_every > 0 ? samples : nullptr;
  a.record_every = record_every > 0 ? record_every : 1;
  a.n_rec = record_every > 0 ? n_iter / record_every : 0;
  a.t0 = t0;
  a.n_iter = n_iter;
  a.refresh_k = s->cfg.refresh_k;
  a.seed = seed;
  a.trim_eps = s->cfg.trim_eps;
  a.margin = s->cfg.residual_margin;
  a.stats = s->dstats;
  a.status = s->dstatus;
  a.wait_ns = s->cfg.wait_limit_us > 0 ? 1000ull * (unsigned long long)s->cfg.wait_limit_us
                                       : 2000000000ull;
  a.hold = hold ? 1 : 0;
  const size_t smem = ess::few_chains_smem(n_chains, m, a.chunk);
  int optin = 0;
  ESS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device));
  if (smem + 2048 > (size_t)optin)
    return fail(ESS_ERR_UNSUPPORTED, "m too large for the few-chain kernel's shared memory");
  ESS_CUDA(ess::launch_few_chains(a, st));
  s->host_steps += (long long)n_chains * n_iter;
  return read_status(s, st);
}
}  // namespace

ess_status ess_cholesky(double* A, int n, int lda, int* info, void* cuda_stream) {
  g_err.clear();
  if (info) *info = 0;
  if (!A || n < 1 || lda < n) return fail(ESS_ERR_ARG, "need A, n >= 1 and lda >= n");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* dinfo = nullptr;
  ESS_CUDA(dev_alloc(&dinfo, (size_t)1));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(dinfo, 0, sizeof(int), st);
  if (e == cudaSuccess) e = ess::launch_cholesky(A, n, lda, dinfo, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dinfo);
  if (e != cudaSuccess) return cuda_fail(e, "Cholesky factorisation");
  if (info) *info = h;
  if (h != 0)
    return fail(ESS_ERR_ARG, "matrix is not positive definite (pivot of row " +
                                 std::to_string(h - 1) + ")");
  return ESS_OK;
}

ess_status ess_run_host(ess_state* s, double* X_host, int n_chains, int t0, int n_iter,
                        uint64_t seed, void* samples_host, int record_every, void* cuda_stream) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (n_chains < 0 || n_iter < 0 || record_every < 0) return fail(ESS_ERR_ARG, "negative size");
  if (n_chains == 0) return ESS_OK;
  if (!X_host) return fail(ESS_ERR_ARG, "X is NULL");
  if (record_every > 0 && !samples_host) return fail(ESS_ERR_ARG, "samples is NULL");
  DeviceGuard g(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int d = s->d;
  const size_t xbytes = sizeof(double) * (size_t)n_chains * d;
  const int n_rec = record_every > 0 ? n_iter / record_every : 0;
  const size_t row = elem(s) * (size_t)d;         // one chain's state
  const size_t slot_bytes = row * (size_t)n_chains;  // one record of every chain
  // device buffers and the copy stream, kept across calls (grow only)
  if (n_chains > s->host_cap) {
    dev_free(s->host_x);
    for (auto& p : s->host_slot)
      if (p) {
        cudaFree(p);
        p = nullptr;
      }
    s->host_cap = 0;
    ESS_CUDA(dev_alloc(&s->host_x, (size_t)n_chains * d));
    for (auto& p : s->host_slot) ESS_CUDA(cudaMalloc(&p, slot_bytes));
    s->host_cap = n_chains;
  }
  if (!s->copy_stream) ESS_CUDA(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    if (!s->slot_ready[k])
      ESS_CUDA(cudaEventCreateWithFlags(&s->slot_ready[k], cudaEventDisableTiming));
    if (!s->slot_free[k])
      ESS_CUDA(cudaEventCreateWithFlags(&s->slot_free[k], cudaEventDisableTiming));
  }
  ESS_CUDA(cudaMemcpyAsync(s->host_x, X_host, xbytes, cudaMemcpyHostToDevice, st));
  ess_status rc = ess_chains_init(s, s->host_x, n_chains, t0, cuda_stream);
  // record r: record_every steps, then a device copy of the states into slot
  // r % 2 and its copy to the host (chain-major rows of n_rec records) on the
  // copy stream while the next steps run; a slot is refilled only after its
  // previous copy to the host has finished
  for (int r = 0; r < n_rec && rc == ESS_OK; ++r) {
    rc = ess_chains_step(s, record_every, seed, nullptr, 0, cuda_stream);
    if (rc != ESS_OK) break;
    const int k = r & 1;
    if (r >= 2) ESS_CUDA(cudaStreamWaitEvent(st, s->slot_free[k], 0));
    ESS_CUDA(cudaMemcpyAsync(s->host_slot[k], chain_states(s), slot_bytes,
                             cudaMemcpyDeviceToDevice, st));
    ESS_CUDA(cudaEventRecord(s->slot_ready[k], st));
    ESS_CUDA(cudaStreamWaitEvent(s->copy_stream, s->slot_ready[k], 0));
    ESS_CUDA(cudaMemcpy2DAsync(static_cast<char*>(samples_host) + (size_t)r * row,
                               row * (size_t)n_rec, s->host_slot[k], row, row, (size_t)n_chains,
                               cudaMemcpyDeviceToHost, s->copy_stream));
    ESS_CUDA(cudaEventRecord(s->slot_free[k], s->copy_stream));
  }
  const int rest = n_iter - n_rec * record_every;
  if (rc == ESS_OK && rest > 0) rc = ess_chains_step(s, rest, seed, nullptr, 0, cuda_stream);
  if (rc == ESS_OK) rc = ess_chains_get(s, s->host_x, cuda_stream);
  if (rc == ESS_OK || rc == ESS_ERR_NUMERIC) {
    cudaError_t e = cudaMemcpyAsync(X_host, s->host_x, xbytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && rc == ESS_OK) rc = cuda_fail(e, "copy results to host");
  }
  // the sample copies have finished before the call returns
  const cudaError_t e = cudaStreamSynchronize(s->copy_stream);
  if (e != cudaSuccess && rc == ESS_OK) rc = cuda_fail(e, "copy samples to host");
  return rc;
}

ess_status ess_step_with_draws(ess_state* s, const double* X, const double* nu, const double* u,
                               int n_chains, double* X_next, double* theta, double* pieces,
                               int max_pieces, int* n_pieces, int* rejected, void* cuda_stream) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (n_chains < 0) return fail(ESS_ERR_ARG, "negative size");
  if (n_chains == 0) return ESS_OK;
  if (!X || !nu || !u || !X_next) return fail(ESS_ERR_ARG, "NULL input");
  if (pieces && max_pieces < 1) return fail(ESS_ERR_ARG, "max_pieces < 1");
  DeviceGuard g(s->device);
  s->n_loaded = 0;  // the work buffers are reused
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  ess_status rc = ensure_capacity(s, n_chains);
  if (rc != ESS_OK) return rc;
  ESS_CUDA(cudaMemsetAsync(s->dstatus, 0, sizeof(int), st));
  const int n = n_chains, d = s->d;
  if (mixed(s)) {
    ESS_CUDA((ess::launch_convert<double, float>(X, d, s->Xw, d, n, d, st)));
    ESS_CUDA((ess::launch_convert<double, float>(nu, d, static_cast<float*>(s->NU), d, n, d, st)));
    ESS_CUDA(ess::tc_split2_rows(static_cast<const float*>(s->NU), d, n, d, s->NU_h[0],
                                 s->NU_h[1], s->ld16, s->nu_unscale, st));
    rc = refresh_p(s, n, s->Xw, false, true, st);
    if (rc == ESS_OK) rc = read_status(s, st);
    if (rc != ESS_OK) return rc;
    rc = compute_q(s, n, st, false);
    if (rc != ESS_OK) return rc;
    ess::ChainParams<float> p = base_params<float>(s, n);
    p.X = s->Xw;
    p.X_out = s->Xw;
    p.U = u;
    p.theta_out = theta;
    p.pieces_out = pieces;
    p.max_pieces = max_pieces;
    p.npieces_out = n_pieces;
    p.rejected_out = rejected;
    rc = launch_step<float>(s, p, st);
    if (rc != ESS_OK) return rc;
    ESS_CUDA((ess::launch_convert<float, double>(s->Xw, d, X_next, d, n, d, st)));
    s->host_steps += n;
  } else {
    ESS_CUDA((ess::launch_convert<double, double>(nu, d, static_cast<double*>(s->NU), d, n, d, st)));
    rc = refresh_p(s, n, X, false, true, st);
    if (rc == ESS_OK) rc = read_status(s, st);
    if (rc != ESS_OK) return rc;
    rc = compute_q(s, n, st);
    if (rc != ESS_OK) return rc;
    ess::ChainParams<double> p = base_params<double>(s, n);
    p.X = X;
    p.X_out = X_next;
    p.U = u;
    p.theta_out = theta;
    p.pieces_out = pieces;
    p.max_pieces = max_pieces;
    p.npieces_out = n_pieces;
    p.rejected_out = rejected;
    rc = launch_step<double>(s, p, st);
    if (rc != ESS_OK) return rc;
    s->host_steps += n;
  }
  return read_status(s, st);
}

ess_status ess_products(ess_state* s, const double* X, const double* nu, int n_chains, double* P,
                        double* Q, void* cuda_stream) {
  g_err.clear();
  if (!s) return fail(ESS_ERR_ARG, "state is NULL");
  if (n_chains < 0) return fail(ESS_ERR_ARG, "negative size");
  if (n_chains == 0) return ESS_OK;
  if ((P && !X) || (Q && !nu)) return fail(ESS_ERR_ARG, "NULL input");
  DeviceGuard g(s->device);
  s->n_loaded = 0;  // the work buffers are reused
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  ess_status rc = ensure_capacity(s, n_chains);
  if (rc != ESS_OK) return rc;
  ESS_CUDA(cudaMemsetAsync(s->dstatus, 0, sizeof(int), st));
  const int n = n_chains, d = s->d, m = s->m;
  if (mixed(s)) {
    if (P) {
      ESS_CUDA((ess::launch_convert<double, float>(X, d, s->Xw, d, n, d, st)));
      rc = refresh_p(s, n, s->Xw, false, false, st);
      if (rc != ESS_OK) return rc;
      ESS_CUDA((ess::launch_convert<float, double>(static_cast<const float*>(s->P), m, P, m, n, m, st)));
    }
    if (Q) {
      ESS_CUDA((ess::launch_convert<double, float>(nu, d, static_cast<float*>(s->NU), d, n, d, st)));
      ESS_CUDA(ess::tc_split2_rows(static_cast<const float*>(s->NU), d, n, d, s->NU_h[0],
                                   s->NU_h[1], s->ld16, s->nu_unscale, st));
      rc = compute_q(s, n, st, false);
      if (rc != ESS_OK) return rc;
      ESS_CUDA((ess::launch_convert<float, double>(static_cast<const float*>(s->Q), m, Q, m, n, m, st)));
    }
  } else {
    if (P) {
      rc = refresh_p(s, n, X, false, false, st);
      if (rc != ESS_OK) return rc;
      ESS_CUDA((ess::launch_convert<double, double>(static_cast<const double*>(s->P), m, P, m, n, m, st)));
    }
    if (Q) {
      ESS_CUDA((ess::launch_convert<double, double>(nu, d, static_cast<double*>(s->NU), d, n, d, st)));
      rc = compute_q(s, n, st);
      if (rc != ESS_OK) return rc;
      ESS_CUDA((ess::launch_convert<double, double>(static_cast<const double*>(s->Q), m, Q, m, n, m, st)));
    }
  }
  return read_status(s, st);
}

ess_status ess_philox_blocks(uint64_t seed, uint32_t chain, uint32_t t, uint32_t problem,
                             uint32_t stream, int n_blocks, uint32_t* out, void* cuda_stream) {
  g_err.clear();
  if (n_blocks < 0 || (n_blocks > 0 && !out)) return fail(ESS_ERR_ARG, "bad output");
  if (problem > 0xFFFFFFu || stream > 0xFFu) return fail(ESS_ERR_ARG, "problem or stream too large");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  ESS_CUDA(ess::launch_philox_blocks(seed, chain, t, problem, stream, n_blocks, out, st));
  ESS_CUDA(cudaStreamSynchronize(st));
  return ESS_OK;
}

ess_status ess_draw_normals(const ess_state* s, int n_chains, int t, uint64_t seed, void* out,
                            void* cuda_stream) {
  g_err.clear();
  if (!s || !out) return fail(ESS_ERR_ARG, "NULL argument");
  if (n_chains < 0 || t < 0) return fail(ESS_ERR_ARG, "negative size");
  DeviceGuard g(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (mixed(s))
    ESS_CUDA(ess::launch_draw_nu_f32(static_cast<float*>(out), s->d, nullptr, 0, n_chains,
                                     s->d, seed, (uint32_t)t, 0u, 0u, st));
  else
    ESS_CUDA(ess::launch_draw_nu_f64(static_cast<double*>(out), n_chains, s->d, s->d, seed,
                                     (uint32_t)t, 0u, 0u, s->bm_tab, st));
  ESS_CUDA(cudaStreamSynchronize(st));
  return ESS_OK;
}

ess_status ess_get_stats(const ess_state* s, ess_stats* out) {
  if (!s || !out) return fail(ESS_ERR_ARG, "NULL argument");
  DeviceGuard g(s->device);
  DevStats h{};
  ESS_CUDA(cudaMemcpy(&h, s->dstats, sizeof(h), cudaMemcpyDeviceToHost));
  out->steps = s->host_steps;
  out->rejections = (long long)h.rejections;
  out->residual_rechecks = (long long)h.rechecks;
  out->tangent_fp64 = (long long)h.tangent_fp64;
  out->numeric_errors = (long long)h.numeric_errors;
  out->sort_keys = (long long)h.sort_keys;
  double drift = 0.0;
  std::memcpy(&drift, &h.max_drift_bits, sizeof(double));
  out->max_refresh_drift = drift;
  out->max_residual = h.max_residual_bits ? ess::dec_ordered(h.max_residual_bits) : -INFINITY;
  return ESS_OK;
}

ess_status ess_reset_stats(ess_state* s) {
  if (!s) return fail(ESS_ERR_ARG, "NULL argument");
  DeviceGuard g(s->device);
  ESS_CUDA(cudaMemset(s->dstats, 0, sizeof(DevStats)));
  s->host_steps = 0;
  return ESS_OK;
}

ess_status ess_whiten(const double* A, const double* b, const double* mu, const double* L, int d,
                      int m, double* A_out, double* b_out) {
  g_err.clear();
  if (!A || !b || !L || !A_out || !b_out) return fail(ESS_ERR_ARG, "NULL argument");
  if (d < 1 || m < 1) return fail(ESS_ERR_ARG, "need d >= 1 and m >= 1");
  // A_out = A L: row i of A_out is sum_j A[i, j] * (row j of L)
  for (int i = 0; i < m; ++i) {
    double* out = A_out + (size_t)i * d;
    for (int k = 0; k < d; ++k) out[k] = 0.0;
    const double* a = A + (size_t)i * d;
    double am = 0.0;
    for (int j = 0; j < d; ++j) {
      const double aij = a[j];
      if (mu) am += aij * mu[j];
      if (aij == 0.0) continue;
      const double* lrow = L + (size_t)j * d;
      for (int k = 0; k < d; ++k) out[k] += aij * lrow[k];
    }
    b_out[i] = b[i] - am;
  }
  return ESS_OK;
}

ess_status ess_unwhiten(const double* L, const double* mu, int d, int n, const double* U, double* X) {
  g_err.clear();
  if (!L || !U || !X) return fail(ESS_ERR_ARG, "NULL argument");
  if (d < 1 || n < 0) return fail(ESS_ERR_ARG, "bad size");
  for (int r = 0; r < n; ++r) {
    const double* u = U + (size_t)r * d;
    double* x = X + (size_t)r * d;
    for (int i = 0; i < d; ++i) {
      const double* lrow = L + (size_t)i * d;
      double acc = 0.0;
      for (int j = 0; j < d; ++j) acc += lrow[j] * u[j];
      x[i] = acc + (mu ? mu[i] : 0.0);
    }
  }
  return ESS_OK;
}

// ---- normal probability of the domain (HDR splitting estimator) -----------
namespace {

// Device scratch of one ess_hdr call (freed by the destructor).
struct HdrScratch {
  double* X64 = nullptr;   // n x d start draws
  void* Xtmp = nullptr;    // n x d states (T) for the gather
  double* g = nullptr;     // n level values
  int* list = nullptr;     // n sample indices
  double* gamma = nullptr; // 1
  int* count = nullptr;    // 1
  double* b0 = nullptr;    // m: saved b (the unshifted bounds)
  float* b32_0 = nullptr;  // m: saved float b (mixed form)
  void* slack0 = nullptr;  // m: saved recheck thresholds
  double* P64 = nullptr;   // n x m FP64 products when the refresh has none to share
  ~HdrScratch() {
    for (void* p : {(void*)X64, Xtmp, (void*)g, (void*)list, (void*)gamma, (void*)count,
                    (void*)b0, (void*)b32_0, slack0, (void*)P64})
      if (p) cudaFree(p);
  }
};

// A x of the loaded states in FP64 for the level values; they also refresh
// the chains' p.  Mixed form with the split refresh: its exact-split FP64
// output; mixed form with the FP64 refresh: a separate FP64 product; FP64
// forms: the refreshed p itself.
ess_status hdr_products(ess_state* s, int n, HdrScratch& w, cudaStream_t st, const double** P) {
  if (mixed(s) && s->cfg.refresh_mode == ESS_REFRESH_SPLIT) {
    // one exact-split product, rounded to float for p and to double here
    ESS_CUDA(ess::tc_refresh(s->tc_plan, s->Xw, s->d, n, s->x_slices, (size_t)n * s->ld16,
                             s->row_scale, static_cast<float*>(s->P), s->P64, s->m, nullptr,
                             s->dstatus, st));
    *P = s->P64;
    return ESS_OK;
  }
  ess_status rc = refresh_p(s, n, chain_states(s), false, false, st);
  if (rc != ESS_OK) return rc;
  if (!mixed(s)) {
    *P = static_cast<const double*>(s->P);
  } else {
    ESS_CUDA((ess::launch_gemm_nt_f64<float, double>(s->Xw, s->d, s->A64, s->d, w.P64, s->m, n,
                                                      s->m, s->d, nullptr, nullptr, st)));
    *P = w.P64;
  }
  return ESS_OK;
}

}  // namespace

ess_status ess_hdr(ess_state* s, int n_samples, double rho, int n_between, uint64_t seed,
                   int max_levels, double* shifts, int* counts, int* counts_ss, int* n_levels,
                   double* log_z, double* log_z_ss, void* cuda_stream) {
  g_err.clear();
  if (!s || !shifts || !n_levels || !log_z) return fail(ESS_ERR_ARG, "NULL argument");
  const int n = n_samples, d = s->d, m = s->m;
  if (n < 2 || !(rho > 0.0 && rho < 1.0) || n_between < 1 || max_levels < 1)
    return fail(ESS_ERR_ARG, "need n_samples >= 2, 0 < rho < 1, n_between >= 1, max_levels >= 1");
  const double kd = std::ceil(rho * (double)n);
  if (!(kd >= 1.0 && kd <= (double)(n - 1)))
    return fail(ESS_ERR_ARG, "need 1 <= ceil(rho n_samples) <= n_samples - 1");
  const int k = (int)kd;
  if ((long long)max_levels * n_between > 0x7fffffffLL)
    return fail(ESS_ERR_ARG, "step index overflow (max_levels * n_between)");
  DeviceGuard guard(s->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  s->n_loaded = 0;
  ess_status rc = ensure_capacity(s, n);
  if (rc != ESS_OK) return rc;
  const size_t esz = elem(s);
  HdrScratch w;
  ESS_CUDA(dev_alloc(&w.X64, (size_t)n * d));
  ESS_CUDA(cudaMalloc(&w.Xtmp, (size_t)n * d * esz));
  ESS_CUDA(dev_alloc(&w.g, (size_t)n));
  ESS_CUDA(dev_alloc(&w.list, (size_t)n));
  ESS_CUDA(dev_alloc(&w.gamma, 1));
  ESS_CUDA(dev_alloc(&w.count, 1));
  ESS_CUDA(dev_alloc(&w.b0, (size_t)m));
  ESS_CUDA(cudaMalloc(&w.slack0, (size_t)m * esz));
  ESS_CUDA(cudaMemcpyAsync(w.b0, s->b64, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  ESS_CUDA(cudaMemcpyAsync(w.slack0, s->slack, esz * m, cudaMemcpyDeviceToDevice, st));
  if (mixed(s)) {
    ESS_CUDA(dev_alloc(&w.b32_0, (size_t)m));
    ESS_CUDA(cudaMemcpyAsync(w.b32_0, s->b32, sizeof(float) * m, cudaMemcpyDeviceToDevice, st));
    if (s->cfg.refresh_mode != ESS_REFRESH_SPLIT) ESS_CUDA(dev_alloc(&w.P64, (size_t)n * m));
  }
  // the level bounds b - gamma can reach 0: the warp step takes long arcs
  // as one union while they are in place (captured periods hold the flag)
  const int long_arcs0 = s->long_arcs;
  if (!s->long_arcs) {
    s->long_arcs = 1;
    drop_graphs(s);
  }
  // the saved bounds come back whatever happens below
  auto restore = [&]() {
    if (s->long_arcs != long_arcs0) {
      s->long_arcs = long_arcs0;
      drop_graphs(s);
    }
    cudaMemcpyAsync(s->b64, w.b0, sizeof(double) * m, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s->slack, w.slack0, esz * m, cudaMemcpyDeviceToDevice, st);
    if (w.b32_0) cudaMemcpyAsync(s->b32, w.b32_0, sizeof(float) * m, cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    s->n_loaded = 0;  // the states left are the last level's, not the caller's
  };
  ESS_CUDA(cudaMemsetAsync(s->dstatus, 0, sizeof(int), st));
  int T = 0;
  double lz[2] = {0.0, 0.0};
  for (int stage = 0; stage < 2 && rc == ESS_OK; ++stage) {
    const uint64_t seed_s = seed + (uint64_t)stage;
    // the stage's start samples: N(0, I) draws, Philox (seed_s, j, t = 0, problem 1)
    rc = [&]() -> ess_status {
      ESS_CUDA(ess::launch_draw_nu_f64(w.X64, n, d, d, seed_s, 0u, 1u, 0u, s->bm_tab, st));
      if (mixed(s)) ESS_CUDA((ess::launch_convert<double, float>(w.X64, d, s->Xw, d, n, d, st)));
      else ESS_CUDA((ess::launch_convert<double, double>(w.X64, d, s->Xd, d, n, d, st)));
      return ESS_OK;
    }();
    for (int level = 0; rc == ESS_OK; ++level) {
      const double* P = nullptr;
      rc = hdr_products(s, n, w, st, &P);
      if (rc != ESS_OK) break;
      rc = [&]() -> ess_status {
        ESS_CUDA(ess::launch_hdr_level(P, m, w.b0, n, m, w.g, st));
        ESS_CUDA(ess::launch_hdr_select(w.g, n, k, stage == 0 ? NAN : shifts[level], w.gamma,
                                        w.count, w.list, st));
        return ESS_OK;
      }();
      if (rc != ESS_OK) break;
      double gamma = 0.0;
      int cnt = 0;
      ESS_CUDA(cudaMemcpyAsync(&gamma, w.gamma, sizeof(double), cudaMemcpyDeviceToHost, st));
      ESS_CUDA(cudaMemcpyAsync(&cnt, w.count, sizeof(int), cudaMemcpyDeviceToHost, st));
      ESS_CUDA(cudaStreamSynchronize(st));
      if (stage == 0) {
        shifts[level] = gamma;
        if (counts_ss) counts_ss[level] = cnt;
        T = level + 1;
      } else if (counts) {
        counts[level] = cnt;
      }
      lz[stage] += cnt > 0 ? std::log((double)cnt / (double)n) : -INFINITY;
      if (gamma == 0.0 || cnt == 0) break;
      if (stage == 0 && level + 1 >= max_levels) {
        rc = fail(ESS_ERR_UNSUPPORTED,
                  "no level reached the domain within max_levels (the domain may be empty)");
        break;
      }
      if (stage == 1 && level + 1 >= T) break;
      // the next level: every sample restarts from a listed one, and the
      // chains run n_between steps on the shifted domain {A x <= b + gamma}
      rc = [&]() -> ess_status {
        if (mixed(s)) {
          ESS_CUDA(ess::launch_hdr_gather<float>(s->Xw, d, w.list, w.count, n, d,
                                                 static_cast<float*>(w.Xtmp), st));
          ESS_CUDA(cudaMemcpyAsync(s->Xw, w.Xtmp, sizeof(float) * n * d,
                                   cudaMemcpyDeviceToDevice, st));
        } else {
          ESS_CUDA(ess::launch_hdr_gather<double>(s->Xd, d, w.list, w.count, n, d,
                                                  static_cast<double*>(w.Xtmp), st));
          ESS_CUDA(cudaMemcpyAsync(s->Xd, w.Xtmp, sizeof(double) * n * d,
                                   cudaMemcpyDeviceToDevice, st));
        }
        ESS_CUDA(ess::launch_hdr_shift(w.b0, s->anorm, m, gamma, s->cfg.residual_margin, s->b64,
                                       mixed(s) ? s->b32 : nullptr, s->slack, mixed(s), st));
        return ESS_OK;
      }();
      if (rc != ESS_OK) break;
      rc = refresh_p(s, n, chain_states(s), false, false, st);
      if (rc != ESS_OK) break;
      s->n_loaded = n;
      s->t_next = level * n_between;
      s->p_fresh_t = s->t_next;
      rc = ess_chains_step(s, n_between, seed_s, nullptr, 0, st);
      if (rc == ESS_OK) rc = read_status(s, st);
    }
  }
  restore();
  if (rc != ESS_OK) return rc;
  *n_levels = T;
  *log_z = lz[1];
  if (log_z_ss) *log_z_ss = lz[0];
  return ESS_OK;
}

const char* ess_last_error(void) { return g_err.c_str(); }

}  // extern "C"
