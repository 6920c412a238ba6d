// ess_batch.cu -- extern "C" entry points of the batched sampler (include/ess.h,
// "batched problems"): hundreds of independent polytopes of uneven d and m,
// each with its own chain count, advanced together on one stream.
//
// Per step (all problems at once):
//   [refresh p = A x]  ->  draw nu  ->  q = A nu (grouped GEMM, work queue)
//   ->  chain step (warp per chain, CTA per chain for overflow chains)
// The chain of problem p with index k inside p draws from Philox with chain
// counter k and problem index p, so its trajectory is the one a one-problem
// run with that problem index produces.  Whole refresh periods (refresh plus
// refresh_k steps) are captured once in a CUDA graph and replayed, the step
// index coming from a device counter that the graph advances.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "ess.h"
#include "ess_kernels.cuh"
#include "ess_gemm_tc.cuh"
#include "ess_batch_persist.cuh"

void ess_internal_set_error(const std::string& msg);  // ess_abi.cu

using ess::BatchItem;
using ess::ChainDesc;
using ess::DevStats;

namespace {

ess_status bfail(ess_status st, const std::string& msg) {
  ess_internal_set_error(msg);
  return st;
}

ess_status bcuda(cudaError_t e, const char* what) {
  return bfail(e == cudaErrorMemoryAllocation ? ESS_ERR_OOM : ESS_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define BESS_CUDA(expr)                              \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return bcuda(e_, #expr);  \
  } while (0)

template <typename T>
void bfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
cudaError_t balloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

struct BDeviceGuard {
  int prev = -1;
  explicit BDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~BDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

struct ess_batch {
  int np = 0;
  ess_config cfg{};
  int device = 0;
  std::vector<int> d, m;
  std::vector<long long> a_off;  // per problem, into A64 / A32
  std::vector<int> b_off;        // per problem, into b, anorm, slack
  std::vector<int> long_arcs;    // per problem: some b_i <= 0
  std::vector<long long> at_off; // per problem, into AT (K-major copy, rows padded to 4)
  int max_d = 0, max_m = 0;
  int chain_threads = 0;         // CTA kernel width for max_m
  // constants (device)
  double* A64 = nullptr;
  float* A32 = nullptr;          // mixed form: A rounded to float (q GEMM, refresh hi part)
  float* Alo = nullptr;          // mixed form: A - A32 rounded to float (refresh lo part)
  void* AT = nullptr;            // FP64 form: K-major A (operand of the FMA q GEMM)
  __half* Ah[2] = {nullptr, nullptr};  // mixed form: fp16 splits of A s_i (rows of dpad)
  float* arow_unscale = nullptr;       // mixed form: 1 / s_i per row
  std::vector<long long> ah_off;       // per problem, into Ah
  std::vector<int> dpad;               // per problem: d rounded up to 8
  double* b64 = nullptr;
  float* b32 = nullptr;
  double* bm_tab = nullptr;      // FP64 Box-Muller tables (ess::bm_table_fill)
  double* anorm = nullptr;
  void* slack = nullptr;         // b - margin ||a||, rounded down in the step's type
  // current chain layout
  std::vector<int> nc;
  int n = 0;
  long long total_x = 0, total_p = 0;
  ChainDesc* desc = nullptr;
  BatchItem* items = nullptr;
  int n_items = 0;
  ess::TcBatchItem* titems = nullptr;  // mixed form: items of the tensor-core q GEMM
  ess::TcBatchItem* ptitems = nullptr; // the same items in the persistent launch's order
  int n_titems = 0, cap_titems = 0;
  CUtensorMap* tmaps = nullptr;  // mixed form: 4 operand maps per problem (A and nu splits)
  CUtensorMap* tmaps_alt = nullptr;  // the same maps over the second nu splits
  int layout_version = 0;
  // work buffers (device)
  int cap_n = 0, cap_items = 0;
  long long cap_x = 0, cap_p = 0;
  void* X = nullptr;             // working states (T)
  void* NU = nullptr;
  void* P = nullptr;
  void* P2 = nullptr;
  void* Q = nullptr;
  __half* H[2] = {nullptr, nullptr};  // mixed form: fp16 splits of nu (rows of dpad)
  // second nu buffers: the draw of step t + 1 runs beside step t
  void* NU_alt = nullptr;
  __half* H_alt[2] = {nullptr, nullptr};
  float* chain_unscale = nullptr;     // per chain 1 / t of caller-supplied nu
  long long cap_h = 0;
  double* P64 = nullptr;
  int* ovf = nullptr;            // [0] overflow count, [1..] overflow chains
  int* queue = nullptr;          // work-queue head of the grouped GEMMs
  unsigned* t_dev = nullptr;     // step index base of replayed graphs
  DevStats* dstats = nullptr;
  int* dstatus = nullptr;
  long long host_steps = 0;
  // CUDA graphs of one refresh period, keyed by layout, seed and P parity
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;   // graph capture: the steps (highest priority)
  cudaStream_t work_stream = nullptr;  // plain launches: the steps (highest priority)
  cudaStream_t side_stream = nullptr;  // the draws one step ahead (lowest priority)
  cudaEvent_t ev_drawn = nullptr, ev_done = nullptr, ev_fork = nullptr, ev_join = nullptr;
  // persistent launch (mixed form): a whole refresh period in one cooperative
  // kernel with work queues (ess_batch_set_persistent)
  bool persist = false;
  int* porder = nullptr;      // chain order of its work queue (largest m first)
  int* pqueue = nullptr;      // 2 ints per step: chain tickets, overflow count
  int cap_pqueue = 0;
  unsigned* pbar = nullptr;   // grid barrier state (2) and abort flag (1)
  int* pdep = nullptr;        // per problem: 4 x its q items, then the counters
  unsigned persist_hold = 0;  // 1 only inside ess_batch_selftest_wait
  long long persist_launches = 0;
  struct GraphEntry {
    int version;
    uint64_t seed;
    void* p_first;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  long long graph_launches = 0;
  // optional per-phase timing (direct launches only)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<int, int>>> ev_pending;
  int ev_used = 0;
  double phase_ms[ESS_N_PHASES] = {0};
  long long phase_launches[ESS_N_PHASES] = {0};
};

namespace {

bool bmixed(const ess_batch* s) { return s->cfg.precision == ESS_PREC_MIXED; }
size_t belem(const ess_batch* s) { return bmixed(s) ? sizeof(float) : sizeof(double); }

int bmark(ess_batch* s, cudaStream_t st) {
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

struct BPhase {
  ess_batch* s;
  cudaStream_t st;
  int phase, start, launches;
  BPhase(ess_batch* s_, cudaStream_t st_, int phase_, int launches_ = 1)
      : s(s_), st(st_), phase(phase_), start(bmark(s_, st_)), launches(launches_) {}
  ~BPhase() {
    s->phase_launches[phase] += launches;
    if (start < 0) return;
    const int stop = bmark(s, st);
    if (stop >= 0) s->ev_pending.push_back({phase, {start, stop}});
  }
};

void bcollect(ess_batch* s) {
  for (auto& pe : s->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ev_pool[pe.second.first], s->ev_pool[pe.second.second]) ==
        cudaSuccess)
      s->phase_ms[pe.first] += ms;
  }
  s->ev_pending.clear();
  s->ev_used = 0;
}

void drop_graphs(ess_batch* s) {
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

void free_work(ess_batch* s) {
  drop_graphs(s);
  bfree(s->desc);
  bfree(s->items);
  bfree(s->titems);
  bfree(s->ptitems);
  s->cap_titems = 0;
  if (s->tmaps) cudaFree(s->tmaps);
  if (s->tmaps_alt) cudaFree(s->tmaps_alt);
  s->tmaps = s->tmaps_alt = nullptr;
  if (s->X) cudaFree(s->X);
  if (s->NU) cudaFree(s->NU);
  if (s->NU_alt) cudaFree(s->NU_alt);
  s->NU_alt = nullptr;
  if (s->P) cudaFree(s->P);
  if (s->P2) cudaFree(s->P2);
  if (s->Q) cudaFree(s->Q);
  s->X = s->NU = s->P = s->P2 = s->Q = nullptr;
  for (auto& h : s->H) bfree(h);
  for (auto& h : s->H_alt) bfree(h);
  bfree(s->chain_unscale);
  s->cap_h = 0;
  bfree(s->P64);
  bfree(s->ovf);
  bfree(s->porder);
  s->cap_n = s->cap_items = 0;
  s->cap_x = s->cap_p = 0;
  s->nc.clear();
  s->n = 0;
}

// Builds the chain views and GEMM work items for chain counts nc and makes
// sure the work buffers hold them.
ess_status prepare(ess_batch* s, const int* nc_in) {
  std::vector<int> nc(nc_in, nc_in + s->np);
  for (int p = 0; p < s->np; ++p)
    if (nc[p] < 0) return bfail(ESS_ERR_ARG, "negative chain count");
  if (nc == s->nc && s->desc) return ESS_OK;
  std::vector<ChainDesc> desc;
  std::vector<BatchItem> items;
  std::vector<ess::TcBatchItem> titems;
  std::vector<long long> ho_of(s->np, 0);  // per problem: offset of its rows in the nu splits
  std::vector<int> ntile_of(s->np, 16);    // per problem: chain tile of the q GEMM
  long long xo = 0, po = 0, ho = 0;
  for (int p = 0; p < s->np; ++p) {
    const int d = s->d[p], m = s->m[p], dp = s->dpad[p];
    const int c_first = (int)desc.size();
    for (int k = 0; k < nc[p]; ++k) {
      ChainDesc cd{};
      cd.d = d;
      cd.m = m;
      cd.chain = (unsigned)k;
      cd.problem = (unsigned)p;
      cd.x_off = xo + (long long)k * d;
      cd.p_off = po + (long long)k * m;
      cd.a_off = s->a_off[p];
      cd.b_off = s->b_off[p];
      cd.dpad = dp;
      cd.h_off = ho + (long long)k * dp;
      cd.long_arcs = s->long_arcs[p];
      desc.push_back(cd);
    }
    const int ct = ess::batch_ctile(nc[p], m), rt = ess::batch_rtile(ct);
    for (int c0 = 0; c0 < nc[p]; c0 += ct)
      for (int r0 = 0; r0 < m; r0 += rt) {
        BatchItem it{};
        it.row0 = r0;
        it.rows = std::min(rt, m - r0);
        it.chains = std::min(ct, nc[p] - c0);
        it.rtile = rt;
        it.ctile = ct;
        it.d = d;
        it.m = m;
        it.b_off = s->b_off[p];
        it.a_off = s->a_off[p];
        it.at_off = s->at_off[p];
        it.mpad = (m + 3) & ~3;
        it.x_off = xo + (long long)c0 * d;
        it.p_off = po + (long long)c0 * m;
        it.dpad = dp;
        it.ah_off = bmixed(s) ? s->ah_off[p] : 0;
        it.xh_off = ho + (long long)c0 * dp;
        it.c_first = c_first + c0;
        items.push_back(it);
      }
    if (bmixed(s) && nc[p] > 0) {
      // tensor-core items: 128 rows of A_p x up to 64 of its chains (N = the
      // problem's chain count rounded up to 16, at most 64)
      const int nt = std::min(64, (nc[p] + 15) / 16 * 16);
      ho_of[p] = ho;
      ntile_of[p] = nt;
      for (int c0 = 0; c0 < nc[p]; c0 += 64)
        for (int r0 = 0; r0 < m; r0 += 128) {
          ess::TcBatchItem it{};
          it.problem = p;
          it.row0 = r0;
          it.rows = std::min(128, m - r0);
          it.chain0 = c0;
          it.chains = std::min(64, nc[p] - c0);
          it.ntile = nt;
          it.kblocks = (d + 63) / 64;
          it.m = m;
          it.q_off = po + (long long)c0 * m;
          it.urow = s->b_off[p] + r0;
          it.c_first = c_first + c0;
          titems.push_back(it);
        }
    }
    xo += (long long)nc[p] * d;
    po += (long long)nc[p] * m;
    ho += (long long)nc[p] * dp;
  }
  // largest items first: the work queue then ends on small items (LPT order)
  auto by_cost = [](const BatchItem& a, const BatchItem& b) {
    return (long long)a.rows * a.chains * a.d > (long long)b.rows * b.chains * b.d;
  };
  std::stable_sort(items.begin(), items.end(), by_cost);
  // persistent tensor-core kernel: CTA b takes items b, b + G, ...; largest first
  std::stable_sort(titems.begin(), titems.end(),
                   [](const ess::TcBatchItem& a, const ess::TcBatchItem& b) {
                     return (long long)a.rows * a.ntile * a.kblocks >
                            (long long)b.rows * b.ntile * b.kblocks;
                   });
  const int n = (int)desc.size();
  if (n > s->cap_n || xo > s->cap_x || po > s->cap_p ||
      (int)items.size() > s->cap_items || (int)titems.size() > s->cap_titems ||
      (bmixed(s) && ho > s->cap_h)) {
    free_work(s);
    const size_t e = belem(s);
    BESS_CUDA(balloc(&s->desc, std::max<size_t>(1, desc.size())));
    BESS_CUDA(balloc(&s->items, std::max<size_t>(1, items.size())));
    BESS_CUDA(balloc(&s->titems, std::max<size_t>(1, titems.size())));
    BESS_CUDA(balloc(&s->ptitems, std::max<size_t>(1, titems.size())));
    s->cap_titems = (int)titems.size();
    BESS_CUDA(cudaMalloc(&s->X, std::max<long long>(1, xo) * e));
    BESS_CUDA(cudaMalloc(&s->NU, std::max<long long>(1, xo) * e));
    BESS_CUDA(cudaMalloc(&s->NU_alt, std::max<long long>(1, xo) * e));
    BESS_CUDA(cudaMalloc(&s->P, std::max<long long>(1, po) * e));
    BESS_CUDA(cudaMalloc(&s->P2, std::max<long long>(1, po) * e));
    BESS_CUDA(cudaMalloc(&s->Q, std::max<long long>(1, po) * e));
    BESS_CUDA(balloc(&s->P64, std::max<long long>(1, po)));
    BESS_CUDA(balloc(&s->ovf, (size_t)n + 1));
    BESS_CUDA(balloc(&s->porder, std::max<size_t>(1, (size_t)n)));
    if (bmixed(s)) {
      for (int k = 0; k < 4; ++k) {
        __half*& h = k < 2 ? s->H[k] : s->H_alt[k - 2];
        BESS_CUDA(balloc(&h, (size_t)std::max<long long>(1, ho)));
        // the padding columns d .. dpad - 1 of every row stay zero
        BESS_CUDA(cudaMemset(h, 0, sizeof(__half) * (size_t)std::max<long long>(1, ho)));
      }
      BESS_CUDA(balloc(&s->chain_unscale, std::max<size_t>(1, (size_t)n)));
      s->cap_h = ho;
    }
    s->cap_n = n;
    s->cap_x = xo;
    s->cap_p = po;
    s->cap_items = (int)items.size();
  }
  if (!desc.empty()) {
    BESS_CUDA(cudaMemcpy(s->desc, desc.data(), sizeof(ChainDesc) * desc.size(), cudaMemcpyHostToDevice));
    // the persistent launch: its chain queue takes chains of the most rows
    // first (LPT order), problem by problem, and its q GEMM walks the items
    // problem by problem in the same order (largest first within a problem),
    // so the problems' q complete in about the order their chains are taken;
    // the dependency target of a problem is 4 counts (one per epilogue warp)
    // per item
    std::vector<int> order(desc.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return desc[a].m > desc[b].m; });
    std::vector<int> rank(s->np, 0), target(s->np, 0);
    for (int k = (int)order.size() - 1; k >= 0; --k) rank[desc[order[k]].problem] = k;
    for (const auto& it : titems) target[it.problem] += 4;
    std::vector<ess::TcBatchItem> pt(titems);
    std::stable_sort(pt.begin(), pt.end(), [&](const ess::TcBatchItem& a, const ess::TcBatchItem& b) {
      return rank[a.problem] < rank[b.problem];
    });
    BESS_CUDA(cudaMemcpy(s->porder, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    if (bmixed(s)) {
      if (!s->pdep) BESS_CUDA(balloc(&s->pdep, 2 * (size_t)s->np));
      BESS_CUDA(cudaMemcpy(s->pdep, target.data(), sizeof(int) * s->np, cudaMemcpyHostToDevice));
      if (!pt.empty())
        BESS_CUDA(cudaMemcpy(s->ptitems, pt.data(), sizeof(ess::TcBatchItem) * pt.size(),
                             cudaMemcpyHostToDevice));
    }
  }
  if (!items.empty())
    BESS_CUDA(cudaMemcpy(s->items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
  if (!titems.empty())
    BESS_CUDA(cudaMemcpy(s->titems, titems.data(), sizeof(ess::TcBatchItem) * titems.size(),
                         cudaMemcpyHostToDevice));
  if (bmixed(s)) {
    // operand maps of the tensor-core q GEMM (the nu splits may have moved),
    // one set per nu split buffer pair
    for (int set = 0; set < 2; ++set) {
      __half* const* hs = set == 0 ? s->H : s->H_alt;
      std::vector<CUtensorMap> maps((size_t)4 * s->np);
      std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
      for (int p = 0; p < s->np; ++p) {
        if (nc[p] == 0) continue;
        const int d = s->d[p], m = s->m[p], dp = s->dpad[p];
        for (int k = 0; k < 2; ++k) {
          BESS_CUDA(ess::tc_batch_map(&maps[4 * p + k], s->Ah[k] + s->ah_off[p], m, d, dp, 128));
          BESS_CUDA(ess::tc_batch_map(&maps[4 * p + 2 + k], hs[k] + ho_of[p], nc[p], d, dp,
                                      ntile_of[p]));
        }
      }
      CUtensorMap*& dst = set == 0 ? s->tmaps : s->tmaps_alt;
      if (!dst) BESS_CUDA(cudaMalloc(&dst, sizeof(CUtensorMap) * maps.size()));
      BESS_CUDA(cudaMemcpy(dst, maps.data(), sizeof(CUtensorMap) * maps.size(),
                           cudaMemcpyHostToDevice));
    }
  }
  drop_graphs(s);
  s->nc = nc;
  s->n = n;
  s->n_items = (int)items.size();
  s->n_titems = (int)titems.size();
  s->total_x = xo;
  s->total_p = po;
  ++s->layout_version;
  return ESS_OK;
}

ess_status bread_status(ess_batch* s, cudaStream_t st) {
  int h = 0;
  BESS_CUDA(cudaMemcpyAsync(&h, s->dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
  BESS_CUDA(cudaStreamSynchronize(st));
  if (h & ess::kStatusInfeasible)
    return bfail(ESS_ERR_INFEASIBLE_X0, "a chain state violates A x <= b (checked in FP64)");
  if (h & ess::kStatusNumeric)
    return bfail(ESS_ERR_NUMERIC, "NaN or Inf in theta or x; affected chains kept their state");
  if (h & ess::kStatusTimeout) return bfail(ESS_ERR_TIMEOUT, "a bounded device wait gave up");
  return ESS_OK;
}

// The hi part of A the refresh reads (A32 in the mixed form; unused in FP64).
template <typename T>
const T* ahi(const ess_batch* s) {
  if constexpr (sizeof(T) == 4) return s->A32;
  else return s->A64;
}

// p = A x for every chain (FP64-class), optionally with drift statistics and
// the FP64 feasibility check of the states.
template <typename T>
ess_status brefresh(ess_batch* s, const T* X, bool drift, bool check, cudaStream_t st) {
  BESS_CUDA(ess::launch_batch_refresh<T>(s->items, s->n_items, s->queue, ahi<T>(s), s->A64,
                                         s->Alo, X, static_cast<T*>(s->P),
                                         check ? s->P64 : nullptr, s->anorm,
                                         drift ? &s->dstats->max_drift_bits : nullptr, st));
  if (check) BESS_CUDA(ess::launch_batch_check(s->desc, s->n, s->P64, s->b64, s->dstatus, st));
  return ESS_OK;
}

// q = A nu for every chain.  Mixed form: FP16x3 on the tensor cores (the nu
// splits come from the draw kernel, or from a per-chain split of a
// caller-supplied nu when user_nu); FP64 form: FP64 FMAs.
template <typename T>
ess_status bq(ess_batch* s, bool user_nu, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (user_nu)
      BESS_CUDA(ess::launch_batch_split(s->desc, s->n, static_cast<const float*>(s->NU), s->H[0],
                                        s->H[1], s->chain_unscale, st));
    BESS_CUDA(ess::tc_batch_q(s->titems, s->n_titems, s->tmaps, s->arow_unscale,
                              user_nu ? s->chain_unscale : nullptr, static_cast<float*>(s->Q),
                              s->dstatus, st));
  } else {
    BESS_CUDA(ess::launch_batch_q<T>(s->items, s->n_items, s->queue, static_cast<const T*>(s->AT),
                                     static_cast<const T*>(s->NU), static_cast<T*>(s->Q), st));
  }
  return ESS_OK;
}

template <typename T>
ess::ChainParams<T> bparams(ess_batch* s) {
  ess::ChainParams<T> p{};
  p.d = s->max_d;
  p.m = s->max_m;
  p.n_chains = s->n;
  p.Q = static_cast<const T*>(s->Q);
  if constexpr (sizeof(T) == 4) p.b = reinterpret_cast<const T*>(s->b32);
  else p.b = reinterpret_cast<const T*>(s->b64);
  p.b64 = s->b64;
  p.A64 = s->A64;
  p.anorm = s->anorm;
  p.slack = static_cast<const T*>(s->slack);
  p.NU = static_cast<const T*>(s->NU);
  p.X = static_cast<const T*>(s->X);
  p.X_out = static_cast<T*>(s->X);
  p.trim_eps = s->cfg.trim_eps;
  p.tangent_thresh = s->cfg.tangent_thresh;
  p.margin = s->cfg.residual_margin;
  p.stats = s->dstats;
  p.status = s->dstatus;
  p.desc = s->desc;
  // the warp step compiles the long-arc union in if any problem has such rows
  // (each chain then follows its problem's ChainDesc::long_arcs)
  p.long_arcs = std::any_of(s->long_arcs.begin(), s->long_arcs.end(), [](int v) { return v != 0; });
  return p;
}

// Kernel launches of one chain step: the warp kernel alone when it steps the
// chains it leaves itself, else it and the CTA kernel.
int bchain_launches(const ess_batch* s) {
  return (bmixed(s) ? ess::chain_warp_local_fallback<float>(s->max_m, s->max_d)
                    : ess::chain_warp_local_fallback<double>(s->max_m, s->max_d)) ? 1 : 2;
}

// Chain step of every chain: warp kernel, then the CTA kernel for the chains
// it listed; reads P, writes P2 (the caller swaps them).
template <typename T>
ess_status bchain(ess_batch* s, ess::ChainParams<T> p, cudaStream_t st) {
  p.P_in = static_cast<const T*>(s->P);
  p.P_out = static_cast<T*>(s->P2);
  if (ess::chain_warp_local_fallback<T>(s->max_m, s->max_d)) {
    // the warp kernel steps the chains it leaves itself (one launch)
    p.overflow_count = nullptr;
    p.overflow_list = nullptr;
    BESS_CUDA(ess::launch_chain_step_warp<T>(p, st));
    return ESS_OK;
  }
  BESS_CUDA(cudaMemsetAsync(s->ovf, 0, sizeof(int), st));
  p.overflow_count = s->ovf;
  p.overflow_list = s->ovf + 1;
  BESS_CUDA(ess::launch_chain_step_warp<T>(p, st));
  p.chain_list = s->ovf + 1;
  p.list_count = s->ovf;
  p.overflow_count = nullptr;
  p.overflow_list = nullptr;
  BESS_CUDA(ess::launch_chain_step<T>(p, s->chain_threads, st));
  return ESS_OK;
}

// The internal streams and events of the draws made one step ahead: the steps
// at the highest priority, the draws at the lowest, so that a draw fills the
// SMs' room beside the q GEMM instead of delaying it.
ess_status bensure_streams(ess_batch* s) {
  if (s->cap_stream) return ESS_OK;
  int least = 0, greatest = 0;
  BESS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  BESS_CUDA(cudaStreamCreateWithPriority(&s->cap_stream, cudaStreamNonBlocking, greatest));
  BESS_CUDA(cudaStreamCreateWithPriority(&s->work_stream, cudaStreamNonBlocking, greatest));
  BESS_CUDA(cudaStreamCreateWithPriority(&s->side_stream, cudaStreamNonBlocking, least));
  for (cudaEvent_t* e : {&s->ev_drawn, &s->ev_done, &s->ev_fork, &s->ev_join})
    BESS_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return ESS_OK;
}

// The second nu buffers become the current ones (and the reverse).
void bswap_nu(ess_batch* s) {
  std::swap(s->NU, s->NU_alt);
  std::swap(s->H[0], s->H_alt[0]);
  std::swap(s->H[1], s->H_alt[1]);
  std::swap(s->tmaps, s->tmaps_alt);
}

// nu of step t (+ *t_dev when t_dev is set) of every chain into the second
// nu buffers (and their fp16 splits, mixed form).
template <typename T>
ess_status bdraw_alt(ess_batch* s, uint64_t seed, uint32_t t, const unsigned* t_dev,
                     cudaStream_t st) {
  BESS_CUDA(ess::launch_batch_draw<T>(s->desc, s->n, static_cast<T*>(s->NU_alt), seed, t, t_dev,
                                      s->bm_tab, st, s->H_alt[0], s->H_alt[1]));
  return ESS_OK;
}

// One step (draw, q, chain step) at step index t (+ *t_dev when t_dev is set);
// without `draw`, nu of step t is already in the current buffers.
template <typename T>
ess_status bstep(ess_batch* s, uint64_t seed, uint32_t t, const unsigned* t_dev, T* samples,
                 cudaStream_t st, bool draw = true) {
  if (draw) {
    BPhase ph(s, st, ESS_PHASE_DRAW);
    BESS_CUDA(ess::launch_batch_draw<T>(s->desc, s->n, static_cast<T*>(s->NU), seed, t, t_dev,
                                        s->bm_tab, st, s->H[0], s->H[1]));
  }
  {
    BPhase ph(s, st, ESS_PHASE_GEMM);
    ess_status rc = bq<T>(s, false, st);
    if (rc != ESS_OK) return rc;
  }
  ess::ChainParams<T> p = bparams<T>(s);
  p.seed = seed;
  p.t = t;
  p.t_dev = t_dev;
  p.samples = samples;
  BPhase ph(s, st, ESS_PHASE_CHAIN, bchain_launches(s));
  ess_status rc = bchain<T>(s, p, st);
  std::swap(s->P, s->P2);
  return rc;
}

// Replays (capturing on first use) the graph of one refresh period that
// starts at a step index held in *t_dev.
template <typename T>
ess_status bgraph_period(ess_batch* s, uint64_t seed, cudaStream_t st) {
  const int k = s->cfg.refresh_k;
  ess_batch::GraphEntry* hit = nullptr;
  for (auto& g : s->graphs)
    if (g.version == s->layout_version && g.seed == seed && g.p_first == s->P) hit = &g;
  if (!hit) {
    ess_status rs = bensure_streams(s);
    if (rs != ESS_OK) return rs;
    void* p_first = s->P;
    const bool timing = s->timing;
    s->timing = false;
    cudaStream_t cs = s->cap_stream, ss = s->side_stream;
    BESS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    // step j's nu is drawn on the side stream one step ahead (draw 0 beside
    // the refresh, draw j + 1 beside step j once step j - 1 is done); every
    // side operation is joined back before the step that reads it, and k is
    // even, so the period leaves the nu buffers where it found them
    ess_status rc = ESS_OK;
    auto cap_ok = [&](cudaError_t e, const char* what) {
      if (rc == ESS_OK && e != cudaSuccess) rc = bcuda(e, what);
      return rc == ESS_OK;
    };
    if (cap_ok(cudaEventRecord(s->ev_done, cs), "graph fork") &&
        cap_ok(cudaStreamWaitEvent(ss, s->ev_done, 0), "graph fork")) {
      bswap_nu(s);
      rc = bdraw_alt<T>(s, seed, 0u, s->t_dev, ss);  // into the current buffers
      bswap_nu(s);
      if (rc == ESS_OK) cap_ok(cudaEventRecord(s->ev_drawn, ss), "graph draw");
    }
    if (rc == ESS_OK) rc = brefresh<T>(s, static_cast<const T*>(s->X), true, false, cs);
    for (int j = 0; j < k && rc == ESS_OK; ++j) {
      if (!cap_ok(cudaStreamWaitEvent(cs, s->ev_drawn, 0), "graph join")) break;
      if (j + 1 < k) {
        if (j > 0 && !cap_ok(cudaStreamWaitEvent(ss, s->ev_done, 0), "graph fork")) break;
        rc = bdraw_alt<T>(s, seed, (uint32_t)(j + 1), s->t_dev, ss);
        if (rc != ESS_OK || !cap_ok(cudaEventRecord(s->ev_drawn, ss), "graph draw")) break;
      }
      rc = bstep<T>(s, seed, (uint32_t)j, s->t_dev, nullptr, cs, false);
      if (rc != ESS_OK || !cap_ok(cudaEventRecord(s->ev_done, cs), "graph step")) break;
      bswap_nu(s);
    }
    if (rc == ESS_OK) {
      cudaError_t e = ess::launch_advance_t(s->t_dev, (unsigned)k, cs);
      if (e != cudaSuccess) rc = bcuda(e, "advance step index");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    s->timing = timing;
    if (rc != ESS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return bcuda(ec, "graph capture");
    cudaGraphExec_t exec = nullptr;
    ec = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return bcuda(ec, "graph instantiate");
    // k is even, so the period leaves P where it found it
    if (s->P != p_first) std::swap(s->P, s->P2);
    s->graphs.push_back({s->layout_version, seed, p_first, exec});
    hit = &s->graphs.back();
  }
  BESS_CUDA(cudaGraphLaunch(hit->exec, st));
  ++s->graph_launches;
  s->phase_launches[ESS_PHASE_REFRESH] += 1;
  s->phase_launches[ESS_PHASE_DRAW] += k;
  s->phase_launches[ESS_PHASE_GEMM] += k;
  s->phase_launches[ESS_PHASE_CHAIN] += (long long)bchain_launches(s) * k;
  return ESS_OK;
}

// Replays (capturing on first use) one refresh period as the persistent
// launch: the refresh of p with the draw of step 0 beside it on the side
// stream, then one cooperative kernel for the period's refresh_k steps (q
// GEMM, draws of steps 1 .. k - 1, chain steps gated by per-problem q
// counters, overflow chains, steps joined by grid barriers), starting at the
// step index in *t_dev.
ess_status bpersist_period(ess_batch* s, uint64_t seed, cudaStream_t st) {
  const int k = s->cfg.refresh_k;
  ess_batch::GraphEntry* hit = nullptr;
  for (auto& g : s->graphs)
    if (g.version == s->layout_version && g.seed == seed && g.p_first == s->P) hit = &g;
  if (!hit) {
    ess_status rs = bensure_streams(s);
    if (rs != ESS_OK) return rs;
    if (s->cap_pqueue < ess::batch_persist_queue_ints(k)) {
      bfree(s->pqueue);
      BESS_CUDA(balloc(&s->pqueue, (size_t)ess::batch_persist_queue_ints(k)));
      s->cap_pqueue = ess::batch_persist_queue_ints(k);
    }
    if (!s->pbar) BESS_CUDA(balloc(&s->pbar, 3));
    ess::BatchPersistArgs a{};
    a.titems = s->ptitems;
    a.n_titems = s->n_titems;
    a.maps[0] = s->tmaps;
    a.maps[1] = s->tmaps_alt;
    a.arow_unscale = s->arow_unscale;
    a.Q = static_cast<float*>(s->Q);
    a.desc = s->desc;
    a.NU[0] = static_cast<float*>(s->NU);
    a.NU[1] = static_cast<float*>(s->NU_alt);
    for (int h = 0; h < 2; ++h) {
      a.H0[h] = h == 0 ? s->H[0] : s->H_alt[0];
      a.H1[h] = h == 0 ? s->H[1] : s->H_alt[1];
    }
    a.prm = bparams<float>(s);
    a.prm.seed = seed;
    a.prm.t = 0;
    a.prm.t_dev = s->t_dev;
    a.P[0] = static_cast<float*>(s->P);
    a.P[1] = static_cast<float*>(s->P2);
    a.order = s->porder;
    a.queue = s->pqueue;
    a.ovf_list = s->ovf + 1;
    a.steps = k;
    a.bar = s->pbar;
    a.abort_flag = reinterpret_cast<int*>(s->pbar + 2);
    a.dep_target = s->pdep;
    a.dep_done = reinterpret_cast<unsigned*>(s->pdep + s->np);
    a.hold = s->persist_hold;
    a.wait_ns = s->cfg.wait_limit_us > 0 ? 1000ull * (unsigned long long)s->cfg.wait_limit_us
                                         : 2000000000ull;
    void* p_first = s->P;
    cudaStream_t cs = s->cap_stream, ss = s->side_stream;
    BESS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    ess_status rc = ESS_OK;
    auto cap_ok = [&](cudaError_t e, const char* what) {
      if (rc == ESS_OK && e != cudaSuccess) rc = bcuda(e, what);
      return rc == ESS_OK;
    };
    if (cap_ok(cudaEventRecord(s->ev_done, cs), "graph fork") &&
        cap_ok(cudaStreamWaitEvent(ss, s->ev_done, 0), "graph fork")) {
      bswap_nu(s);
      rc = bdraw_alt<float>(s, seed, 0u, s->t_dev, ss);  // into the current buffers
      bswap_nu(s);
      if (rc == ESS_OK) cap_ok(cudaEventRecord(s->ev_drawn, ss), "graph draw");
    }
    if (rc == ESS_OK) rc = brefresh<float>(s, static_cast<const float*>(s->X), true, false, cs);
    if (rc == ESS_OK && cap_ok(cudaStreamWaitEvent(cs, s->ev_drawn, 0), "graph join") &&
        cap_ok(cudaMemsetAsync(s->pqueue, 0, sizeof(int) * ess::batch_persist_queue_ints(k), cs),
               "persistent queue reset") &&
        cap_ok(cudaMemsetAsync(s->pbar, 0, 3 * sizeof(unsigned), cs), "grid barrier reset") &&
        cap_ok(cudaMemsetAsync(s->pdep + s->np, 0, sizeof(int) * s->np, cs), "dependency reset"))
      cap_ok(ess::launch_batch_persist(a, cs), "persistent batched launch");
    if (rc == ESS_OK) cap_ok(ess::launch_advance_t(s->t_dev, (unsigned)k, cs), "advance step index");
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (rc != ESS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return bcuda(ec, "graph capture");
    cudaGraphExec_t exec = nullptr;
    ec = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return bcuda(ec, "graph instantiate");
    s->graphs.push_back({s->layout_version, seed, p_first, exec});
    hit = &s->graphs.back();
  }
  BESS_CUDA(cudaGraphLaunch(hit->exec, st));
  ++s->graph_launches;
  ++s->persist_launches;
  s->phase_launches[ESS_PHASE_REFRESH] += 1;
  s->phase_launches[ESS_PHASE_DRAW] += 1;
  s->phase_launches[ESS_PHASE_CHAIN] += 1;
  return ESS_OK;
}

template <typename T>
ess_status brun(ess_batch* s, double* X, int t0, int n_iter, uint64_t seed, void* samples,
                int record_every, cudaStream_t st) {
  T* Xw = static_cast<T*>(s->X);
  BESS_CUDA(cudaMemsetAsync(s->dstatus, 0, sizeof(int), st));
  BESS_CUDA((ess::launch_convert<double, T>(X, (int)s->total_x, Xw, (int)s->total_x, 1,
                                            (int)s->total_x, st)));
  ess_status rc = brefresh<T>(s, Xw, false, true, st);
  if (rc == ESS_OK) rc = bread_status(s, st);
  if (rc != ESS_OK) return rc;
  const int k = s->cfg.refresh_k;
  const int n_rec = record_every > 0 ? n_iter / record_every : 0;
  const bool graphs_ok = s->use_graphs && !s->timing && record_every == 0 && k % 2 == 0;
  // Unless per-phase timing is on, the steps run on the internal high-priority
  // work stream and each plain step t that another plain step follows draws
  // nu of step t + 1 on the low-priority side stream beside it; both streams
  // are forked from st here and joined back after the loop.
  const bool ahead = !s->timing && n_iter > 1;
  cudaStream_t wst = st;
  if (ahead) {
    rc = bensure_streams(s);
    if (rc != ESS_OK) return rc;
    BESS_CUDA(cudaEventRecord(s->ev_fork, st));
    BESS_CUDA(cudaStreamWaitEvent(s->work_stream, s->ev_fork, 0));
    wst = s->work_stream;
  }
  int fresh = t0;
  auto graph_at = [&](int it_) {
    const int t_ = t0 + it_;
    return graphs_ok && t_ % k == 0 && t_ != fresh && n_iter - it_ >= k;
  };
  auto loop = [&]() -> ess_status {
    bool drawn = false;  // the current nu buffers hold step t's draw
    int it = 0;
    while (it < n_iter) {
      const int t = t0 + it;
      if (graph_at(it)) {
        BESS_CUDA(ess::launch_set_t(s->t_dev, (unsigned)t, wst));
        while (n_iter - it >= k) {
          ess_status r = (sizeof(T) == 4 && s->persist) ? bpersist_period(s, seed, wst)
                                                        : bgraph_period<T>(s, seed, wst);
          if (r != ESS_OK) return r;
          it += k;
        }
        fresh = t0 + it - k;
        continue;
      }
      const bool next = ahead && it + 1 < n_iter && !graph_at(it + 1);
      if (next) {
        BESS_CUDA(cudaEventRecord(s->ev_done, wst));  // step t - 1 is done here
        BESS_CUDA(cudaStreamWaitEvent(s->side_stream, s->ev_done, 0));
        ess_status r = bdraw_alt<T>(s, seed, (uint32_t)(t + 1), nullptr, s->side_stream);
        if (r != ESS_OK) return r;
        s->phase_launches[ESS_PHASE_DRAW] += 1;
        BESS_CUDA(cudaEventRecord(s->ev_drawn, s->side_stream));
      }
      if (t % k == 0 && t != fresh) {
        BPhase ph(s, wst, ESS_PHASE_REFRESH);
        ess_status r = brefresh<T>(s, Xw, true, false, wst);
        if (r != ESS_OK) return r;
        fresh = t;
      }
      const bool rec = record_every > 0 && (it + 1) % record_every == 0 &&
                       (it + 1) / record_every <= n_rec;
      T* srow = rec ? static_cast<T*>(samples) + (long long)((it + 1) / record_every - 1) * s->total_x
                    : nullptr;
      ess_status r = bstep<T>(s, seed, (uint32_t)t, nullptr, srow, wst, !drawn);
      if (r != ESS_OK) return r;
      if (next) {
        // step t + 1 reads the buffers just drawn, after the draw
        bswap_nu(s);
        BESS_CUDA(cudaStreamWaitEvent(wst, s->ev_drawn, 0));
      }
      drawn = next;
      ++it;
    }
    return ESS_OK;
  };
  rc = loop();
  if (ahead) {
    // join even after an error: no internal work may outlive st's order
    cudaError_t e = cudaEventRecord(s->ev_join, s->work_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->ev_join, 0);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_join, s->side_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->ev_join, 0);
    if (e != cudaSuccess && rc == ESS_OK) rc = bcuda(e, "join internal streams");
  }
  if (rc != ESS_OK) return rc;
  BESS_CUDA((ess::launch_convert<T, double>(Xw, (int)s->total_x, X, (int)s->total_x, 1,
                                            (int)s->total_x, st)));
  s->host_steps += (long long)s->n * n_iter;
  rc = bread_status(s, st);
  bcollect(s);
  return rc;
}

}  // namespace

extern "C" {

ess_status ess_batch_create(int n_problems, const int* d, const int* m, const double* A,
                            const double* b, const ess_config* cfg, ess_batch** out) {
  ess_internal_set_error("");
  if (!out) return bfail(ESS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_problems < 1 || !d || !m || !A || !b) return bfail(ESS_ERR_ARG, "bad argument");
  ess_config c;
  if (cfg) c = *cfg;
  else ess_default_config(ESS_PREC_FP64, &c);
  if (c.precision != ESS_PREC_FP64 && c.precision != ESS_PREC_MIXED)
    return bfail(ESS_ERR_ARG, "unknown precision");
  if (c.refresh_k < 1) return bfail(ESS_ERR_ARG, "refresh_k must be >= 1");
  if (!(c.trim_eps >= 0.0) || !(c.tangent_thresh >= 0.0) || !(c.residual_margin >= 0.0))
    return bfail(ESS_ERR_ARG, "negative tolerance");
  ess_batch* s = new ess_batch();
  s->np = n_problems;
  s->cfg = c;
  cudaGetDevice(&s->device);
  long long ta = 0, tat = 0, tah = 0;
  int tb = 0;
  for (int p = 0; p < n_problems; ++p) {
    if (d[p] < 1 || m[p] < 1) {
      delete s;
      return bfail(ESS_ERR_ARG, "need d >= 1 and m >= 1 for every problem");
    }
    s->d.push_back(d[p]);
    s->m.push_back(m[p]);
    s->a_off.push_back(ta);
    s->b_off.push_back(tb);
    int long_arcs = 0;  // rows with b_i <= 0 (see ChainParams::long_arcs)
    for (int i = 0; b && i < m[p]; ++i) long_arcs |= b[tb + i] <= 0.0 ? 1 : 0;
    s->long_arcs.push_back(long_arcs);
    s->at_off.push_back(tat);
    tat += (long long)d[p] * ((m[p] + 3) & ~3);
    s->dpad.push_back((d[p] + 7) & ~7);
    s->ah_off.push_back(tah);
    tah += (long long)m[p] * ((d[p] + 7) & ~7);
    ta += (long long)m[p] * d[p];
    tb += m[p];
    s->max_d = std::max(s->max_d, d[p]);
    s->max_m = std::max(s->max_m, m[p]);
  }
  for (long long i = 0; i < ta; ++i)
    if (!std::isfinite(A[i])) {
      delete s;
      return bfail(ESS_ERR_ARG, "A has a non-finite entry");
    }
  for (int i = 0; i < tb; ++i)
    if (!std::isfinite(b[i])) {
      delete s;
      return bfail(ESS_ERR_ARG, "b has a non-finite entry");
    }
  if (bmixed(s))
    for (int p = 0; p < n_problems; ++p)
      if (!ess::rows_fit_float_scales(A + s->a_off[p], b + s->b_off[p], m[p], d[p], true, 30)) {
        delete s;
        return bfail(ESS_ERR_ARG,
                     "a row of A or an entry of b is outside the mixed form's float scaling "
                     "range (nonzero row maxima in [2^-30, 2^30], |b| <= 2^30)");
      }
  s->chain_threads = ess::chain_threads_for(s->max_m);
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
  const size_t need = bmixed(s) ? ess::chain_smem_bytes<float>(s->chain_threads, s->max_d)
                                : ess::chain_smem_bytes<double>(s->chain_threads, s->max_d);
  if (s->chain_threads == 0 || (long long)need > (long long)smem_optin - 1024) {
    delete s;
    return bfail(ESS_ERR_UNSUPPORTED, "a problem is larger than the chain-step kernels support");
  }
  auto cleanup = [&](cudaError_t e) {
    ess_batch_destroy(s);
    return bcuda(e, "ess_batch_create device setup");
  };
  BDeviceGuard g(s->device);
  std::vector<double> norms(tb);
  for (int p = 0; p < n_problems; ++p)
    for (int i = 0; i < m[p]; ++i) {
      const double* a = A + s->a_off[p] + (long long)i * d[p];
      double acc = 0.0;
      for (int j = 0; j < d[p]; ++j) acc += a[j] * a[j];
      norms[s->b_off[p] + i] = std::sqrt(acc);
    }
  const size_t esz = belem(s);
  std::vector<unsigned char> sl(esz * tb);
  for (int i = 0; i < tb; ++i) {
    const double v = b[i] - c.residual_margin * norms[i];
    if (bmixed(s)) {
      float f = (float)v;
      if ((double)f > v) f = std::nextafter(f, -INFINITY);
      std::memcpy(&sl[esz * i], &f, esz);
    } else {
      std::memcpy(&sl[esz * i], &v, esz);
    }
  }
  cudaError_t e = balloc(&s->A64, (size_t)ta);
  if (e == cudaSuccess) e = cudaMemcpy(s->A64, A, sizeof(double) * ta, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = balloc(&s->b64, (size_t)tb);
  if (e == cudaSuccess) e = cudaMemcpy(s->b64, b, sizeof(double) * tb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = balloc(&s->anorm, (size_t)tb);
  if (e == cudaSuccess) e = cudaMemcpy(s->anorm, norms.data(), sizeof(double) * tb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&s->slack, esz * tb);
  if (e == cudaSuccess) e = cudaMemcpy(s->slack, sl.data(), esz * tb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && bmixed(s)) {
    std::vector<float> a32(ta), alo(ta), b32(tb);
    for (long long i = 0; i < ta; ++i) {
      a32[i] = (float)A[i];
      alo[i] = (float)(A[i] - (double)a32[i]);
    }
    for (int i = 0; i < tb; ++i) b32[i] = (float)b[i];
    e = balloc(&s->A32, (size_t)ta);
    if (e == cudaSuccess) e = cudaMemcpy(s->A32, a32.data(), sizeof(float) * ta, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = balloc(&s->Alo, (size_t)ta);
    if (e == cudaSuccess) e = cudaMemcpy(s->Alo, alo.data(), sizeof(float) * ta, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = balloc(&s->b32, (size_t)tb);
    if (e == cudaSuccess) e = cudaMemcpy(s->b32, b32.data(), sizeof(float) * tb, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && bmixed(s)) {
    // fp16 splits of every row a_i s_i, s_i = 2^(15 - e_i) with max_j |a_ij| in
    // [2^(e_i - 1), 2^e_i) (A rounded to float first), rows padded to dpad
    std::vector<__half> h0((size_t)std::max<long long>(1, tah), __float2half_rn(0.f)), h1 = h0;
    std::vector<float> ru(tb);
    for (int p = 0; p < n_problems; ++p)
      for (int i = 0; i < m[p]; ++i) {
        const double* a = A + s->a_off[p] + (long long)i * d[p];
        float mx = 0.f;
        for (int j = 0; j < d[p]; ++j) mx = std::fmax(mx, std::fabs((float)a[j]));
        int ex = 0;
        if (mx > 0.f) (void)std::frexp(mx, &ex);
        const float t = mx > 0.f ? std::ldexp(1.f, 15 - ex) : 1.f;
        ru[s->b_off[p] + i] = mx > 0.f ? std::ldexp(1.f, ex - 15) : 0.f;
        const size_t o = (size_t)(s->ah_off[p] + (long long)i * s->dpad[p]);
        for (int j = 0; j < d[p]; ++j) {
          const float y = (float)a[j] * t;
          const __half hv = __float2half_rn(y);
          h0[o + j] = hv;
          h1[o + j] = __float2half_rn(y - __half2float(hv));
        }
      }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = balloc(&s->Ah[k], h0.size());
      if (e == cudaSuccess)
        e = cudaMemcpy(s->Ah[k], (k ? h1 : h0).data(), sizeof(__half) * h0.size(),
                       cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = balloc(&s->arow_unscale, (size_t)tb);
    if (e == cudaSuccess)
      e = cudaMemcpy(s->arow_unscale, ru.data(), sizeof(float) * tb, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && !bmixed(s)) {
    // K-major copy of every A_p (rows padded to a multiple of 4 with zeros)
    std::vector<unsigned char> at((size_t)tat * esz, 0);
    for (int p = 0; p < n_problems; ++p) {
      const int mp = (m[p] + 3) & ~3;
      for (int i = 0; i < m[p]; ++i)
        for (int k = 0; k < d[p]; ++k) {
          const double v = A[s->a_off[p] + (long long)i * d[p] + k];
          const size_t o = (size_t)(s->at_off[p] + (long long)k * mp + i);
          if (bmixed(s)) {
            const float f = (float)v;
            std::memcpy(&at[o * esz], &f, esz);
          } else {
            std::memcpy(&at[o * esz], &v, esz);
          }
        }
    }
    e = cudaMalloc(&s->AT, std::max<size_t>(1, at.size()));
    if (e == cudaSuccess) e = cudaMemcpy(s->AT, at.data(), at.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = balloc(&s->queue, 1);
  if (e == cudaSuccess) e = balloc(&s->t_dev, 1);
  if (e == cudaSuccess) {
    std::vector<double> tab(ess::kBmTableSize);
    ess::bm_table_fill(tab.data());
    e = balloc(&s->bm_tab, tab.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(s->bm_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = balloc(&s->dstats, 1);
  if (e == cudaSuccess) e = balloc(&s->dstatus, 1);
  if (e == cudaSuccess) e = cudaMemset(s->dstats, 0, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(s->dstatus, 0, sizeof(int));
  if (e != cudaSuccess) return cleanup(e);
  // mixed form: refresh periods run as one persistent launch where the device
  // holds it (ess_batch_set_persistent switches back to per-step graphs)
  if (bmixed(s)) s->persist = ess::batch_persist_supported(s->max_m, s->max_d);
  cudaGetLastError();  // an unsupported probe leaves no error behind
  *out = s;
  return ESS_OK;
}

void ess_batch_destroy(ess_batch* s) {
  if (!s) return;
  BDeviceGuard g(s->device);
  free_work(s);
  bfree(s->A64);
  bfree(s->A32);
  bfree(s->Alo);
  if (s->AT) cudaFree(s->AT);
  bfree(s->Ah[0]);
  bfree(s->Ah[1]);
  bfree(s->arow_unscale);
  bfree(s->b64);
  bfree(s->b32);
  bfree(s->anorm);
  if (s->slack) cudaFree(s->slack);
  bfree(s->queue);
  bfree(s->pqueue);
  bfree(s->pbar);
  bfree(s->pdep);
  bfree(s->t_dev);
  bfree(s->bm_tab);
  bfree(s->dstats);
  bfree(s->dstatus);
  for (cudaStream_t q : {s->cap_stream, s->work_stream, s->side_stream})
    if (q) cudaStreamDestroy(q);
  for (cudaEvent_t e : {s->ev_drawn, s->ev_done, s->ev_fork, s->ev_join})
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  delete s;
}

ess_status ess_batch_run(ess_batch* s, const int* n_chains, double* X, int t0, int n_iter,
                         uint64_t seed, void* samples, int record_every, void* cuda_stream) {
  ess_internal_set_error("");
  if (!s || !n_chains) return bfail(ESS_ERR_ARG, "NULL argument");
  if (n_iter < 0 || t0 < 0 || record_every < 0) return bfail(ESS_ERR_ARG, "negative size");
  if ((long long)t0 + n_iter > 0x7fffffffLL) return bfail(ESS_ERR_ARG, "step index overflow");
  if (record_every > 0 && !samples) return bfail(ESS_ERR_ARG, "samples is NULL");
  BDeviceGuard g(s->device);
  ess_status rc = prepare(s, n_chains);
  if (rc != ESS_OK) return rc;
  if (s->n == 0) return ESS_OK;
  if (!X) return bfail(ESS_ERR_ARG, "X is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return bmixed(s) ? brun<float>(s, X, t0, n_iter, seed, samples, record_every, st)
                   : brun<double>(s, X, t0, n_iter, seed, samples, record_every, st);
}

ess_status ess_batch_selftest_wait(ess_batch* s, const int* n_chains, double* X) {
  ess_internal_set_error("");
  if (!s || !n_chains || !X) return bfail(ESS_ERR_ARG, "NULL argument");
  if (!bmixed(s) || !s->persist)
    return bfail(ESS_ERR_UNSUPPORTED, "the self-test runs the persistent launch (mixed form)");
  if (s->cfg.refresh_k % 2) return bfail(ESS_ERR_UNSUPPORTED, "refresh_k must be even");
  BDeviceGuard g(s->device);
  ess_status rc = prepare(s, n_chains);
  if (rc != ESS_OK) return rc;
  if (s->n == 0) return bfail(ESS_ERR_ARG, "no chains");
  const bool graphs = s->use_graphs, timing = s->timing;
  s->use_graphs = true;
  s->timing = false;
  // a period captured with the hold: the first refresh period runs plain
  // steps, the second one the persistent launch
  drop_graphs(s);
  s->persist_hold = 1;
  rc = brun<float>(s, X, 0, 2 * s->cfg.refresh_k, 0, nullptr, 0, nullptr);
  s->persist_hold = 0;
  drop_graphs(s);
  s->use_graphs = graphs;
  s->timing = timing;
  return rc;
}

ess_status ess_batch_step_with_draws(ess_batch* s, const int* n_chains, const double* X,
                                     const double* nu, const double* u, double* X_next,
                                     double* theta, int* rejected, void* cuda_stream) {
  ess_internal_set_error("");
  if (!s || !n_chains) return bfail(ESS_ERR_ARG, "NULL argument");
  BDeviceGuard g(s->device);
  ess_status rc = prepare(s, n_chains);
  if (rc != ESS_OK) return rc;
  if (s->n == 0) return ESS_OK;
  if (!X || !nu || !u || !X_next) return bfail(ESS_ERR_ARG, "NULL input");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  BESS_CUDA(cudaMemsetAsync(s->dstatus, 0, sizeof(int), st));
  const int tx = (int)s->total_x;
  auto one = [&](auto tag) -> ess_status {
    using T = decltype(tag);
    T* Xw = static_cast<T*>(s->X);
    BESS_CUDA((ess::launch_convert<double, T>(X, tx, Xw, tx, 1, tx, st)));
    BESS_CUDA((ess::launch_convert<double, T>(nu, tx, static_cast<T*>(s->NU), tx, 1, tx, st)));
    ess_status r = brefresh<T>(s, Xw, false, true, st);
    if (r == ESS_OK) r = bread_status(s, st);
    if (r != ESS_OK) return r;
    r = bq<T>(s, true, st);
    if (r != ESS_OK) return r;
    ess::ChainParams<T> p = bparams<T>(s);
    p.U = u;
    p.theta_out = theta;
    p.rejected_out = rejected;
    r = bchain<T>(s, p, st);
    std::swap(s->P, s->P2);
    if (r != ESS_OK) return r;
    BESS_CUDA((ess::launch_convert<T, double>(Xw, tx, X_next, tx, 1, tx, st)));
    s->host_steps += s->n;
    return bread_status(s, st);
  };
  return bmixed(s) ? one(float{}) : one(double{});
}

ess_status ess_batch_products(ess_batch* s, const int* n_chains, const double* X,
                              const double* nu, double* P, double* Q, void* cuda_stream) {
  ess_internal_set_error("");
  if (!s || !n_chains) return bfail(ESS_ERR_ARG, "NULL argument");
  BDeviceGuard g(s->device);
  ess_status rc = prepare(s, n_chains);
  if (rc != ESS_OK) return rc;
  if (s->n == 0) return ESS_OK;
  if ((P && !X) || (Q && !nu)) return bfail(ESS_ERR_ARG, "NULL input");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int tx = (int)s->total_x, tp = (int)s->total_p;
  auto one = [&](auto tag) -> ess_status {
    using T = decltype(tag);
    if (P) {
      BESS_CUDA((ess::launch_convert<double, T>(X, tx, static_cast<T*>(s->X), tx, 1, tx, st)));
      BESS_CUDA(ess::launch_batch_refresh<T>(s->items, s->n_items, s->queue, ahi<T>(s), s->A64,
                                             s->Alo, static_cast<const T*>(s->X), nullptr, P,
                                             s->anorm, nullptr, st));
    }
    if (Q) {
      BESS_CUDA((ess::launch_convert<double, T>(nu, tx, static_cast<T*>(s->NU), tx, 1, tx, st)));
      ess_status r = bq<T>(s, true, st);
      if (r != ESS_OK) return r;
      BESS_CUDA((ess::launch_convert<T, double>(static_cast<const T*>(s->Q), tp, Q, tp, 1, tp, st)));
    }
    BESS_CUDA(cudaStreamSynchronize(st));
    return ESS_OK;
  };
  return bmixed(s) ? one(float{}) : one(double{});
}

ess_status ess_batch_get_stats(const ess_batch* s, ess_stats* out) {
  if (!s || !out) return bfail(ESS_ERR_ARG, "NULL argument");
  BDeviceGuard g(s->device);
  DevStats h{};
  BESS_CUDA(cudaMemcpy(&h, s->dstats, sizeof(h), cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof(*out));
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

ess_status ess_batch_reset_stats(ess_batch* s) {
  if (!s) return bfail(ESS_ERR_ARG, "NULL argument");
  BDeviceGuard g(s->device);
  BESS_CUDA(cudaMemset(s->dstats, 0, sizeof(DevStats)));
  s->host_steps = 0;
  return ESS_OK;
}

ess_status ess_batch_set_graphs(ess_batch* s, int enable) {
  if (!s) return bfail(ESS_ERR_ARG, "NULL argument");
  s->use_graphs = enable != 0;
  return ESS_OK;
}

ess_status ess_batch_set_persistent(ess_batch* s, int enable) {
  if (!s) return bfail(ESS_ERR_ARG, "NULL argument");
  if (enable) {
    if (!bmixed(s))
      return bfail(ESS_ERR_UNSUPPORTED, "the persistent launch runs the mixed form only");
    BDeviceGuard g(s->device);
    if (!ess::batch_persist_supported(s->max_m, s->max_d))
      return bfail(ESS_ERR_UNSUPPORTED,
                   "the device cannot hold the persistent launch (cooperative launch, one "
                   "1024-thread CTA per SM) for these problem sizes");
  }
  if ((enable != 0) != s->persist) drop_graphs(s);  // captured periods hold the other form
  s->persist = enable != 0;
  return ESS_OK;
}

ess_status ess_batch_set_timing(ess_batch* s, int enable) {
  if (!s) return bfail(ESS_ERR_ARG, "NULL argument");
  s->timing = enable != 0;
  return ESS_OK;
}

ess_status ess_batch_get_timing(ess_batch* s, double* ms, long long* launches, int n_phases) {
  if (!s || n_phases < 0) return bfail(ESS_ERR_ARG, "bad argument");
  BDeviceGuard g(s->device);
  BESS_CUDA(cudaDeviceSynchronize());
  bcollect(s);
  for (int i = 0; i < n_phases && i < ESS_N_PHASES; ++i) {
    if (ms) ms[i] = s->phase_ms[i];
    if (launches) launches[i] = s->phase_launches[i];
  }
  return ESS_OK;
}

ess_status ess_batch_reset_timing(ess_batch* s) {
  if (!s) return bfail(ESS_ERR_ARG, "NULL argument");
  BDeviceGuard g(s->device);
  BESS_CUDA(cudaDeviceSynchronize());
  bcollect(s);
  for (int i = 0; i < ESS_N_PHASES; ++i) {
    s->phase_ms[i] = 0.0;
    s->phase_launches[i] = 0;
  }
  s->graph_launches = 0;
  return ESS_OK;
}

ess_status ess_batch_info(const ess_batch* s, long long* total_x, long long* total_p,
                          int* n_items, long long* graph_launches) {
  if (!s) return bfail(ESS_ERR_ARG, "NULL argument");
  if (total_x) *total_x = s->total_x;
  if (total_p) *total_p = s->total_p;
  if (n_items) *n_items = s->n_items;
  if (graph_launches) *graph_launches = s->graph_launches;
  return ESS_OK;
}

}  // extern "C"
