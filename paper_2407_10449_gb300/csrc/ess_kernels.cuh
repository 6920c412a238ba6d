// ess_kernels.cuh -- launchers of the sampler's kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ess_common.cuh"

namespace ess {

// ---------------------------------------------------------------- draws ----
// nu[c, j] for chains chain0 .. chain0 + n_chains - 1 at step t (row stride ld);
// with t_dev set the step index is t + *t_dev (replayable CUDA graphs);
// bm_tab: the FP64 Box-Muller tables (bm_table_fill) in device memory.
cudaError_t launch_draw_nu_f64(double* nu, int n_chains, int d, int ld, uint64_t seed,
                               uint32_t t, uint32_t problem, uint32_t chain0,
                               const double* bm_tab, cudaStream_t s,
                               const unsigned* t_dev = nullptr);
// float nu plus (if split != nullptr) the two-way fp16 split of nu * kNuSplitScale
// (h0 = fp16(y), h1 = fp16(y - h0)), rows of ld16 elements; columns
// d .. ld16 - 1 of the split are left untouched.
cudaError_t launch_draw_nu_f32(float* nu, int ld, __half* const split[2], int ld16, int n_chains,
                               int d, uint64_t seed, uint32_t t, uint32_t problem, uint32_t chain0,
                               cudaStream_t s, const unsigned* t_dev = nullptr);
cudaError_t launch_philox_blocks(uint64_t seed, uint32_t chain, uint32_t t, uint32_t problem,
                                 uint32_t stream, int n_blocks, uint32_t* out, cudaStream_t s);

// ------------------------------------------------------------ conversion ---
// dst[r, j] = (To) src[r, j] for an rows x cols block with strides.
template <typename Ti, typename To>
cudaError_t launch_convert(const Ti* src, int lds, To* dst, int ldd, int rows, int cols,
                           cudaStream_t s);

// ------------------------------------------------------------ FP64 GEMM ----
// C[r, i] = sum_j X[r, j] * A[i, j] in FP64 (X: M x K, A: N x K, both K
// contiguous), stored as TOut.  If drift_stats != nullptr the previous
// content of C is compared first: max |C_new - C_old| / anorm[i] is folded
// into drift_stats->max_drift_bits.
template <typename TX, typename TOut>
cudaError_t launch_gemm_nt_f64(const TX* X, int ldx, const double* A, int lda, TOut* C, int ldc,
                               int M, int N, int K, const double* anorm, DevStats* drift_stats,
                               cudaStream_t s);

// Feasibility of start points: status |= kStatusInfeasible if any
// P[r, i] > b[i] (P computed in FP64).
cudaError_t launch_check_feasible(const double* P, int ldp, const double* b, int rows, int m,
                                  int* status, cudaStream_t s);

// Feasibility of states X (float or double) from a product P known to within
// bound * row_scale[r] * col_scale[i]; undecided entries recomputed in FP64.
template <typename TX>
cudaError_t launch_check_feasible_bounded(const double* P, int ldp, const double* b, int rows,
                                          int m, const float* row_scale, const float* col_scale,
                                          double bound, const TX* X, int ldx, const double* A,
                                          int d, int* status, cudaStream_t s);

// ------------------------------------------------------------ chain step ---
// One chain of a packed batch of problems (uneven d, m and chain counts).
struct ChainDesc {
  int d, m;             // the chain's problem size
  unsigned chain;       // Philox chain counter: the chain's index within its problem
  unsigned problem;     // Philox problem index
  long long x_off;      // element offset of the chain's row in X, X_out, NU, samples
  long long p_off;      // element offset of the chain's row in P_in, P_out, Q
  long long a_off;      // element offset of the problem's A64 (m x d, row-major)
  int b_off;            // element offset of the problem's b, b64, anorm, slack
  int dpad;             // row stride of the fp16 nu slices (d rounded up to 8)
  long long h_off;      // element offset of the chain's row in the fp16 nu slices
  int long_arcs;        // the problem has rows with b_i <= 0 (see ChainParams)
};

template <typename T>
struct ChainParams {
  int d, m, n_chains;
  int ldx;              // row stride of X, X_out, NU (elements)
  int ldp;              // row stride of P_in, P_out, Q (elements)
  const T* P_in;        // carried p = A x (n_chains x m)
  T* P_out;             // next p (may alias P_in)
  const T* Q;           // q = A nu
  const T* b;           // m, in T
  const double* b64;    // m, exact b
  const double* A64;    // m x d, exact A (residual rechecks)
  const double* anorm;  // m, ||a_i||_2
  const T* slack;       // m, b_i - margin ||a_i|| rounded down (nullptr: computed from
                        // b64, margin and anorm)
  const T* X;           // current states
  T* X_out;             // next states (may alias X)
  const T* NU;          // nu (n_chains x d)
  const double* U;      // n_chains uniforms, or nullptr: drawn from Philox
  uint64_t seed;
  uint32_t t, problem, chain0;
  double trim_eps, tangent_thresh, margin;
  T* samples;           // nullptr or record target for this step
  long long sample_stride;  // elements between consecutive chains in samples
  double* theta_out;    // optional per-chain outputs
  double* pieces_out;
  int max_pieces;
  int* npieces_out;
  int* rejected_out;
  DevStats* stats;
  int* status;
  // CTA kernel, list mode: process the chains chain_list[0 .. *list_count)
  const int* chain_list;
  const int* list_count;
  // warp kernel: chains with too many arcs to sort in a warp are appended here
  int* overflow_list;
  int* overflow_count;
  // batch mode: per-chain problem views (d, m above are then the maxima and
  // ldx, ldp, chain0, problem, sample_stride are unused)
  const ChainDesc* desc;
  // if set, the step index is t + *t_dev (replayable CUDA graphs)
  const unsigned* t_dev;
  // streamed warp kernel: chain tickets (zero before each launch)
  int* work_counter;
  // wide-row kernel: per-CTA scratch slots of 4 wide_cap elements (arcs and
  // their merge-sort buffer, used when a chain's arcs outgrow shared memory)
  T* wide_scratch;
  long long wide_cap;
  // the problem has rows with b_i <= 0 (infeasible arcs of at least a half
  // circle, which together form one arc): the warp step then drops the arcs
  // inside that union; 0 skips the test (always correct, faster without such
  // rows).  Batch mode: per problem, ChainDesc::long_arcs.
  int long_arcs;
};

// The rows of one chain as a kernel sees them.
template <typename T>
struct ChainView {
  int d, m;
  const T* P;            // p (m)
  const T* Q;            // q (m)
  T* P_out;
  const T* X;            // x (d)
  const T* NU;           // nu (d)
  T* X_out;
  T* S;                  // sample row or nullptr
  const T* b;            // problem rows (m each)
  const double* b64;
  const double* anorm;
  const T* slack;
  const double* A64;     // m x d
  unsigned chain, problem, t;
  bool long_arcs;
};

template <typename T, bool BATCH>
__device__ __forceinline__ ChainView<T> chain_view(const ChainParams<T>& prm, int c) {
  ChainView<T> v;
  size_t xo, po;
  if constexpr (BATCH) {
    const ChainDesc cd = prm.desc[c];
    v.d = cd.d;
    v.m = cd.m;
    xo = (size_t)cd.x_off;
    po = (size_t)cd.p_off;
    v.b = prm.b + cd.b_off;
    v.b64 = prm.b64 + cd.b_off;
    v.anorm = prm.anorm + cd.b_off;
    v.slack = prm.slack ? prm.slack + cd.b_off : nullptr;
    v.A64 = prm.A64 + cd.a_off;
    v.chain = cd.chain;
    v.long_arcs = cd.long_arcs != 0;
    v.problem = cd.problem;
    v.S = prm.samples ? prm.samples + xo : nullptr;
  } else {
    v.d = prm.d;
    v.m = prm.m;
    xo = (size_t)c * prm.ldx;
    po = (size_t)c * prm.ldp;
    v.b = prm.b;
    v.b64 = prm.b64;
    v.anorm = prm.anorm;
    v.slack = prm.slack;
    v.A64 = prm.A64;
    v.chain = prm.chain0 + (unsigned)c;
    v.long_arcs = prm.long_arcs != 0;
    v.problem = prm.problem;
    v.S = prm.samples ? prm.samples + (size_t)c * prm.sample_stride : nullptr;
  }
  v.P = prm.P_in + po;
  v.Q = prm.Q + po;
  v.P_out = prm.P_out + po;
  v.X = prm.X + xo;
  v.NU = prm.NU + xo;
  v.X_out = prm.X_out + xo;
  v.t = prm.t + (prm.t_dev ? *prm.t_dev : 0u);
  return v;
}

template <typename T>
cudaError_t launch_chain_step(const ChainParams<T>& p, int threads, cudaStream_t s);

// One warp per chain: prune, sort up to kWarpSortCap arcs in registers, sweep,
// draw and move.  Chains with more arcs left after the prune are appended to
// p.overflow_list (untouched) for launch_chain_step in list mode, or, with
// p.overflow_list == nullptr (see chain_warp_local_fallback), stepped by the
// CTA-per-chain step inside the same launch.
// p.P_out must differ from p.P_in (a rejected move restores p from P_in).
template <typename T>
cudaError_t launch_chain_step_warp(const ChainParams<T>& p, cudaStream_t s);
template <typename T>
size_t chain_warp_smem_bytes(int m);
// Whether the warp kernel can step the chains it leaves itself, at the end of
// each CTA (launch with p.overflow_list == nullptr): float chains with m up to
// 2048 whose CTA-per-chain step fits the warp kernel's shared memory.
template <typename T>
bool chain_warp_local_fallback(int m, int d);
constexpr int kWarpSortCap = 128;

// One warp per chain, warps taking chains from *p.work_counter (zeroed before
// the launch), each chain's p and q rows streamed through shared memory in
// chunks by 1-D bulk copies (for the classification and again for the move).
// Float chains of one problem with m, d multiples of 4, m <= 4096 and 16-byte
// aligned rows (chain_stream_supported / chain_stream_aligned); chains with
// more than kWarpSortCap surviving arcs are appended to p.overflow_list
// (untouched) for launch_chain_step in list mode.  p.P_out must differ from
// p.P_in.
bool chain_stream_supported(int m, int d);
bool chain_stream_aligned(const ChainParams<float>& p);
cudaError_t launch_chain_step_stream(const ChainParams<float>& p, cudaStream_t s);

// ------------------------------------------------------------ wide rows ----
// One CTA per chain for any m up to kMaxRows: the rows are streamed (three
// passes), the exact arcs merged per alpha bucket, short arcs and the sort
// spilled to a per-CTA scratch slot when they outgrow shared memory
// (k_chain_wide.cu).  All chains of p (chain_list == nullptr) or, in list
// mode, the chains of p.chain_list[0 .. *p.list_count).  Single-problem
// chains only (p.desc == nullptr); p.P_out must differ from p.P_in.
// p.wide_scratch holds `slots` slots of 4 chain_wide_cap<T>(m) elements; the
// launch uses at most `slots` CTAs.
constexpr int kMaxRows = 1 << 22;  // rows a chain step takes (warp kernel's row code)
template <typename T>
size_t chain_wide_smem_bytes(int d);
template <typename T>
long long chain_wide_cap(int m);
int chain_wide_slots(int device);
template <typename T>
cudaError_t launch_chain_step_wide(const ChainParams<T>& p, int slots, cudaStream_t s);

// ------------------------------------------------------------ HDR levels ---
// The level steps of the normal-probability estimator (k_hdr.cu).
// g[j] = max_i (P[j, i] - b[i]) (NaN if a product is NaN), one warp per sample.
cudaError_t launch_hdr_level(const double* P, int ldp, const double* b, int n, int m, double* g,
                             cudaStream_t s);
// One CTA: gamma = shift, or (shift NaN) the midpoint of the k-th and
// (k + 1)-th smallest g (0 once the k-th is <= 0), 1 <= k <= n - 1; *count
// and list[0 .. count) = the samples with g <= gamma in index order.
cudaError_t launch_hdr_select(const double* g, int n, int k, double shift, double* gamma_out,
                              int* count_out, int* list, cudaStream_t s);
// dst[j] = src[list[j mod *count]] (rows of d elements, stride ld); nothing if
// *count is 0.
template <typename T>
cudaError_t launch_hdr_gather(const T* src, int ld, const int* list, const int* count, int n,
                              int d, T* dst, cudaStream_t s);
// b64 = b0 + gamma, b32 = float(b64) (if b32), slack = b64 - margin anorm
// (float rounded down, or double).
cudaError_t launch_hdr_shift(const double* b0, const double* anorm, int m, double gamma,
                             double margin, double* b64, float* b32, void* slack,
                             bool float_slack, cudaStream_t s);

// ------------------------------------------------------------ few chains ---
// FP64 chains of one polytope, 1 .. kMaxFew at a time: all steps of a run in
// one cooperative persistent kernel (k_few.cu).  Buffers (device):
//   X[2], NU[2]: C x d; P[2]: C x m; Q: C x m; bmin, bmax: C x kFewBuckets
//   (double bits); shorts: C x m x 2; nshort, rej[2], cur[2], bad, bad_prev:
//   C ints; theta, cth, sth: C doubles; bar: 2 unsigned (zero), abort_flag:
//   1 int (zero).
// Before the launch: bmin all kEmptyBucket, bmax, nshort, bad, bad_prev zero;
// cur[(t0 - 1) & 1] zero and rej[(t0 - 1) & 1] one (so that step t0 starts
// from buffer 0).  X_user holds the start points and receives the final
// states; samples (or null): C x n_rec x d, the state after every
// record_every-th step.
constexpr int kMaxFew = 16;
constexpr int kFewMaxM = 6144;
constexpr int kFewBuckets = 2048;
constexpr unsigned long long kEmptyBucket = 0x7FF0000000000000ull;  // +inf
struct FewArgs {
  const double* A;
  const double* b;
  const double* anorm;
  const double* bm_tab;
  int d, m, C, chunk;
  double* X[2];
  double* P[2];
  double* Q;
  double* NU[2];
  // arcs merged per bucket, short arcs and non-finite flags, one set per step
  // parity (phase D of step t reads the set that phase B of step t wrote;
  // step t + 1 clears it)
  unsigned long long* bmin[2];
  unsigned long long* bmax[2];
  double* shorts[2];
  int* nshort[2];
  double* theta;
  double* cth;
  double* sth;
  int* rej[2];
  int* cur[2];
  int* bad[2];
  int* bad_prev;
  unsigned* bar;
  int* abort_flag;
  double* X_user;
  double* samples;
  int record_every, n_rec;
  int t0, n_iter, refresh_k;
  uint64_t seed;
  double trim_eps, margin;
  DevStats* stats;
  int* status;
  unsigned long long wait_ns;  // bound of a grid-barrier wait
  int hold;                    // self-test: CTA 0 never arrives at the first barrier
};
// chunk of d staged per round in shared memory, and the dynamic shared memory
size_t few_chains_smem(int C, int m, int chunk);
int few_chains_chunk(int C, int d);
cudaError_t launch_few_chains(const FewArgs& args, cudaStream_t s);

// --------------------------------------------------------------- Cholesky ---
// Lower Cholesky factor of the row-major n x n matrix A (leading dimension
// lda), in place on its lower triangle (the strict upper triangle is left as
// it is); *info (device, zero on entry) receives the 1-based row of the first
// pivot that is not positive.
cudaError_t launch_cholesky(double* A, int n, int lda, int* info, cudaStream_t s);

// ---------------------------------------------------------------- batch ---
// A work item of the grouped GEMMs: rows row0 .. row0 + rows - 1 of one
// problem's A times `chains` consecutive chains of that problem, computed as
// an rtile x ctile tile (rows <= rtile, chains <= ctile, rtile ctile = 4096).
struct BatchItem {
  int row0, rows, chains;
  int rtile, ctile;
  int d, m;
  int b_off;           // element offset of the problem's b / anorm
  long long a_off;     // element offset of the problem's A (row 0)
  long long x_off;     // element offset of the first chain's row in X / NU
  long long p_off;     // element offset of the first chain's row in P / Q
  long long at_off;    // element offset of the problem's K-major copy of A (q GEMM)
  int mpad;            // row stride of that copy: m rounded up to 4 (zero padded)
  int dpad;            // row stride of the fp16 splits of A and nu (d rounded up to 8)
  long long ah_off;    // element offset of the problem's fp16 A splits (row 0)
  long long xh_off;    // element offset of the first chain's row in the fp16 nu splits
  int c_first;         // index of the first chain in the whole batch
  int pad_;
};
// Chain tile of a problem with n chains and m rows: the one of 16, 32 or 64
// chains (row tile 4096 / chain tile) whose items cover the fewest (row,
// chain) slots, ceil(m / rt) ceil(n / ct) rt ct; on a tie the smallest chain
// tile that holds n.  Every output is summed over k in the same order
// whatever the tile, so the choice changes no result.
inline int batch_rtile(int ctile) { return 4096 / ctile; }
inline int batch_ctile(int n, int m) {
  const int pref = n <= 16 ? 16 : n <= 32 ? 32 : 64;
  long long best = -1;
  int pick = pref;
  for (int ct : {pref, 16, 32, 64}) {
    const int rt = batch_rtile(ct);
    const long long slots = (long long)((m + rt - 1) / rt) * ((n + ct - 1) / ct) * rt * ct;
    if (best < 0 || slots < best) {
      best = slots;
      pick = ct;
    }
  }
  return pick;
}

// nu for every chain of the batch (T = float: float Box-Muller, T = double:
// 53-bit), written at desc[c].x_off; the step index is t (+ *t_dev if set).
// T = float with H0, H1 set also writes the fp16 split of nu * kNuSplitScale
// at desc[c].h_off (rows of desc[c].dpad).
// bm_tab: the FP64 Box-Muller tables (T = double; unused for float).
template <typename T>
cudaError_t launch_batch_draw(const ChainDesc* desc, int n_chains, T* NU, uint64_t seed,
                              uint32_t t, const unsigned* t_dev, const double* bm_tab,
                              cudaStream_t s, __half* H0 = nullptr, __half* H1 = nullptr);
// Scaled fp16 split of caller-supplied float nu rows (per chain: t = 2^(15-e)
// with max |nu| in [2^(e-1), 2^e); unscale[c] = 1 / t).
cudaError_t launch_batch_split(const ChainDesc* desc, int n_chains, const float* NU, __half* H0,
                               __half* H1, float* unscale, cudaStream_t s);
// Q = A nu per item, in T; AT holds every problem's A K-major (d x mpad at
// at_off); queue: one int of scratch (reset by the launcher).
template <typename T>
cudaError_t launch_batch_q(const BatchItem* items, int n_items, int* queue, const T* AT,
                           const T* NU, T* Q, cudaStream_t s);
// P = A64 X with FP64-class accuracy (see k_batch.cu); P64 and drift optional.
// T = float reads A64 as Ahi + Alo (A rounded to float and the float
// remainder), T = double reads A64 (Ahi, Alo unused).
template <typename T>
cudaError_t launch_batch_refresh(const BatchItem* items, int n_items, int* queue,
                                 const T* Ahi, const double* A64, const float* Alo, const T* X,
                                 T* P, double* P64, const double* anorm,
                                 unsigned long long* drift_bits, cudaStream_t s);
// status |= kStatusInfeasible if any P64 row entry exceeds b.
cudaError_t launch_batch_check(const ChainDesc* desc, int n_chains, const double* P64,
                               const double* b64, int* status, cudaStream_t s);
// *t_dev += by (advances the step index of a replayed CUDA graph); *t_dev = v.
cudaError_t launch_advance_t(unsigned* t_dev, unsigned by, cudaStream_t s);
cudaError_t launch_set_t(unsigned* t_dev, unsigned v, cudaStream_t s);

// Threads per chain the chain-step kernel uses for m constraints (0 if m is
// beyond the supported maximum), and the dynamic shared memory it needs.
int chain_threads_for(int m);
template <typename T>
size_t chain_smem_bytes(int threads, int d);
constexpr int kChainItems = 8;
constexpr int kChainMaxThreads = 1024;

}  // namespace ess
