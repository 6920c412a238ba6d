// ess_kernels.cuh -- launchers of the sampler's kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ess_common.cuh"

namespace ess {

// ---------------------------------------------------------------- draws ----
// nu[c, j] for chains chain0 .. chain0 + n_chains - 1 at step t (row stride ld).
cudaError_t launch_draw_nu_f64(double* nu, int n_chains, int d, int ld, uint64_t seed,
                               uint32_t t, uint32_t problem, uint32_t chain0, cudaStream_t s);
// float nu plus (if split != nullptr) the two-way fp16 split of nu * kNuSplitScale
// (h0 = fp16(y), h1 = fp16(y - h0)), rows of ld16 elements; columns
// d .. ld16 - 1 of the split are left untouched.
cudaError_t launch_draw_nu_f32(float* nu, int ld, __half* const split[2], int ld16, int n_chains,
                               int d, uint64_t seed, uint32_t t, uint32_t problem, uint32_t chain0,
                               cudaStream_t s);
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

// Feasibility of float states X from a product P known to within
// bound * row_scale[r] * col_scale[i]; undecided entries recomputed in FP64.
cudaError_t launch_check_feasible_bounded(const double* P, int ldp, const double* b, int rows,
                                          int m, const float* row_scale, const float* col_scale,
                                          double bound, const float* X, int ldx, const double* A,
                                          int d, int* status, cudaStream_t s);

// ------------------------------------------------------------ chain step ---
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
};

template <typename T>
cudaError_t launch_chain_step(const ChainParams<T>& p, int threads, cudaStream_t s);

// One warp per chain: prune, sort up to kWarpSortCap arcs in registers, sweep,
// draw and move.  Chains with more arcs left after the prune are appended to
// p.overflow_list (untouched) for launch_chain_step in list mode.
// p.P_out must differ from p.P_in (a rejected move restores p from P_in).
template <typename T>
cudaError_t launch_chain_step_warp(const ChainParams<T>& p, cudaStream_t s);
template <typename T>
size_t chain_warp_smem_bytes(int m);
constexpr int kWarpSortCap = 128;

// Threads per chain the chain-step kernel uses for m constraints (0 if m is
// beyond the supported maximum), and the dynamic shared memory it needs.
int chain_threads_for(int m);
template <typename T>
size_t chain_smem_bytes(int threads, int d);
constexpr int kChainItems = 8;
constexpr int kChainMaxThreads = 1024;

}  // namespace ess
