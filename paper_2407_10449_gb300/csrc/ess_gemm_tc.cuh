// ess_gemm_tc.cuh -- tcgen05 (5th-generation tensor core) GEMM for q = A nu.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace ess {

struct TcGemmPlan;

// Prepares the constant operand: A (m x d) as bf16 hi/lo splits with row
// stride ld_bf elements (a multiple of 8).
cudaError_t tc_gemm_create(TcGemmPlan** plan, const __nv_bfloat16* A_hi, const __nv_bfloat16* A_lo,
                           int ld_bf, int m, int d);
void tc_gemm_destroy(TcGemmPlan* plan);

// Q[c, i] = sum_j (nu_hi nu_lo split of nu[c, :]) . (A_hi A_lo split of a_i)
// with the three products hi.hi + lo.hi + hi.lo accumulated in FP32 (the
// BF16x3 scheme), for chains c < n_chains.  Q has row stride ldq floats.
cudaError_t tc_gemm_bf16x3(TcGemmPlan* plan, const __nv_bfloat16* nu_hi,
                           const __nv_bfloat16* nu_lo, int ld_bf, int n_chains, float* Q, int ldq,
                           int* status, cudaStream_t s);

// Plain BF16 GEMM with one product per K block (used by tests of the
// tensor-core path): Q = X . B^T, X n x d, B m x d (bf16, stride ld_bf).
cudaError_t tc_gemm_bf16(const __nv_bfloat16* X, const __nv_bfloat16* B, int ld_bf, int n, int m,
                         int d, float* Q, int ldq, int* status, cudaStream_t s);

// Tile width (constraints per CTA) and pipeline depth chosen for a shape.
void tc_gemm_tile_for(int n_chains, int m, int* bn, int* stages);

}  // namespace ess
