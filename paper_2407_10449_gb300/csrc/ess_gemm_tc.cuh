// ess_gemm_tc.cuh -- tcgen05 (5th-generation tensor core) GEMMs of the mixed form.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace ess {

struct TcGemmPlan;

// Prepares the constant operand A (host, m x d row-major doubles): the exact
// three-way bf16 split of A rounded to float (for q = A nu) and the
// fixed-point slices of A with per-row power-of-two scales (for the exact
// refresh).  Operand rows are padded to a multiple of 8 elements.
cudaError_t tc_gemm_create(TcGemmPlan** plan, const double* A, int m, int d);
void tc_gemm_destroy(TcGemmPlan* plan);

// Q[c, i] = a_i . nu_c with nu = nu0 + nu1 + nu2 (exact bf16 split of the
// float nu, rows of ld_bf elements) and a = a0 + a1 + a2, using the six
// products whose weight is at least 2^-16 (BF16x6), accumulated in FP32 in
// tensor memory: the leading product in one accumulator, the five smaller
// ones in a second, added in the epilogue.
cudaError_t tc_gemm_q(TcGemmPlan* plan, __nv_bfloat16* const nu[3], int ld_bf, int n_chains,
                      float* Q, int ldq, int* status, cudaStream_t s);

// Exact split of a float matrix into three bf16 slices (v = s0 + s1 + s2).
cudaError_t tc_split3(const float* src, int ld, int rows, int cols, __nv_bfloat16* s0,
                      __nv_bfloat16* s1, __nv_bfloat16* s2, int ld_bf, cudaStream_t s);

// p = A x for float chain states X (n_chains x d, row stride ldx) with every
// product exact: x and A are cut into w-bit integer slices scaled by powers of
// two (t_c per chain, s_i per row), each slice pair's dot products are exact
// integers in the FP32 tensor-core accumulator ((2^w - 1)^2 d <= 2^24), and the
// pairs are combined error-free in (hi, lo) float pairs.  The result differs
// from A x by at most bound_factor * s_i * t_c (truncated slices and dropped
// pairs).  Writes P32 (rounded once to float) and/or P64; if drift_bits is
// set, folds max |P32_new - P32_old| / anorm_i into it.  x_slices needs
// K x slice_stride bf16 (slice_stride >= n_chains * ld_bf) and row_scale
// n_chains floats of scratch.
cudaError_t tc_refresh(TcGemmPlan* plan, const float* X, int ldx, int n_chains,
                       __nv_bfloat16* x_slices, size_t slice_stride, float* row_scale,
                       float* P32, double* P64, int ldp, const double* anorm,
                       unsigned long long* drift_bits, int* status, cudaStream_t s);

// Slice count K and width w of the refresh for dimension d.
int tc_refresh_slices(int d, int* w);
int tc_refresh_num_slices(const TcGemmPlan* plan);
double tc_refresh_bound_factor(const TcGemmPlan* plan);
const float* tc_refresh_col_scale(const TcGemmPlan* plan);

// Tile width (constraints per CTA) and pipeline depth chosen for a shape.
void tc_gemm_tile_for(int n_chains, int m, int* bn, int* stages);

}  // namespace ess
