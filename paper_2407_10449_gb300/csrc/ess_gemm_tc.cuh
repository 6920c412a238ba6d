// ess_gemm_tc.cuh -- tcgen05 (5th-generation tensor core) GEMMs of the mixed form.
#pragma once

#include <cstddef>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace ess {

struct TcGemmPlan;

// Prepares the constant operand A (host, m x d row-major doubles): the scaled
// two-way fp16 split of A rounded to float (for q = A nu; only if with_q) and
// the fixed-point slices of A with per-row power-of-two scales (for the exact
// products: ceil(exact_bits / w) slices of w bits).  Operand rows are padded
// to a multiple of 8 elements.
cudaError_t tc_gemm_create(TcGemmPlan** plan, const double* A, int m, int d,
                           int exact_bits = 35, bool with_q = true);
void tc_gemm_destroy(TcGemmPlan* plan);

// Q[c, i] = a_i . nu_c from the scaled fp16 splits nu_c t_c = h0 + h1 (rows of
// ld16 elements) and a_i s_i = a0 + a1, using the three products h0.a0,
// h1.a0, h0.a1 (FP16x3), accumulated in FP32 in tensor memory (the leading
// product in one accumulator, the other two in a second, added in the
// epilogue), then multiplied by 1 / s_i and 1 / t_c (powers of two).
// nu_unscale holds 1 / t_c per chain; nullptr means 1 / kNuSplitScale for all
// (drawn nu, see ess_common.cuh).
cudaError_t tc_gemm_q(TcGemmPlan* plan, __half* const nu[2], const float* nu_unscale, int ld16,
                      int n_chains, float* Q, int ldq, int* status, cudaStream_t s);

// Scaled fp16 split of float rows (see tc_gemm_q): per row t = 2^(15 - e) with
// max |v| in [2^(e-1), 2^e); unscale[row] = 1 / t.
cudaError_t tc_split2_rows(const float* src, int ld, int rows, int cols, __half* h0, __half* h1,
                           int ld16, float* unscale, cudaStream_t s);

// p = A x for float chain states X (n_chains x d, row stride ldx) with every
// product exact: x and A are cut into w-bit integer slices scaled by powers of
// two (t_c per chain, s_i per row), each slice pair's dot products are exact
// integers in the FP32 tensor-core accumulator ((2^w - 1)^2 d <= 2^24), and the
// pairs are combined error-free in (hi, lo) float pairs.  The result differs
// from A x by at most bound_factor * s_i * t_c (truncated slices and dropped
// pairs).  Writes P32 (rounded once to float) and/or P64; if drift_bits is
// set, folds max |P32_new - P32_old| / ||a_i|| (evaluated in FP32) into it
// (the bits of a non-negative double).  x_slices needs
// K x slice_stride bf16 (slice_stride >= n_chains * ld16) and row_scale
// n_chains floats of scratch.
cudaError_t tc_refresh(TcGemmPlan* plan, const float* X, int ldx, int n_chains,
                       __nv_bfloat16* x_slices, size_t slice_stride, float* row_scale,
                       float* P32, double* P64, int ldp, unsigned long long* drift_bits,
                       int* status, cudaStream_t s);

// ---- q = A_p nu for a batch of problems (mixed form) -------------------------
// One work item: rows row0 .. row0 + rows - 1 (rows <= 128) of problem
// `problem`'s A against its chains chain0 .. chain0 + chains - 1 (chains <= 64,
// ntile = chains rounded up to 16), over kblocks = ceil(d / 64) K blocks.  The
// operands come from maps[4 problem + k]: k = 0, 1 the scaled fp16 splits of
// A_p (m_p x d, row stride dpad, boxes of 128 rows x 64), k = 2, 3 those of the
// problem's nu rows (its chains x d, boxes of ntile rows x 64).
// Q[q_off + c m + row0 + r] = (h0.a0 + h1.a0 + h0.a1)(r, c) * arow_unscale[urow + r]
//   * (chain_unscale ? chain_unscale[c_first + c] : 1 / kNuSplitScale).
struct TcBatchItem {
  int problem, row0, rows, chain0, chains, ntile, kblocks, m;
  long long q_off;   // element offset of chain chain0's row of Q
  int urow;          // offset of row row0 in arow_unscale
  int c_first;       // batch index of chain chain0 (chain_unscale)
};
// 2-D map of a 16-bit operand (rows x cols, row stride ld elements) with boxes
// of box_rows x 64 elements, 128-byte swizzle, zero fill out of bounds.
cudaError_t tc_batch_map(CUtensorMap* map, const __half* base, int rows, int cols, int ld,
                         int box_rows);
cudaError_t tc_batch_q(const TcBatchItem* items, int n_items, const CUtensorMap* maps,
                       const float* arow_unscale, const float* chain_unscale, float* Q,
                       int* status, cudaStream_t s);

// FP64 products P64 = A x for double rows X with the same exact split (the
// plan's slices; with 56 bits the truncation leaves d (3 + K(K-1)/2) 2^-(wK)
// s_i t_c, e.g. 4e-13 s_i t_c at d = 1000), the N = K(K+1)/2 exact slice
// products summed into (hi, lo) float pairs (every addition error-free, the
// low parts summed in float: at most N^2 2^-48 sum_j |a_ij x_j| more) and
// rounded once to double; with drift_bits, max |P64_new - P64_old| / ||a_i||
// is folded in.
cudaError_t tc_exact_f64(TcGemmPlan* plan, const double* X, int ldx, int n_chains,
                         __nv_bfloat16* x_slices, size_t slice_stride, float* row_scale,
                         double* P64, int ldp, unsigned long long* drift_bits, int* status,
                         cudaStream_t s);

// Slice count K and width w of the exact products for dimension d and a
// budget of `bits` bits per operand.
int tc_refresh_slices(int d, int* w, int bits = 35);
int tc_refresh_num_slices(const TcGemmPlan* plan);
double tc_refresh_bound_factor(const TcGemmPlan* plan);
const float* tc_refresh_col_scale(const TcGemmPlan* plan);

// Tile of the q GEMM chosen for a shape: BN for one-SM tiles of 128 chains x
// BN rows of A, 2000 + BN for SM-pair tiles (tcgen05 cta_group::2) of 256
// chains x BN rows with one launch per tile, 3000 + BN for the same tiles in a
// persistent kernel (one cluster per SM pair, TMA-stored Q; used when the Q
// row stride is a multiple of 4 floats, else 2000 + BN).  *stages (if given)
// is set to 0.
void tc_gemm_tile_for(int n_chains, int m, int* bn, int* stages);
// Tile codes the q GEMM supports, and a fixed code for a plan (0: the cost
// model of tc_gemm_tile_for); the code tc_gemm_q uses for n_chains.
extern const int kTcWidths[16];
cudaError_t tc_gemm_set_width(TcGemmPlan* plan, int bn);
int tc_gemm_width(const TcGemmPlan* plan, int n_chains);

}  // namespace ess
