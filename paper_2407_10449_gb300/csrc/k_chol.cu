// k_chol.cu -- Cholesky factor Sigma = L L^T in FP64 on the GPU (App. A: the
// change of variables x = L u + mu needs L).
//
// Blocked right-looking factorisation with 64 x 64 blocks, in place on the
// lower triangle of a row-major matrix:
//   1. the diagonal block is factored in shared memory by one CTA (columns in
//      turn: pivot square root, column scaled, the block's trailing triangle
//      updated);
//   2. the panel below it is solved against L11^T, one row per thread
//      (forward substitution with L11 in shared memory);
//   3. the trailing matrix loses L21 L21^T: tiles of 64 x 64 on and below the
//      diagonal, both panels in shared memory, 4 x 4 outputs per thread.
// FP64 fused multiply-adds throughout: GB300's tensor cores have no FP64
// operand kind.  A pivot that is not positive (or not finite) records its
// 1-based row in *info; every later kernel sees it and returns at once.
#include <algorithm>
#include <cmath>

#include "ess_kernels.cuh"

namespace ess {
namespace {

constexpr int kNB = 64;

__global__ void chol_diag_kernel(double* __restrict__ A, int lda, int k, int nb,
                                 int* __restrict__ info) {
  __shared__ double s[kNB][kNB + 1];
  __shared__ int s_bad;
  if (*reinterpret_cast<volatile int*>(info) != 0) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < nb * nb; idx += nt) {
    const int r = idx / nb, c = idx % nb;
    s[r][c] = c <= r ? A[(size_t)(k + r) * lda + k + c] : 0.0;
  }
  if (tid == 0) s_bad = 0;
  for (int j = 0; j < nb; ++j) {
    __syncthreads();
    if (tid == 0) {
      const double v = s[j][j];
      if (!(v > 0.0) || !isfinite(v)) {
        s_bad = 1;
        atomicCAS(info, 0, k + j + 1);
      } else {
        s[j][j] = sqrt(v);
      }
    }
    __syncthreads();
    if (s_bad) return;
    const double djj = s[j][j];
    for (int i = j + 1 + tid; i < nb; i += nt) s[i][j] /= djj;
    __syncthreads();
    const int w = nb - j - 1;
    for (int idx = tid; idx < w * w; idx += nt) {
      const int i = j + 1 + idx / w, l = j + 1 + idx % w;
      if (l <= i) s[i][l] = fma(-s[i][j], s[l][j], s[i][l]);
    }
  }
  __syncthreads();
  for (int idx = tid; idx < nb * nb; idx += nt) {
    const int r = idx / nb, c = idx % nb;
    if (c <= r) A[(size_t)(k + r) * lda + k + c] = s[r][c];
  }
}

// rows k + nb .. n - 1 of the panel: x L11^T = a, one row per thread
constexpr int kTrsmRows = 128;
__global__ void chol_trsm_kernel(double* __restrict__ A, int lda, int k, int nb, int n,
                                 const int* __restrict__ info) {
  extern __shared__ double smem[];
  double* L11 = smem;                       // nb x (nb + 1)
  double* X = smem + (size_t)kNB * (kNB + 1);  // nb x (kTrsmRows + 1), X[j][row]
  if (*reinterpret_cast<const volatile int*>(info) != 0) return;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nb * nb; idx += kTrsmRows) {
    const int r = idx / nb, c = idx % nb;
    L11[r * (kNB + 1) + c] = c <= r ? A[(size_t)(k + r) * lda + k + c] : 0.0;
  }
  const int i = k + nb + blockIdx.x * kTrsmRows + tid;
  const bool valid = i < n;
  for (int j = 0; j < nb; ++j) X[j * (kTrsmRows + 1) + tid] = valid ? A[(size_t)i * lda + k + j] : 0.0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    double sum = X[j * (kTrsmRows + 1) + tid];
    for (int l = 0; l < j; ++l) sum = fma(-X[l * (kTrsmRows + 1) + tid], L11[j * (kNB + 1) + l], sum);
    X[j * (kTrsmRows + 1) + tid] = sum / L11[j * (kNB + 1) + j];
  }
  if (valid)
    for (int j = 0; j < nb; ++j) A[(size_t)i * lda + k + j] = X[j * (kTrsmRows + 1) + tid];
}

// trailing update T[i][l] -= sum_j L21[i][j] L21[l][j] on 64 x 64 tiles with
// l-tile <= i-tile (the lower triangle); 256 threads, 4 x 4 outputs each
__global__ void chol_syrk_kernel(double* __restrict__ A, int lda, int k, int nb, int n,
                                 const int* __restrict__ info) {
  extern __shared__ double smem[];
  double* Pi = smem;                          // nb x (64 + 1): Pi[j][row]
  double* Pl = smem + (size_t)kNB * (kNB + 1);
  if (*reinterpret_cast<const volatile int*>(info) != 0) return;
  // tile index -> (ti, tl), tl <= ti
  int t = blockIdx.x, ti = 0;
  while (t > ti) {
    t -= ti + 1;
    ++ti;
  }
  const int tl = t;
  const int base = k + nb;
  const int r0 = base + ti * kNB, c0 = base + tl * kNB;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kNB * nb; idx += 256) {
    const int r = idx / nb, j = idx % nb;
    Pi[j * (kNB + 1) + r] = r0 + r < n ? A[(size_t)(r0 + r) * lda + k + j] : 0.0;
    Pl[j * (kNB + 1) + r] = c0 + r < n ? A[(size_t)(c0 + r) * lda + k + j] : 0.0;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int j = 0; j < nb; ++j) {
    double ri[4], cl[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      ri[a] = Pi[j * (kNB + 1) + ty * 4 + a];
      cl[a] = Pl[j * (kNB + 1) + tx * 4 + a];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(ri[a], cl[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (r < n && c <= r) A[(size_t)r * lda + c] -= acc[a][b];
    }
  }
}

}  // namespace

cudaError_t launch_cholesky(double* A, int n, int lda, int* info, cudaStream_t s) {
  if (n < 1 || lda < n || !A || !info) return cudaErrorInvalidValue;
  const size_t trsm_smem = sizeof(double) * ((size_t)kNB * (kNB + 1) + (size_t)kNB * (kTrsmRows + 1));
  const size_t syrk_smem = sizeof(double) * 2 * (size_t)kNB * (kNB + 1);
  cudaError_t e = cudaFuncSetAttribute(chol_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)trsm_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_syrk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)syrk_smem);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < n; k += kNB) {
    const int nb = std::min(kNB, n - k);
    chol_diag_kernel<<<1, 256, 0, s>>>(A, lda, k, nb, info);
    const int rest = n - k - nb;
    if (rest > 0) {
      chol_trsm_kernel<<<(rest + kTrsmRows - 1) / kTrsmRows, kTrsmRows, trsm_smem, s>>>(
          A, lda, k, nb, n, info);
      const int nt = (rest + kNB - 1) / kNB;
      chol_syrk_kernel<<<nt * (nt + 1) / 2, 256, syrk_smem, s>>>(A, lda, k, nb, n, info);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ess
