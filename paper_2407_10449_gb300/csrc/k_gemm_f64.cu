// k_gemm_f64.cu -- C = X A^T in FP64 fused multiply-adds.
//
// Used for q = A nu in the plain FP64 form and for the A x refresh (the
// cached products of Sec. 2.2 "computed anyway").  X is M x K (chains x d),
// A is N x K (constraints x d), both with K contiguous; C is M x N (chain
// rows, constraint columns), i.e. the layout the chain-step kernel reads.
// FP64 throughput on GB300 is ~1.2 TFLOP/s, so a register-tiled DFMA kernel
// with shared-memory staging already runs at the FP64 pipe's limit.
#include "ess_kernels.cuh"

namespace ess {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NTHR = 256;

template <typename TX, typename TOut>
__global__ void __launch_bounds__(NTHR)
gemm_nt_f64_kernel(const TX* __restrict__ X, int ldx, const double* __restrict__ A, int lda,
                   TOut* C, int ldc, int M, int N, int K, const double* __restrict__ anorm,
                   DevStats* drift_stats) {
  __shared__ double Xs[BK][BM + 1];
  __shared__ double As[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e = 0; e < (BM * BK) / NTHR; ++e) {
      const int idx = tid + e * NTHR;
      const int row = idx / BK, kk = idx % BK;
      const int gm = m0 + row, gk = k0 + kk;
      Xs[kk][row] = (gm < M && gk < K) ? (double)X[(size_t)gm * ldx + gk] : 0.0;
      const int gn = n0 + row;
      As[kk][row] = (gn < N && gk < K) ? A[(size_t)gn * lda + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double xv[4], av[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = Xs[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) av[j] = As[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(xv[i], av[j], acc[i][j]);
    }
    __syncthreads();
  }

  double drift = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      TOut* dst = C + (size_t)gm * ldc + gn;
      if (drift_stats != nullptr) {
        const double old = (double)*dst;
        const double diff = fabs(acc[i][j] - old) / (anorm[gn] > 0.0 ? anorm[gn] : 1.0);
        drift = fmax(drift, diff);
      }
      *dst = (TOut)acc[i][j];
    }
  }
  if (drift_stats != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) drift = fmax(drift, __shfl_xor_sync(0xffffffffu, drift, o));
    if ((tid & 31) == 0) atomic_max_nonneg(&drift_stats->max_drift_bits, drift);
  }
}

}  // namespace

template <typename TX, typename TOut>
cudaError_t launch_gemm_nt_f64(const TX* X, int ldx, const double* A, int lda, TOut* C, int ldc,
                               int M, int N, int K, const double* anorm, DevStats* drift_stats,
                               cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  gemm_nt_f64_kernel<TX, TOut><<<grid, NTHR, 0, s>>>(X, ldx, A, lda, C, ldc, M, N, K, anorm,
                                                     drift_stats);
  return cudaGetLastError();
}

template cudaError_t launch_gemm_nt_f64<double, double>(const double*, int, const double*, int,
                                                        double*, int, int, int, int,
                                                        const double*, DevStats*, cudaStream_t);
template cudaError_t launch_gemm_nt_f64<float, float>(const float*, int, const double*, int,
                                                      float*, int, int, int, int, const double*,
                                                      DevStats*, cudaStream_t);
template cudaError_t launch_gemm_nt_f64<float, double>(const float*, int, const double*, int,
                                                       double*, int, int, int, int,
                                                       const double*, DevStats*, cudaStream_t);

}  // namespace ess
