// ess_whiten.cu -- the App. A map x = L u + mu on the GPU (ess_whitener_*).
//
// A run in whitened coordinates samples u under (A L) u <= b - A mu; the
// samples of the truncation of N(mu, L L^T) by A x <= b are x = L u + mu.  For
// many recorded samples this is one GEMM X = U L^T plus a broadcast add:
//   float U  (the mixed form's samples): the scaled FP16x3 tensor-core GEMM of
//            q = A nu (tc_gemm_q) with L in the role of A, then + mu in FP32;
//   double U (the FP64 form's samples): the FP64 FMA GEMM, then + mu in FP64.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ess.h"
#include "ess_gemm_tc.cuh"
#include "ess_kernels.cuh"

void ess_internal_set_error(const std::string& msg);  // ess_abi.cu

struct ess_whitener {
  int d = 0;
  int device = 0;
  double* L64 = nullptr;            // d x d row-major (device)
  double* mu64 = nullptr;           // d or nullptr
  float* mu32 = nullptr;
  ess::TcGemmPlan* plan = nullptr;  // fp16 splits of L for the float path
  int ld16 = 0;
  int cap = 0;                      // rows the split buffers hold
  __half* h[2] = {nullptr, nullptr};
  float* unscale = nullptr;
  int* status = nullptr;
};

namespace {

ess_status wfail(ess_status st, const std::string& msg) {
  ess_internal_set_error(msg);
  return st;
}

ess_status wcuda(cudaError_t e, const char* what) {
  return wfail(e == cudaErrorMemoryAllocation ? ESS_ERR_OOM : ESS_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define WESS_CUDA(expr)                              \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return wcuda(e_, #expr);  \
  } while (0)

template <typename T>
__global__ void add_rows_kernel(T* X, int n, int d, const T* __restrict__ mu) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n * d) return;
  X[gid] += mu[gid % d];
}

template <typename T>
cudaError_t add_rows(T* X, int n, int d, const T* mu, cudaStream_t s) {
  const long long total = (long long)n * d;
  if (total == 0 || !mu) return cudaSuccess;
  add_rows_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, n, d, mu);
  return cudaGetLastError();
}

void free_splits(ess_whitener* w) {
  for (auto& p : w->h)
    if (p) cudaFree(p), p = nullptr;
  if (w->unscale) cudaFree(w->unscale), w->unscale = nullptr;
  w->cap = 0;
}

}  // namespace

extern "C" {

ess_status ess_whitener_create(const double* L, const double* mu, int d, ess_whitener** out) {
  ess_internal_set_error("");
  if (!out) return wfail(ESS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!L || d < 1) return wfail(ESS_ERR_ARG, "need L and d >= 1");
  for (long long i = 0; i < (long long)d * d; ++i)
    if (!std::isfinite(L[i])) return wfail(ESS_ERR_ARG, "L has a non-finite entry");
  if (mu)
    for (int i = 0; i < d; ++i)
      if (!std::isfinite(mu[i])) return wfail(ESS_ERR_ARG, "mu has a non-finite entry");
  ess_whitener* w = new ess_whitener();
  w->d = d;
  cudaGetDevice(&w->device);
  w->ld16 = (d + 7) & ~7;
  cudaError_t e = cudaMalloc(&w->L64, sizeof(double) * (size_t)d * d);
  if (e == cudaSuccess) e = cudaMemcpy(w->L64, L, sizeof(double) * (size_t)d * d, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && mu) {
    std::vector<float> m32(mu, mu + d);
    e = cudaMalloc(&w->mu64, sizeof(double) * d);
    if (e == cudaSuccess) e = cudaMemcpy(w->mu64, mu, sizeof(double) * d, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&w->mu32, sizeof(float) * d);
    if (e == cudaSuccess) e = cudaMemcpy(w->mu32, m32.data(), sizeof(float) * d, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&w->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(w->status, 0, sizeof(int));
  if (e == cudaSuccess) e = ess::tc_gemm_create(&w->plan, L, d, d);
  if (e != cudaSuccess) {
    ess_whitener_destroy(w);
    return wcuda(e, "ess_whitener_create");
  }
  *out = w;
  return ESS_OK;
}

void ess_whitener_destroy(ess_whitener* w) {
  if (!w) return;
  free_splits(w);
  if (w->L64) cudaFree(w->L64);
  if (w->mu64) cudaFree(w->mu64);
  if (w->mu32) cudaFree(w->mu32);
  if (w->status) cudaFree(w->status);
  ess::tc_gemm_destroy(w->plan);
  delete w;
}

ess_status ess_whitener_apply(ess_whitener* w, const void* U, int u_double, int n, void* X,
                              void* cuda_stream) {
  ess_internal_set_error("");
  if (!w) return wfail(ESS_ERR_ARG, "whitener is NULL");
  if (n < 0) return wfail(ESS_ERR_ARG, "negative size");
  if (n == 0) return ESS_OK;
  if (!U || !X) return wfail(ESS_ERR_ARG, "NULL buffer");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int d = w->d;
  if (u_double) {
    WESS_CUDA((ess::launch_gemm_nt_f64<double, double>(static_cast<const double*>(U), d, w->L64,
                                                        d, static_cast<double*>(X), d, n, d, d,
                                                        nullptr, nullptr, st)));
    WESS_CUDA(add_rows<double>(static_cast<double*>(X), n, d, w->mu64, st));
  } else {
    if (n > w->cap) {
      free_splits(w);
      for (auto& p : w->h) {
        WESS_CUDA(cudaMalloc(&p, sizeof(__half) * (size_t)n * w->ld16));
        // the padding columns d .. ld16 - 1 stay zero
        WESS_CUDA(cudaMemset(p, 0, sizeof(__half) * (size_t)n * w->ld16));
      }
      WESS_CUDA(cudaMalloc(&w->unscale, sizeof(float) * n));
      w->cap = n;
    }
    WESS_CUDA(ess::tc_split2_rows(static_cast<const float*>(U), d, n, d, w->h[0], w->h[1],
                                  w->ld16, w->unscale, st));
    WESS_CUDA(ess::tc_gemm_q(w->plan, w->h, w->unscale, w->ld16, n, static_cast<float*>(X), d,
                             w->status, st));
    WESS_CUDA(add_rows<float>(static_cast<float*>(X), n, d, w->mu32, st));
  }
  int h = 0;
  WESS_CUDA(cudaMemcpyAsync(&h, w->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  WESS_CUDA(cudaStreamSynchronize(st));
  if (h & ess::kStatusTimeout) return wfail(ESS_ERR_TIMEOUT, "a bounded device wait gave up");
  return ESS_OK;
}

}  // extern "C"
