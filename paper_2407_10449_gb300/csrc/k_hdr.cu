// k_hdr.cu -- the level steps of the normal-probability estimator (the
// Holmes-Diaconis-Ross splitting estimator with subset-simulation shifts,
// driven by the chain steps; the method the paper cites for Z = P(A x <= b)):
//   * level values g_j = max_i (P[j, i] - b_i) of the samples, P = A x in FP64
//     (x lies in the shifted domain {A x <= b + gamma} exactly when g <= gamma);
//   * one CTA: the k-th and (k + 1)-th smallest g by a radix select over the
//     order-preserving 64-bit keys of the doubles, the shift gamma (their
//     midpoint, 0 once the k-th is <= 0, or a given shift), and the stable
//     list of the samples with g <= gamma;
//   * the next level's start states: sample j takes the (j mod count)-th
//     listed state;
//   * the shifted bounds b + gamma, their float rounding and the residual
//     recheck thresholds b + gamma - margin ||a_i||, from saved originals.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "chain_block_ops.cuh"
#include "ess_kernels.cuh"

namespace ess {
namespace {

using blockops::OpAdd;
using blockops::block_exclusive_scan;

constexpr int kSelT = 1024;  // threads of the select kernel

__global__ void hdr_level_kernel(const double* __restrict__ P, int ldp,
                                 const double* __restrict__ b, int n, int m,
                                 double* __restrict__ g) {
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = P + (size_t)warp * ldp;
  double mx = -INFINITY;
  for (int i = lane; i < m; i += 32) mx = fmax(mx, __dsub_rn(row[i], b[i]));
  // a NaN product makes the sample fall in no level
  bool nan = false;
  for (int i = lane; i < m; i += 32) nan |= isnan(row[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nan |= __shfl_xor_sync(0xffffffffu, (int)nan, o) != 0;
  }
  if (lane == 0) g[warp] = nan ? (double)NAN : mx;
}

// Order-preserving map of doubles to unsigned keys (NaN above +inf).
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)u);
}

// One CTA.  shift_in: NaN for the adaptive shift, else the level's fixed
// shift.  Writes out[0] = gamma, ((int*)(out + 1))[0] = count, list[0 ..
// count) = the samples with g <= gamma in index order.
__global__ void __launch_bounds__(kSelT) hdr_select_kernel(const double* __restrict__ g, int n,
                                                           int k, double shift_in,
                                                           double* __restrict__ out,
                                                           int* __restrict__ count_out,
                                                           int* __restrict__ list) {
  __shared__ unsigned hist[256];
  __shared__ unsigned long long s_prefix, s_mask;
  __shared__ unsigned s_rank;
  __shared__ unsigned long long s_next;
  __shared__ unsigned s_le;
  __shared__ int s_itmp[kSelT / 32];
  __shared__ double s_gamma;
  const int tid = threadIdx.x;
  double gamma = shift_in;
  if (isnan(shift_in)) {
    // ---- radix select of the k-th smallest key, 8 bits at a time ----------
    if (tid == 0) {
      s_prefix = 0ull;
      s_mask = 0ull;
      s_rank = (unsigned)k;
    }
    for (int pass = 0; pass < 8; ++pass) {
      const int shift = 56 - 8 * pass;
      for (int i = tid; i < 256; i += kSelT) hist[i] = 0u;
      __syncthreads();
      const unsigned long long prefix = s_prefix, mask = s_mask;
      for (int j = tid; j < n; j += kSelT) {
        const unsigned long long key = dkey(g[j]);
        if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 0xFFu], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        unsigned rank = s_rank, cum = 0u;
        int digit = 255;
        for (int dgt = 0; dgt < 256; ++dgt) {
          if (cum + hist[dgt] >= rank) {
            digit = dgt;
            break;
          }
          cum += hist[dgt];
        }
        s_rank = rank - cum;
        s_prefix = prefix | ((unsigned long long)digit << shift);
        s_mask = mask | (0xFFull << shift);
      }
      __syncthreads();
    }
    // ---- the (k + 1)-th smallest: the same key if it repeats, else the
    // smallest key above it -------------------------------------------------
    const unsigned long long kth = s_prefix;
    if (tid == 0) {
      s_next = ~0ull;
      s_le = 0u;
    }
    __syncthreads();
    unsigned le = 0u;
    unsigned long long nxt = ~0ull;
    for (int j = tid; j < n; j += kSelT) {
      const unsigned long long key = dkey(g[j]);
      le += key <= kth ? 1u : 0u;
      if (key > kth && key < nxt) nxt = key;
    }
    atomicAdd(&s_le, le);
    atomicMin(&s_next, nxt);
    __syncthreads();
    const double gk = dkey_inv(kth);
    const double gk1 = s_le >= (unsigned)k + 1u ? gk : dkey_inv(s_next);
    gamma = gk <= 0.0 ? 0.0 : gk + (gk1 - gk) * 0.5;
  }
  if (tid == 0) s_gamma = gamma;
  __syncthreads();
  gamma = s_gamma;
  // ---- stable list of the samples inside ----------------------------------
  int total = 0;
  for (int base = 0; base < n; base += kSelT) {
    const int j = base + tid;
    const int in = j < n && g[j] <= gamma ? 1 : 0;
    int chunk;
    const int at = block_exclusive_scan<kSelT>(in, 0, OpAdd(), s_itmp, chunk);
    if (in) list[total + at] = j;
    total += chunk;
  }
  if (tid == 0) {
    out[0] = gamma;
    *count_out = total;
  }
}

template <typename T>
__global__ void hdr_gather_kernel(const T* __restrict__ src, int ld, const int* __restrict__ list,
                                  const int* __restrict__ count, int n, int d, T* __restrict__ dst) {
  const int cnt = *count;
  if (cnt <= 0) return;
  const size_t total = (size_t)n * d;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / d), c = (int)(e % d);
    dst[(size_t)j * ld + c] = src[(size_t)list[j % cnt] * ld + c];
  }
}

template <typename TS>
__global__ void hdr_shift_kernel(const double* __restrict__ b0, const double* __restrict__ anorm,
                                 int m, double gamma, double margin, double* __restrict__ b64,
                                 float* __restrict__ b32, TS* __restrict__ slack) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double bi = __dadd_rn(b0[i], gamma);
    b64[i] = bi;
    if (b32) b32[i] = __double2float_rn(bi);
    const double v = __dsub_rn(bi, __dmul_rn(margin, anorm[i]));
    if constexpr (sizeof(TS) == 4) slack[i] = __double2float_rd(v);  // rounded down
    else slack[i] = v;
  }
}

}  // namespace

cudaError_t launch_hdr_level(const double* P, int ldp, const double* b, int n, int m, double* g,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)(((size_t)n * 32 + threads - 1) / threads);
  hdr_level_kernel<<<blocks, threads, 0, s>>>(P, ldp, b, n, m, g);
  return cudaGetLastError();
}

cudaError_t launch_hdr_select(const double* g, int n, int k, double shift, double* gamma_out,
                              int* count_out, int* list, cudaStream_t s) {
  if (n < 1 || k < 1 || k > n - 1) return cudaErrorInvalidValue;
  hdr_select_kernel<<<1, kSelT, 0, s>>>(g, n, k, shift, gamma_out, count_out, list);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hdr_gather(const T* src, int ld, const int* list, const int* count, int n,
                              int d, T* dst, cudaStream_t s) {
  const size_t total = (size_t)n * d;
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 4096);
  hdr_gather_kernel<T><<<blocks, 256, 0, s>>>(src, ld, list, count, n, d, dst);
  return cudaGetLastError();
}

cudaError_t launch_hdr_shift(const double* b0, const double* anorm, int m, double gamma,
                             double margin, double* b64, float* b32, void* slack,
                             bool float_slack, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min(1024, (m + 255) / 256);
  if (float_slack)
    hdr_shift_kernel<float><<<blocks, 256, 0, s>>>(b0, anorm, m, gamma, margin, b64, b32,
                                                   static_cast<float*>(slack));
  else
    hdr_shift_kernel<double><<<blocks, 256, 0, s>>>(b0, anorm, m, gamma, margin, b64, b32,
                                                    static_cast<double*>(slack));
  return cudaGetLastError();
}

template cudaError_t launch_hdr_gather<float>(const float*, int, const int*, const int*, int, int,
                                              float*, cudaStream_t);
template cudaError_t launch_hdr_gather<double>(const double*, int, const int*, const int*, int,
                                               int, double*, cudaStream_t);

}  // namespace ess
