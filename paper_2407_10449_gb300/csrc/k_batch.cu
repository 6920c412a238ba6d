// k_batch.cu -- kernels of the batched sampler: many independent polytopes of
// uneven d and m, each with its own chains, advanced together.
//
// Packed layout (chain-major): the chains of problem 0, then those of
// problem 1, ...; chain c's state row has d_p elements and its p, q rows m_p
// elements, at the offsets of its ChainDesc.  A_p (m_p x d_p, row-major) and
// b_p are packed the same way.  Per step:
//   batch_draw_kernel      nu ~ N(0, I_{d_p}) per chain (Alg. 1, "sample nu"),
//                          the same Philox counters as the one-problem path
//                          with the problem index in the counter;
//   batch_q_kernel         q = A_p nu for every chain: a grouped GEMM over work
//                          items (problem, 64 rows of A_p, <= 64 of its chains)
//                          taken from a global work queue by a persistent grid;
//   the chain-step kernels (k_chain_warp.cu, k_chain.cu) with per-chain views.
// Every refresh_k steps batch_refresh_kernel recomputes p = A_p x with
// FP64-class accuracy (Sec. 2.2: A x carried forward; the refresh bounds the
// drift): FP64 FMAs in the FP64 form, double-float sums on the FP32 pipe in
// the mixed form (a = hi + lo in float, hi x split exactly by an FMA, partial
// sums kept as error-free (s, c) pairs).
#include <algorithm>
#include <type_traits>

#include "ess_kernels.cuh"

namespace ess {
namespace {

constexpr int kBT = 64;      // rows of A and chains per work item
constexpr int kBK = 16;      // K chunk staged in shared memory
constexpr int kBThreads = 256;

// Takes the next work item for the whole CTA (uniform result).
__device__ __forceinline__ int next_item(int* queue, int* s_item) {
  __syncthreads();  // the previous item's shared-memory reads are done
  if (threadIdx.x == 0) *s_item = atomicAdd(queue, 1);
  __syncthreads();
  return *s_item;
}

template <typename T>
__global__ void batch_draw_kernel(const ChainDesc* __restrict__ desc, int n_chains,
                                  T* __restrict__ NU, uint64_t seed, uint32_t t,
                                  const unsigned* t_dev) {
  const int c = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= n_chains) return;
  const ChainDesc cd = desc[c];
  const uint32_t tt = t + (t_dev ? *t_dev : 0u);
  T* row = NU + cd.x_off;
  const int nblk = (cd.d + 3) >> 2;
  for (int n = lane; n < nblk; n += 32) {
    uint32_t r[4];
    rng_block(seed, (uint32_t)n, cd.chain, tt, cd.problem, 0u, r);
    T z[4];
    box_muller4(r, z);
    const int left = cd.d - 4 * n;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < left) row[4 * n + k] = z[k];
  }
}

// q[c, i] = a_i . nu_c in T (FP32 FMAs in the mixed form, FP64 in the FP64
// form).  Thread (ty, tx) of a 64 x 64 item owns chains ty + 16 i and rows
// tx + 16 j.
template <typename T>
__global__ void __launch_bounds__(kBThreads)
batch_q_kernel(const BatchItem* __restrict__ items, int n_items, int* queue,
               const T* __restrict__ A, const T* __restrict__ NU, T* __restrict__ Q) {
  __shared__ T As[kBK][kBT + 1];
  __shared__ T Xs[kBK][kBT + 1];
  __shared__ int s_item;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (;;) {
    const int it = next_item(queue, &s_item);
    if (it >= n_items) break;
    const BatchItem I = items[it];
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const T* Ab = A + I.a_off + (size_t)I.row0 * I.d;
    const T* Xb = NU + I.x_off;
    for (int k0 = 0; k0 < I.d; k0 += kBK) {
#pragma unroll
      for (int e = 0; e < kBT * kBK / kBThreads; ++e) {
        const int idx = tid + e * kBThreads;
        const int r = idx / kBK, kk = idx % kBK, gk = k0 + kk;
        As[kk][r] = (r < I.rows && gk < I.d) ? Ab[(size_t)r * I.d + gk] : T(0);
        Xs[kk][r] = (r < I.chains && gk < I.d) ? Xb[(size_t)r * I.d + gk] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kBK; ++kk) {
        T xv[4], av[4];
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
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ci = ty + 16 * i;
      if (ci >= I.chains) continue;
      T* qrow = Q + I.p_off + (size_t)ci * I.m + I.row0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int rj = tx + 16 * j;
        if (rj < I.rows) qrow[rj] = acc[i][j];
      }
    }
  }
}

// Error-free sum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// p[c, i] = a_i . x_c with FP64-class accuracy.  T = double: FP64 FMAs.
// T = float: a_i = hi + lo (floats), hi x exactly as (prod, fma error), the
// running sum as an error-free (s, c) pair; the result (s + c) has relative
// error ~2^-44 of sum |a||x|.  Writes P (rounded to T) and, if P64 is set, the
// double value; with drift set, folds max |P_new - P_old| / ||a_i|| into it.
template <typename T>
__global__ void __launch_bounds__(kBThreads)
batch_refresh_kernel(const BatchItem* __restrict__ items, int n_items, int* queue,
                     const double* __restrict__ A64, const T* __restrict__ X, T* P, double* P64,
                     const double* __restrict__ anorm, unsigned long long* drift_bits) {
  constexpr bool kDF = sizeof(T) == 4;
  using S = typename std::conditional<kDF, float, double>::type;
  __shared__ S Ah[kBK][kBT + 1];
  __shared__ S Al[kDF ? kBK : 1][kBT + 1];
  __shared__ T Xs[kBK][kBT + 1];
  __shared__ int s_item;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double drift = 0.0;
  for (;;) {
    const int it = next_item(queue, &s_item);
    if (it >= n_items) break;
    const BatchItem I = items[it];
    S hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        hi[i][j] = S(0);
        lo[i][j] = S(0);
      }
    const double* Ab = A64 + I.a_off + (size_t)I.row0 * I.d;
    const T* Xb = X + I.x_off;
    for (int k0 = 0; k0 < I.d; k0 += kBK) {
#pragma unroll
      for (int e = 0; e < kBT * kBK / kBThreads; ++e) {
        const int idx = tid + e * kBThreads;
        const int r = idx / kBK, kk = idx % kBK, gk = k0 + kk;
        const double a = (r < I.rows && gk < I.d) ? Ab[(size_t)r * I.d + gk] : 0.0;
        if constexpr (kDF) {
          const float h = __double2float_rn(a);
          Ah[kk][r] = h;
          Al[kk][r] = __double2float_rn(a - (double)h);
        } else {
          Ah[kk][r] = a;
        }
        Xs[kk][r] = (r < I.chains && gk < I.d) ? Xb[(size_t)r * I.d + gk] : T(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < kBK; ++kk) {
        T xv[4];
        S ah[4], al[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[i] = Xs[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ah[j] = Ah[kk][tx + 16 * j];
          al[j] = kDF ? Al[kk][tx + 16 * j] : S(0);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if constexpr (kDF) {
              const float pr = ah[j] * xv[i];
              const float pe = fmaf(ah[j], xv[i], -pr);  // hi x = pr + pe exactly
              float s, e;
              two_sum_f(hi[i][j], pr, s, e);
              hi[i][j] = s;
              lo[i][j] += e + pe + al[j] * xv[i];
            } else {
              hi[i][j] = fma(ah[j], (double)xv[i], hi[i][j]);
            }
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ci = ty + 16 * i;
      if (ci >= I.chains) continue;
      const size_t base = I.p_off + (size_t)ci * I.m + I.row0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int rj = tx + 16 * j;
        if (rj >= I.rows) continue;
        const double v = (double)hi[i][j] + (double)lo[i][j];
        if (P64) P64[base + rj] = v;
        if (P) {
          const T pn = (T)v;
          if (drift_bits) {
            const double old = (double)P[base + rj];
            drift = fmax(drift, fabs((double)pn - old) / anorm[I.b_off + I.row0 + rj]);
          }
          P[base + rj] = pn;
        }
      }
    }
  }
  if (drift_bits) atomic_max_nonneg(drift_bits, drift);
}

// status |= kStatusInfeasible where the FP64-class product exceeds b.
__global__ void batch_check_kernel(const ChainDesc* __restrict__ desc, int n_chains,
                                   const double* __restrict__ P64, const double* __restrict__ b64,
                                   int* status) {
  const int c = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= n_chains) return;
  const ChainDesc cd = desc[c];
  bool bad = false;
  for (int i = lane; i < cd.m; i += 32) bad |= !(P64[cd.p_off + i] <= b64[cd.b_off + i]);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStatusInfeasible);
}

__global__ void advance_t_kernel(unsigned* t_dev, unsigned by) { *t_dev += by; }

inline unsigned warps_grid(int n) { return (unsigned)(((size_t)n * 32 + 255) / 256); }

int persistent_grid(int n_items) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return std::max(1, std::min(n_items, sms * 6));
}

}  // namespace

template <typename T>
cudaError_t launch_batch_draw(const ChainDesc* desc, int n_chains, T* NU, uint64_t seed,
                              uint32_t t, const unsigned* t_dev, cudaStream_t s) {
  if (n_chains <= 0) return cudaSuccess;
  batch_draw_kernel<T><<<warps_grid(n_chains), 256, 0, s>>>(desc, n_chains, NU, seed, t, t_dev);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_q(const BatchItem* items, int n_items, int* queue, const T* A,
                           const T* NU, T* Q, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_q_kernel<T><<<persistent_grid(n_items), kBThreads, 0, s>>>(items, n_items, queue, A, NU, Q);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_refresh(const BatchItem* items, int n_items, int* queue,
                                 const double* A64, const T* X, T* P, double* P64,
                                 const double* anorm, unsigned long long* drift_bits,
                                 cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_refresh_kernel<T><<<persistent_grid(n_items), kBThreads, 0, s>>>(
      items, n_items, queue, A64, X, P, P64, anorm, drift_bits);
  return cudaGetLastError();
}

cudaError_t launch_batch_check(const ChainDesc* desc, int n_chains, const double* P64,
                               const double* b64, int* status, cudaStream_t s) {
  if (n_chains <= 0) return cudaSuccess;
  batch_check_kernel<<<warps_grid(n_chains), 256, 0, s>>>(desc, n_chains, P64, b64, status);
  return cudaGetLastError();
}

cudaError_t launch_advance_t(unsigned* t_dev, unsigned by, cudaStream_t s) {
  advance_t_kernel<<<1, 1, 0, s>>>(t_dev, by);
  return cudaGetLastError();
}

template cudaError_t launch_batch_draw<float>(const ChainDesc*, int, float*, uint64_t, uint32_t,
                                              const unsigned*, cudaStream_t);
template cudaError_t launch_batch_draw<double>(const ChainDesc*, int, double*, uint64_t, uint32_t,
                                               const unsigned*, cudaStream_t);
template cudaError_t launch_batch_q<float>(const BatchItem*, int, int*, const float*, const float*,
                                           float*, cudaStream_t);
template cudaError_t launch_batch_q<double>(const BatchItem*, int, int*, const double*,
                                            const double*, double*, cudaStream_t);
template cudaError_t launch_batch_refresh<float>(const BatchItem*, int, int*, const double*,
                                                 const float*, float*, double*, const double*,
                                                 unsigned long long*, cudaStream_t);
template cudaError_t launch_batch_refresh<double>(const BatchItem*, int, int*, const double*,
                                                  const double*, double*, double*, const double*,
                                                  unsigned long long*, cudaStream_t);

}  // namespace ess
