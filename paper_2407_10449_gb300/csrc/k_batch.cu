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
//   batch_gemm_kernel      q = A_p nu for every chain: a grouped GEMM over work
//                          items (problem, a tile of A_p's rows, a tile of its
//                          chains) taken from a global work queue by a
//                          persistent grid;
//   the chain-step kernels (k_chain_warp.cu, k_chain.cu) with per-chain views.
// Every refresh_k steps the same kernel recomputes p = A_p x with
// FP64-class accuracy (Sec. 2.2: A x carried forward; the refresh bounds the
// drift): FP64 FMAs in the FP64 form, double-float sums on the FP32 pipe in
// the mixed form (a = hi + lo in float, hi x split exactly by an FMA, partial
// sums kept as error-free (s, c) pairs).
#include <algorithm>
#include <type_traits>

#include "ess_kernels.cuh"

namespace ess {
namespace {

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
                                  const unsigned* t_dev, const double* __restrict__ bm_tab,
                                  __half* __restrict__ H0, __half* __restrict__ H1) {
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
    if constexpr (sizeof(T) == 8)
      box_muller4(r, z, bm_tab);
    else
      box_muller4(r, z);
    const int left = cd.d - 4 * n;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < left) row[4 * n + k] = z[k];
    if (sizeof(T) == 4 && H0) {
      // two-way fp16 split of nu * 2^12 (see ess_common.cuh)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= left) break;
        const float y = (float)z[k] * kNuSplitScale;
        const __half a = __float2half_rn(y);
        H0[cd.h_off + 4 * n + k] = a;
        H1[cd.h_off + 4 * n + k] = __float2half_rn(y - __half2float(a));
      }
    }
  }
}

// Per-chain scaled fp16 split of caller-supplied nu (warp per chain).
__global__ void batch_split_kernel(const ChainDesc* __restrict__ desc, int n_chains,
                                   const float* __restrict__ NU, __half* __restrict__ H0,
                                   __half* __restrict__ H1, float* __restrict__ unscale) {
  const int c = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= n_chains) return;
  const ChainDesc cd = desc[c];
  const float* v = NU + cd.x_off;
  float mx = 0.f;
  for (int j = lane; j < cd.d; j += 32) mx = fmaxf(mx, fabsf(v[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int e = 0;
  if (mx > 0.f) (void)frexpf(mx, &e);
  const float tsc = mx > 0.f ? ldexpf(1.f, 15 - e) : 1.f;
  if (lane == 0) unscale[c] = mx > 0.f ? ldexpf(1.f, e - 15) : 0.f;
  for (int j = lane; j < cd.d; j += 32) {
    const float y = v[j] * tsc;
    const __half a = __float2half_rn(y);
    H0[cd.h_off + j] = a;
    H1[cd.h_off + j] = __float2half_rn(y - __half2float(a));
  }
}

// Error-free sum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <typename V> struct Vec4;
template <> struct Vec4<float> {
  __device__ static void load(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
};
template <> struct Vec4<double> {
  __device__ static void load(const double* p, double (&v)[4]) {
    const double2 t0 = reinterpret_cast<const double2*>(p)[0];
    const double2 t1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
  }
};

inline unsigned warps_grid(int n) { return (unsigned)(((size_t)n * 32 + 255) / 256); }

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// A persistent grid: as many CTAs as fit on the GPU at once (per_sm each), at
// most one per work item.
int persistent_grid(int n_items, int per_sm = 6) {
  return std::max(1, std::min(n_items, num_sms() * std::max(1, per_sm)));
}

// CTAs of kernel k (threads, dynamic shared memory smem) resident per SM.
template <typename K>
int resident_per_sm(K k, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) n = 1;
  return std::max(1, n);
}

enum { kGemmQ = 0, kGemmRefresh = 1 };

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Asynchronous global -> shared copy of one element (4 or 8 bytes); copies
// zeros when ok is false (no bytes are read then).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_addr(dst)), "l"(src),
               "n"(BYTES), "r"(ok ? BYTES : 0)
               : "memory");
}
// 16 bytes (both addresses 16-byte aligned), zeros when ok is false.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_one() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// Staged tile sizes (elements): A chunk 16 x (256 + 4), X chunk 16 x (64 + 4);
// rows padded to 16-byte multiples for the 128-bit shared loads.
constexpr int kAS = 256 + 4;
constexpr int kXS = 64 + 4;

template <typename TA, typename TX, bool kDF>
constexpr size_t gemm_smem_bytes() {
  return 2 * ((kDF ? 2 : 1) * sizeof(TA) * kBK * kAS + sizeof(TX) * kBK * kXS);
}

// One grouped-GEMM launch over work items taken from a device queue.  An item
// is rows row0 .. row0 + rows - 1 of one problem's A times `chains` of its
// chains, tile shape rtile x ctile (256 x 16, 128 x 32 or 64 x 64, chosen per
// problem from its chain count).  Thread (tx, ty) owns rows 4 tx .. 4 tx + 3
// and chains 4 ty .. 4 ty + 3 (4 x 4 register tile, 128-bit shared loads);
// a warp covers an 8 x 4 block of such threads.
// K is staged 16 columns at a time by cp.async into two shared-memory
// buffers, the next chunk's copies in flight while the current one is used.
//   kGemmQ:       out[c, i] = a_i . nu_c in T (FP32 or FP64 FMAs); A is read
//                 from its K-major copy (16-byte copies of consecutive rows).
//   kGemmRefresh: p[c, i] = a_i . x_c with FP64-class accuracy:
//                 T = double: FP64 FMAs on A64; T = float: A64 = hi + lo with
//                 hi = Aq (A rounded to float) and lo = Alo (float), hi x
//                 exactly as (product, FMA error), sums as error-free (s, c)
//                 pairs (relative error ~2^-44 of sum |a||x|).  Also writes
//                 P64 and folds max |P_new - P_old| / ||a_i|| into drift_bits.
template <typename T, int MODE>
__global__ void __launch_bounds__(kBThreads)
batch_gemm_kernel(const BatchItem* __restrict__ items, int n_items, int* queue,
                  const T* __restrict__ Aq, const double* __restrict__ A64,
                  const float* __restrict__ Alo, const T* __restrict__ X, T* out, double* P64,
                  const double* __restrict__ anorm, unsigned long long* drift_bits) {
  constexpr bool kDF = MODE == kGemmRefresh && sizeof(T) == 4;  // double-float sums
  // staged A type: T for q and the double-float refresh, double otherwise
  using TA = typename std::conditional<MODE == kGemmQ || kDF, T, double>::type;
  constexpr int kASlices = kDF ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TA* As = reinterpret_cast<TA*>(smem_raw);  // [2][kASlices][kBK][kAS]
  T* Xs = reinterpret_cast<T*>(smem_raw + 2 * kASlices * sizeof(TA) * kBK * kAS);  // [2][kBK][kXS]
  __shared__ int s_item;
  const int tid = threadIdx.x;
  const TA* Asrc = MODE == kGemmQ || kDF ? reinterpret_cast<const TA*>(Aq)
                                         : reinterpret_cast<const TA*>(A64);
  const TA* Alsrc = reinterpret_cast<const TA*>(Alo);
  double drift = 0.0;
  float driftf = 0.f;
  for (;;) {
    const int it = next_item(queue, &s_item);
    if (it >= n_items) break;
    const BatchItem I = items[it];
    // warp w covers 8 row quads x 4 chain quads (lane & 7, lane >> 3), so a
    // k step reads 128 bytes of A and 64 bytes of X per warp from shared memory
    const int wpr = I.rtile >> 5;  // warps across the row quads (rtile / 4 / 8)
    const int warp = tid >> 5, lane = tid & 31;
    const int tx = (warp % wpr) * 8 + (lane & 7);
    const int ty = (warp / wpr) * 4 + (lane >> 3);
    // a warp whose 32 rows or 16 chains all lie past the item's edge stores
    // nothing: it skips the arithmetic (the FP32 and FP64 pipes charge a warp
    // instruction whatever its lanes hold) but still stages and syncs
    const bool warp_live = (warp % wpr) * 32 < I.rows && (warp / wpr) * 16 < I.chains;
    T hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        hi[i][j] = T(0);
        lo[i][j] = T(0);
      }
    const TA* Ab = MODE == kGemmQ ? Asrc + I.at_off : Asrc + I.a_off + (size_t)I.row0 * I.d;
    const TA* Alb = kDF ? Alsrc + I.a_off + (size_t)I.row0 * I.d : nullptr;
    const T* Xb = X + I.x_off;
    const int nchunk = (I.d + kBK - 1) / kBK;
    // chunk c of A and X into buffer c & 1 (zero fill outside the item);
    // consecutive threads read consecutive k of one row
    auto stage = [&](int c) {
      const int k0 = c * kBK;
      TA* as = As + (c & 1) * kASlices * kBK * kAS;
      T* xs = Xs + (c & 1) * kBK * kXS;
      if constexpr (MODE == kGemmQ) {
        // K-major A: 16-byte copies of V consecutive rows (zero padding up to mpad)
        constexpr int V = 16 / sizeof(TA);
        const int lg = 31 - __clz(I.rtile / V);  // vectors per k-row: a power of two
        for (int idx = tid; idx < (kBK << lg); idx += kBThreads) {
          const int kk = idx >> lg, r = V * (idx & ((1 << lg) - 1)), gk = k0 + kk;
          const bool ok = gk < I.d && I.row0 + r < I.mpad;
          cp_async16(&as[kk * kAS + r], ok ? Ab + (size_t)gk * I.mpad + I.row0 + r : Ab, ok);
        }
      } else {
        for (int idx = tid; idx < I.rtile * kBK; idx += kBThreads) {
          const int r = idx >> 4, kk = idx & 15, gk = k0 + kk;
          const bool ok = r < I.rows && gk < I.d;
          const size_t o = ok ? (size_t)r * I.d + gk : 0;
          cp_async_elem<sizeof(TA)>(&as[kk * kAS + r], Ab + o, ok);
          if constexpr (kDF) cp_async_elem<sizeof(TA)>(&as[(kBK + kk) * kAS + r], Alb + o, ok);
        }
      }
      for (int idx = tid; idx < I.ctile * kBK; idx += kBThreads) {
        const int r = idx >> 4, kk = idx & 15, gk = k0 + kk;
        const bool ok = r < I.chains && gk < I.d;
        cp_async_elem<sizeof(T)>(&xs[kk * kXS + r], ok ? Xb + (size_t)r * I.d + gk : Xb, ok);
      }
    };
    stage(0);
    cp_async_commit();
    for (int c = 0; c < nchunk; ++c) {
      if (c + 1 < nchunk) stage(c + 1);
      cp_async_commit();
      cp_async_wait_one();  // chunk c has landed (this thread's copies)
      __syncthreads();      // ... and every thread's
      const TA* as = As + (c & 1) * kASlices * kBK * kAS;
      const T* xs = Xs + (c & 1) * kBK * kXS;
      const int kn = min(kBK, I.d - c * kBK);
      auto kstep = [&](int kk) {
        T xv[4];
        TA av[4];
        Vec4<T>::load(xs + kk * kXS + 4 * ty, xv);
        Vec4<TA>::load(as + kk * kAS + 4 * tx, av);
        if constexpr (kDF) {
          TA alv[4];
          Vec4<TA>::load(as + (kBK + kk) * kAS + 4 * tx, alv);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float pr = av[j] * xv[i];
              const float pe = fmaf(av[j], xv[i], -pr);  // hi x = pr + pe exactly
              float sum, e;
              two_sum_f(hi[i][j], pr, sum, e);
              hi[i][j] = sum;
              lo[i][j] += e + pe + alv[j] * xv[i];
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) hi[i][j] = fma(xv[i], (T)av[j], hi[i][j]);
        }
      };
      if (!warp_live) {
      } else if (kn == kBK) {
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) kstep(kk);
      } else {
        for (int kk = 0; kk < kn; ++kk) kstep(kk);
      }
      __syncthreads();  // buffer c & 1 is free for chunk c + 2
    }
    // refresh with drift: every old value is loaded before the first store,
    // so the loads are in flight together
    T old[4][4];
    if constexpr (MODE != kGemmQ) {
      if (out && drift_bits) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int ci = 4 * ty + i;
          const size_t base = (size_t)I.p_off + (size_t)ci * I.m + I.row0;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int rj = 4 * tx + j;
            old[i][j] = ci < I.chains && rj < I.rows ? out[base + rj] : T(0);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ci = 4 * ty + i;
      if (ci >= I.chains) continue;
      const size_t base = (size_t)I.p_off + (size_t)ci * I.m + I.row0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int rj = 4 * tx + j;
        if (rj >= I.rows) continue;
        if constexpr (MODE == kGemmQ) {
          out[base + rj] = hi[i][j];
        } else {
          const double v = (double)hi[i][j] + (double)lo[i][j];
          if (P64) P64[base + rj] = v;
          if (out) {
            const T pn = (T)v;
            if (drift_bits) {
              if constexpr (sizeof(T) == 4) {
                // the drift statistic in FP32: a diagnostic, far coarser than FP32
                const float dv = __fdividef(fabsf(pn - old[i][j]),
                                            (float)anorm[I.b_off + I.row0 + rj]);
                driftf = fmaxf(driftf, dv);
              } else {
                drift = fmax(drift, fabs((double)pn - (double)old[i][j]) /
                                        anorm[I.b_off + I.row0 + rj]);
              }
            }
            out[base + rj] = pn;
          }
        }
      }
    }
  }
  if (drift_bits) atomic_max_nonneg(drift_bits, fmax(drift, (double)driftf));
}

template <typename T, int MODE>
cudaError_t launch_gemm(const BatchItem* items, int n_items, int* queue, const T* Aq,
                        const double* A64, const float* Alo, const T* X, T* out, double* P64,
                        const double* anorm, unsigned long long* drift_bits, cudaStream_t s) {
  constexpr bool kDF = MODE == kGemmRefresh && sizeof(T) == 4;
  using TA = typename std::conditional<MODE == kGemmQ || kDF, T, double>::type;
  constexpr size_t smem = gemm_smem_bytes<TA, T, kDF>();
  auto k = batch_gemm_kernel<T, MODE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k<<<persistent_grid(n_items), kBThreads, smem, s>>>(items, n_items, queue, Aq, A64, Alo, X, out,
                                                      P64, anorm, drift_bits);
  return cudaGetLastError();
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
__global__ void set_t_kernel(unsigned* t_dev, unsigned v) { *t_dev = v; }

}  // namespace

template <typename T>
cudaError_t launch_batch_draw(const ChainDesc* desc, int n_chains, T* NU, uint64_t seed,
                              uint32_t t, const unsigned* t_dev, const double* bm_tab,
                              cudaStream_t s, __half* H0, __half* H1) {
  if (n_chains <= 0) return cudaSuccess;
  if (sizeof(T) == 8 && bm_tab == nullptr) return cudaErrorInvalidValue;
  batch_draw_kernel<T><<<warps_grid(n_chains), 256, 0, s>>>(desc, n_chains, NU, seed, t, t_dev,
                                                            bm_tab, H0, H1);
  return cudaGetLastError();
}

cudaError_t launch_batch_split(const ChainDesc* desc, int n_chains, const float* NU, __half* H0,
                               __half* H1, float* unscale, cudaStream_t s) {
  if (n_chains <= 0) return cudaSuccess;
  batch_split_kernel<<<warps_grid(n_chains), 256, 0, s>>>(desc, n_chains, NU, H0, H1, unscale);
  return cudaGetLastError();
}


template <typename T>
cudaError_t launch_batch_q(const BatchItem* items, int n_items, int* queue, const T* A,
                           const T* NU, T* Q, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  return launch_gemm<T, kGemmQ>(items, n_items, queue, A, nullptr, nullptr, NU, Q, nullptr,
                                nullptr, nullptr, s);
}

template <typename T>
cudaError_t launch_batch_refresh(const BatchItem* items, int n_items, int* queue,
                                 const T* Ahi, const double* A64, const float* Alo, const T* X,
                                 T* P, double* P64, const double* anorm,
                                 unsigned long long* drift_bits, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  return launch_gemm<T, kGemmRefresh>(items, n_items, queue, Ahi, A64, Alo, X, P, P64, anorm,
                                      drift_bits, s);
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

cudaError_t launch_set_t(unsigned* t_dev, unsigned v, cudaStream_t s) {
  set_t_kernel<<<1, 1, 0, s>>>(t_dev, v);
  return cudaGetLastError();
}

template cudaError_t launch_batch_draw<float>(const ChainDesc*, int, float*, uint64_t, uint32_t,
                                              const unsigned*, const double*, cudaStream_t,
                                              __half*, __half*);
template cudaError_t launch_batch_draw<double>(const ChainDesc*, int, double*, uint64_t, uint32_t,
                                               const unsigned*, const double*, cudaStream_t,
                                               __half*, __half*);
template cudaError_t launch_batch_q<float>(const BatchItem*, int, int*, const float*, const float*,
                                           float*, cudaStream_t);
template cudaError_t launch_batch_q<double>(const BatchItem*, int, int*, const double*,
                                            const double*, double*, cudaStream_t);
template cudaError_t launch_batch_refresh<float>(const BatchItem*, int, int*, const float*,
                                                 const double*, const float*, const float*,
                                                 float*, double*, const double*,
                                                 unsigned long long*, cudaStream_t);
template cudaError_t launch_batch_refresh<double>(const BatchItem*, int, int*, const double*,
                                                  const double*, const float*, const double*,
                                                  double*, double*, const double*,
                                                  unsigned long long*, cudaStream_t);

}  // namespace ess
