// k_draw.cu -- nu ~ N(0, I_d) for every chain (Alg. 1, "sample nu_t"),
// Philox4x32-10 + Box-Muller (see ess_common.cuh), plus small conversion and
// checking kernels.
#include "ess_kernels.cuh"

namespace ess {
namespace {

__device__ __forceinline__ uint32_t h2_bits(__half2 v) {
  return *reinterpret_cast<const uint32_t*>(&v);
}

// One thread per (chain, Philox block): 4 consecutive coordinates.
__global__ void draw_nu_f64_kernel(double* __restrict__ nu, int n_chains, int d, int ld,
                                   uint64_t seed, uint32_t t, const unsigned* t_dev,
                                   uint32_t problem, uint32_t chain0,
                                   const double* __restrict__ bm_tab) {
  const int nblk = (d + 3) >> 2;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n_chains * nblk) return;
  if (t_dev) t += *t_dev;
  const int c = (int)(gid / nblk), n = (int)(gid % nblk);
  uint32_t r[4];
  rng_block(seed, (uint32_t)n, chain0 + (uint32_t)c, t, problem, 0u, r);
  double z[4];
  box_muller4(r, z, bm_tab);
  double* row = nu + (size_t)c * ld + 4 * n;
  const int left = d - 4 * n;
  if (left >= 4 && ((reinterpret_cast<uintptr_t>(row) & 15) == 0)) {
    reinterpret_cast<double2*>(row)[0] = make_double2(z[0], z[1]);
    reinterpret_cast<double2*>(row)[1] = make_double2(z[2], z[3]);
  } else {
    for (int k = 0; k < 4 && k < left; ++k) row[k] = z[k];
  }
}

__global__ void draw_nu_f32_kernel(float* __restrict__ nu, int ld, __half* __restrict__ h0,
                                   __half* __restrict__ h1, int ld16, int n_chains, int d,
                                   uint64_t seed, uint32_t t, const unsigned* t_dev,
                                   uint32_t problem, uint32_t chain0) {
  const int nblk = (d + 3) >> 2;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n_chains * nblk) return;
  if (t_dev) t += *t_dev;
  const int c = (int)(gid / nblk), n = (int)(gid % nblk);
  uint32_t r[4];
  rng_block(seed, (uint32_t)n, chain0 + (uint32_t)c, t, problem, 0u, r);
  float z[4];
  box_muller4(r, z);
  const int left = d - 4 * n;
  float* row = nu + (size_t)c * ld + 4 * n;
  if (left >= 4 && (reinterpret_cast<uintptr_t>(row) & 15) == 0) {
    *reinterpret_cast<float4*>(row) = make_float4(z[0], z[1], z[2], z[3]);
  } else {
    for (int k = 0; k < 4 && k < left; ++k) row[k] = z[k];
  }
  if (h0 != nullptr) {
    // two-way fp16 split of nu * 2^12 (|nu| < 6.67 keeps it below 2^15):
    // y = a + b + r with a = fp16(y), b = fp16(y - a), two values per
    // conversion instruction
    __half2 a[2], b[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float2 y = make_float2(z[2 * k] * kNuSplitScale, z[2 * k + 1] * kNuSplitScale);
      a[k] = __float22half2_rn(y);
      const float2 af = __half22float2(a[k]);
      b[k] = __float22half2_rn(make_float2(y.x - af.x, y.y - af.y));
    }
    const size_t o = (size_t)c * ld16 + 4 * n;
    if (left >= 4 && (o & 3) == 0) {
      // 8-byte stores of four fp16 values (ld16 is a multiple of 8)
      *reinterpret_cast<uint2*>(h0 + o) = make_uint2(h2_bits(a[0]), h2_bits(a[1]));
      *reinterpret_cast<uint2*>(h1 + o) = make_uint2(h2_bits(b[0]), h2_bits(b[1]));
    } else {
      for (int k = 0; k < 4 && k < left; ++k) {
        h0[o + k] = (k & 1) ? __high2half(a[k >> 1]) : __low2half(a[k >> 1]);
        h1[o + k] = (k & 1) ? __high2half(b[k >> 1]) : __low2half(b[k >> 1]);
      }
    }
  }
}

__global__ void philox_blocks_kernel(uint64_t seed, uint32_t chain, uint32_t t, uint32_t problem,
                                     uint32_t stream, int n_blocks, uint32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_blocks) return;
  uint32_t r[4];
  rng_block(seed, (uint32_t)i, chain, t, problem, stream, r);
  out[4 * i + 0] = r[0];
  out[4 * i + 1] = r[1];
  out[4 * i + 2] = r[2];
  out[4 * i + 3] = r[3];
}

template <typename Ti, typename To>
__global__ void convert_kernel(const Ti* __restrict__ src, int lds, To* __restrict__ dst, int ldd,
                               int rows, int cols) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)rows * cols) return;
  const int r = (int)(gid / cols), j = (int)(gid % cols);
  dst[(size_t)r * ldd + j] = (To)src[(size_t)r * lds + j];
}

__global__ void check_feasible_kernel(const double* __restrict__ P, int ldp,
                                      const double* __restrict__ b, int rows, int m, int* status) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)rows * m) return;
  const int r = (int)(gid / m), i = (int)(gid % m);
  const double v = P[(size_t)r * ldp + i];
  if (!(v <= b[i])) atomicOr(status, kStatusInfeasible);
}

// Feasibility of float states from an exact-split product P (error at most
// bound * s_i * t_c): certain violations and certain passes are decided from
// P; the few entries within the bound are recomputed with FP64 FMAs.
template <typename TX>
__global__ void check_feasible_bounded_kernel(const double* __restrict__ P, int ldp,
                                              const double* __restrict__ b, int rows, int m,
                                              const float* __restrict__ row_scale,
                                              const float* __restrict__ col_scale, double bound,
                                              const TX* __restrict__ X, int ldx,
                                              const double* __restrict__ A, int d, int* status) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)rows * m) return;
  const int r = (int)(gid / m), i = (int)(gid % m);
  const double v = P[(size_t)r * ldp + i];
  const double e = bound * (double)row_scale[r] * (double)col_scale[i];
  if (!(v <= b[i] + e)) {
    atomicOr(status, kStatusInfeasible);
  } else if (v > b[i] - e) {
    const TX* x = X + (size_t)r * ldx;
    const double* a = A + (size_t)i * d;
    double acc = 0.0;
    for (int j = 0; j < d; ++j) acc = fma(a[j], (double)x[j], acc);
    if (acc > b[i]) atomicOr(status, kStatusInfeasible);
  }
}

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

cudaError_t launch_draw_nu_f64(double* nu, int n_chains, int d, int ld, uint64_t seed, uint32_t t,
                               uint32_t problem, uint32_t chain0, const double* bm_tab,
                               cudaStream_t s, const unsigned* t_dev) {
  const long long n = (long long)n_chains * ((d + 3) / 4);
  if (n == 0) return cudaSuccess;
  if (bm_tab == nullptr) return cudaErrorInvalidValue;
  draw_nu_f64_kernel<<<grid_for(n, 256), 256, 0, s>>>(nu, n_chains, d, ld, seed, t, t_dev,
                                                      problem, chain0, bm_tab);
  return cudaGetLastError();
}

cudaError_t launch_draw_nu_f32(float* nu, int ld, __half* const split[2], int ld16, int n_chains,
                               int d, uint64_t seed, uint32_t t, uint32_t problem, uint32_t chain0,
                               cudaStream_t s, const unsigned* t_dev) {
  const long long n = (long long)n_chains * ((d + 3) / 4);
  if (n == 0) return cudaSuccess;
  __half* h0 = split ? split[0] : nullptr;
  __half* h1 = split ? split[1] : nullptr;
  draw_nu_f32_kernel<<<grid_for(n, 256), 256, 0, s>>>(nu, ld, h0, h1, ld16, n_chains, d, seed, t,
                                                      t_dev, problem, chain0);
  return cudaGetLastError();
}

cudaError_t launch_philox_blocks(uint64_t seed, uint32_t chain, uint32_t t, uint32_t problem,
                                 uint32_t stream, int n_blocks, uint32_t* out, cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  philox_blocks_kernel<<<grid_for(n_blocks, 256), 256, 0, s>>>(seed, chain, t, problem, stream,
                                                               n_blocks, out);
  return cudaGetLastError();
}

template <typename Ti, typename To>
cudaError_t launch_convert(const Ti* src, int lds, To* dst, int ldd, int rows, int cols,
                           cudaStream_t s) {
  const long long n = (long long)rows * cols;
  if (n == 0) return cudaSuccess;
  convert_kernel<Ti, To><<<grid_for(n, 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_check_feasible(const double* P, int ldp, const double* b, int rows, int m,
                                  int* status, cudaStream_t s) {
  const long long n = (long long)rows * m;
  if (n == 0) return cudaSuccess;
  check_feasible_kernel<<<grid_for(n, 256), 256, 0, s>>>(P, ldp, b, rows, m, status);
  return cudaGetLastError();
}

template <typename TX>
cudaError_t launch_check_feasible_bounded(const double* P, int ldp, const double* b, int rows,
                                          int m, const float* row_scale, const float* col_scale,
                                          double bound, const TX* X, int ldx, const double* A,
                                          int d, int* status, cudaStream_t s) {
  const long long n = (long long)rows * m;
  if (n == 0) return cudaSuccess;
  check_feasible_bounded_kernel<TX><<<grid_for(n, 256), 256, 0, s>>>(P, ldp, b, rows, m, row_scale,
                                                                 col_scale, bound, X, ldx, A, d,
                                                                 status);
  return cudaGetLastError();
}

template cudaError_t launch_check_feasible_bounded<float>(const double*, int, const double*, int,
                                                         int, const float*, const float*, double,
                                                         const float*, int, const double*, int,
                                                         int*, cudaStream_t);
template cudaError_t launch_check_feasible_bounded<double>(const double*, int, const double*, int,
                                                          int, const float*, const float*, double,
                                                          const double*, int, const double*, int,
                                                          int*, cudaStream_t);

template cudaError_t launch_convert<double, float>(const double*, int, float*, int, int, int,
                                                   cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, int, double*, int, int, int,
                                                   cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, int, double*, int, int, int,
                                                    cudaStream_t);

}  // namespace ess
