// ess_common.cuh -- device helpers shared by the sampler's kernels.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11), written from its published
// round function, with counter (block n, chain, step t, (problem << 8) |
// stream) and key = the 64-bit seed.  Normals come from the Box-Muller
// transform on two uniforms u1 = (r0 + 1) / 2^32 in (0, 1], u2 = r1 / 2^32 in
// [0, 1); the theta draw uses a 53-bit uniform from block 0 of stream 1.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace ess {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kTwoPiF = 6.28318548202514648f;  // 2 pi rounded to float (upwards)
// Scale of drawn nu in its fp16 split for the tensor-core product: the float
// Box-Muller radius sqrt(-2 ln u1) with u1 >= 2^-32 stays below 6.67, so
// nu * 2^12 stays below 2^15, inside the fp16 range, with no per-chain scan.
constexpr float kNuSplitScale = 4096.f;

// Device-side counters of one launch sequence (accumulated over a run).
struct DevStats {
  unsigned long long steps;
  unsigned long long rejections;
  unsigned long long rechecks;
  unsigned long long tangent_fp64;
  unsigned long long numeric_errors;
  unsigned long long max_drift_bits;     // double bits of a non-negative max
  unsigned long long max_residual_bits;  // ordered bits of max residual (see enc)
  unsigned long long sort_keys;          // arcs left for the sort after the prune
};

// Error flags in the device status word.
enum : int { kStatusNumeric = 1, kStatusInfeasible = 2, kStatusTimeout = 4 };

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ void rng_block(uint64_t seed, uint32_t n, uint32_t chain, uint32_t t,
                                          uint32_t problem, uint32_t stream, uint32_t out[4]) {
  philox4x32_10(n, chain, t, (problem << 8) | (stream & 0xFFu), (uint32_t)seed,
                (uint32_t)(seed >> 32), out);
}

// ln u1 for u1 = x / 2^32, x an integer in [1, 2^32], in double precision
// without the general-purpose logarithm (GB300's FP64 pipe is narrow): with
// x = 2^e m, m in [0.75, 1.5) (e and m from integer operations),
//   ln u1 = (e - 32) ln 2 + ln m,  ln m = 2 atanh(f),  f = (m - 1) / (m + 1),
// f in [-1/7, 1/5], and the atanh series 2 f (1 + f^2/3 + ... + f^20/21), whose
// next term is below 2^-54 of the sum.  Near u1 = 1 (e = 32) m - 1 is exact,
// so the result keeps its relative accuracy there.
__device__ __forceinline__ double ln_u32(uint64_t x) {
  constexpr double kLn2Hi = 0.6931471805599452862267639829951804131269;  // ln 2 rounded
  constexpr double kLn2Lo = 2.3190468138462996154948555e-17;               // ln 2 - kLn2Hi
  const int lz = __clzll((long long)x);
  int e = 63 - lz;
  const uint64_t frac = ((x << lz) << 1) >> 12;  // the bits below the leading one
  double m = __longlong_as_double((long long)(0x3FF0000000000000ull | frac));  // [1, 2)
  if (m >= 1.5) {
    m *= 0.5;
    ++e;
  }
  const double f = (m - 1.0) / (m + 1.0);
  const double f2 = f * f;
  double sum = 1.0 / 21.0;
  sum = fma(sum, f2, 1.0 / 19.0);
  sum = fma(sum, f2, 1.0 / 17.0);
  sum = fma(sum, f2, 1.0 / 15.0);
  sum = fma(sum, f2, 1.0 / 13.0);
  sum = fma(sum, f2, 1.0 / 11.0);
  sum = fma(sum, f2, 1.0 / 9.0);
  sum = fma(sum, f2, 1.0 / 7.0);
  sum = fma(sum, f2, 1.0 / 5.0);
  sum = fma(sum, f2, 1.0 / 3.0);
  const double lnm = fma(f * f2, sum, f) * 2.0;  // 2 (f + f^3 (1/3 + ...))
  const double n = (double)(e - 32);
  return fma(n, kLn2Hi, fma(n, kLn2Lo, lnm));
}

// cos and sin of 2 pi r / 2^32 for a 32-bit r: the quadrant k = round(r / 2^30)
// is taken exactly in integers, the rest t = 2 pi (r - k 2^30) / 2^32 lies in
// [-pi/4, pi/4], where the Taylor series of sin through t^17 and of cos
// through t^16 leave a truncation below 2^-54.
__device__ __forceinline__ void sincos_2pi_u32(uint32_t r, double& s, double& c) {
  constexpr double kStep = kTwoPi * 2.3283064365386962890625e-10;  // 2 pi / 2^32
  const uint32_t k = ((r + 0x20000000u) >> 30) & 3u;  // r near 2^32 wraps to quadrant 0
  const int f = (int)(r - (k << 30));                // in [-2^29, 2^29)
  const double t = (double)f * kStep;
  const double t2 = t * t;
  // sin t = t + t^3 P(t^2),  P = -1/3! + t^2/5! - ... + t^14/17!
  double ps = 1.0 / 355687428096000.0;       // 1/17!
  ps = fma(ps, t2, -1.0 / 1307674368000.0);  // 1/15!
  ps = fma(ps, t2, 1.0 / 6227020800.0);      // 1/13!
  ps = fma(ps, t2, -1.0 / 39916800.0);       // 1/11!
  ps = fma(ps, t2, 1.0 / 362880.0);          // 1/9!
  ps = fma(ps, t2, -1.0 / 5040.0);           // 1/7!
  ps = fma(ps, t2, 1.0 / 120.0);             // 1/5!
  ps = fma(ps, t2, -1.0 / 6.0);              // 1/3!
  const double st = fma(t * t2, ps, t);
  // cos t = 1 + t^2 Q(t^2),  Q = -1/2! + t^2/4! - ... + t^14/16!
  double pc = 1.0 / 20922789888000.0;        // 1/16!
  pc = fma(pc, t2, -1.0 / 87178291200.0);    // 1/14!
  pc = fma(pc, t2, 1.0 / 479001600.0);       // 1/12!
  pc = fma(pc, t2, -1.0 / 3628800.0);        // 1/10!
  pc = fma(pc, t2, 1.0 / 40320.0);           // 1/8!
  pc = fma(pc, t2, -1.0 / 720.0);            // 1/6!
  pc = fma(pc, t2, 1.0 / 24.0);              // 1/4!
  pc = fma(pc, t2, -0.5);                    // 1/2!
  const double ct = fma(t2, pc, 1.0);
  // rotate by k quarter turns
  const double sa = (k & 1u) ? ct : st, ca = (k & 1u) ? st : ct;
  s = (k & 2u) ? -sa : sa;
  c = ((k + 1u) & 2u) ? -ca : ca;
}

// Box-Muller, double precision: 4 normals from one block.
__device__ __forceinline__ void box_muller4(const uint32_t r[4], double z[4]) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double rad = sqrt(-2.0 * ln_u32((uint64_t)r[2 * k] + 1u));
    double s, c;
    sincos_2pi_u32(r[2 * k + 1], s, c);
    z[2 * k] = rad * c;
    z[2 * k + 1] = rad * s;
  }
}

// Box-Muller, single precision: 4 normals from one block.
__device__ __forceinline__ void box_muller4(const uint32_t r[4], float z[4]) {
  const float inv32 = 2.3283064365386963e-10f;  // 2^-32
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    // ln u1 with u1 = (r + 1) / 2^32: for u1 <= 1/2 directly, by the fast
    // hardware logarithm (ln u1 <= -ln 2 there, so its relative error stays
    // below 2^-21); for u1 > 1/2 as log1p(-v) with v = 1 - u1 =
    // (2^32 - 1 - r) / 2^32, so that the rounding of r to 24 bits never
    // dominates a logarithm close to zero
    const uint32_t r0 = r[2 * k];
    const float lnu = r0 < 0x80000000u ? __logf(fmaf((float)r0, inv32, inv32))
                                       : log1pf(-(float)(~r0) * inv32);
    const float u2 = (float)r[2 * k + 1] * inv32;
    const float rad = sqrtf(-2.0f * lnu);
    // cos and sin of 2 pi u2 by the hardware approximations on the reduced
    // angle 2 pi (u2 - rint(u2)) in [-pi, pi] (absolute error below 2^-21)
    float s, c;
    __sincosf(6.28318530717958648f * (u2 - rintf(u2)), &s, &c);
    z[2 * k] = rad * c;
    z[2 * k + 1] = rad * s;
  }
}

__device__ __forceinline__ void box_muller4(const uint32_t r[4], double* out, int n) {
  double z[4];
  box_muller4(r, z);
  for (int k = 0; k < n; ++k) out[k] = z[k];
}

// 53-bit uniform in [0, 1) for the theta draw.
__device__ __forceinline__ double theta_uniform(uint64_t seed, uint32_t chain, uint32_t t,
                                                uint32_t problem) {
  uint32_t r[4];
  rng_block(seed, 0u, chain, t, problem, 1u, r);
  unsigned long long hi = r[0] >> 5, lo = r[1] >> 6;
  return (double)(hi * 67108864ull + lo) * 1.1102230246251565404236316680908203125e-16;  // 2^-53
}

// Non-negative double max via its bit pattern (monotone for x >= 0).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  if (!(v > 0.0)) return;
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Order-preserving encoding of any double into uint64 for atomicMax.
__host__ __device__ __forceinline__ unsigned long long enc_ordered(double v) {
  long long b;
#ifdef __CUDA_ARCH__
  b = __double_as_longlong(v);
#else
  __builtin_memcpy(&b, &v, 8);
#endif
  unsigned long long u = (unsigned long long)b;
  return (b < 0) ? ~u : (u | 0x8000000000000000ull);
}

__host__ __device__ __forceinline__ double dec_ordered(unsigned long long u) {
  unsigned long long b = (u & 0x8000000000000000ull) ? (u & ~0x8000000000000000ull) : ~u;
  double v;
#ifdef __CUDA_ARCH__
  v = __longlong_as_double((long long)b);
#else
  __builtin_memcpy(&v, &b, 8);
#endif
  return v;
}

}  // namespace ess
