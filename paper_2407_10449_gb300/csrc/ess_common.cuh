// ess_common.cuh -- device helpers shared by the sampler's kernels.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11), written from its published
// round function, with counter (block n, chain, step t, (problem << 8) |
// stream) and key = the 64-bit seed.  Normals come from the Box-Muller
// transform on two uniforms u1 = (r0 + 1) / 2^32 in (0, 1], u2 = r1 / 2^32 in
// [0, 1); the theta draw uses a 53-bit uniform from block 0 of stream 1.
#pragma once

#include <cmath>
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

// Host: whether every nonzero row of the m x d matrix A has its largest |a_ij|
// in [2^-e, 2^e] (and, with check_b, |b_i| <= 2^e).  The split FP64 products
// keep per-row power-of-two scales as floats (e = 100).  The mixed form keeps
// A, b, p and q in float and compares b^2 with p^2 + q^2, which must neither
// overflow nor flush to zero for |x| and |nu| of the order of 1 (e = 30).
inline bool rows_fit_float_scales(const double* A, const double* b, long long m, long long d,
                                  bool check_b, int e) {
  const double hi = std::ldexp(1.0, e), lo = std::ldexp(1.0, -e);
  for (long long i = 0; i < m; ++i) {
    double mx = 0.0;
    for (long long j = 0; j < d; ++j) mx = std::fmax(mx, std::fabs(A[i * d + j]));
    if (mx != 0.0 && (mx < lo || mx > hi)) return false;
    if (check_b && std::fabs(b[i]) > hi) return false;
  }
  return true;
}

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

// FP64 Box-Muller without the general-purpose logarithm and sine / cosine
// (GB300's FP64 pipe is narrow), from small tables built on the host
// (bm_table_fill) and short series on reduced arguments.  Table layout
// (kBmTableSize doubles):
//   [0, 97)      c_j = 1 / (1 + (j - 32) / 128) rounded to float, j = 0 .. 96
//                (c_32 = 1 exactly);
//   [97, 194)    -ln c_j;
//   [194, 450)   sin(2 pi k / 256), k = 0 .. 255;
//   [450, 706)   cos(2 pi k / 256).
constexpr int kBmLnC = 0, kBmLnT = 97, kBmSin = 194, kBmCos = 450, kBmTableSize = 706;

// ln u1 for u1 = x / 2^32, x an integer in [1, 2^32]: x = 2^e m with
// m in [0.75, 1.5) (e, m and the table index from integer operations),
// ln u1 = (e - 32) ln 2 - ln c_j + ln(1 + r), r = m c_j - 1 for the table
// entry j nearest m (|r| < 0.0053), ln(1 + r) by its series through r^8 (the
// next term is below 2^-55 of the sum).  Near u1 = 1, c_j = 1 and r = m - 1
// exactly, so the result keeps its relative accuracy there.
__device__ __forceinline__ double ln_u32(uint64_t x, const double* __restrict__ tab) {
  constexpr double kLn2Hi = 0.6931471805599452862267639829951804131269;  // ln 2 rounded
  constexpr double kLn2Lo = 2.3190468138462996154948555e-17;               // ln 2 - kLn2Hi
  const int lz = __clzll((long long)x);
  int e = 63 - lz;
  const uint64_t frac = ((x << lz) << 1) >> 12;  // the 52 bits below the leading one
  uint64_t mbits = 0x3FF0000000000000ull | frac;  // m in [1, 2)
  int j;
  if (frac >= (1ull << 51)) {
    // m in [1.5, 2): use m / 2 in [0.75, 1), entry round((m / 2 - 1) 128)
    mbits -= 1ull << 52;
    ++e;
    j = (int)((frac + (1ull << 45)) >> 46) - 64;
  } else {
    j = (int)((frac + (1ull << 44)) >> 45);  // round((m - 1) 128)
  }
  j += 32;
  const double m = __longlong_as_double((long long)mbits);
  const double r = fma(m, __ldg(tab + kBmLnC + j), -1.0);
  // ln(1 + r) = r (1 - r/2 + r^2/3 - ... - r^7/8)
  double sum = -1.0 / 8.0;
  sum = fma(sum, r, 1.0 / 7.0);
  sum = fma(sum, r, -1.0 / 6.0);
  sum = fma(sum, r, 1.0 / 5.0);
  sum = fma(sum, r, -1.0 / 4.0);
  sum = fma(sum, r, 1.0 / 3.0);
  sum = fma(sum, r, -1.0 / 2.0);
  const double l1p = fma(r * r, sum, r);
  const double n = (double)(e - 32);
  return fma(n, kLn2Hi, fma(n, kLn2Lo, __ldg(tab + kBmLnT + j) + l1p));
}

// cos and sin of 2 pi r / 2^32 for a 32-bit r: k = round(r / 2^24) (mod 256)
// taken exactly in integers, the rest t = 2 pi (r - k 2^24) / 2^32 in
// [-pi/256, pi/256], Taylor sin t through t^7 and cos t through t^6 (the next
// terms are below 2^-60), and the angle-sum formulas with the table's sin and
// cos of 2 pi k / 256.
__device__ __forceinline__ void sincos_2pi_u32(uint32_t r, const double* __restrict__ tab,
                                               double& s, double& c) {
  constexpr double kStep = kTwoPi * 2.3283064365386962890625e-10;  // 2 pi / 2^32
  const uint32_t k = ((r + 0x800000u) >> 24) & 255u;  // r near 2^32 wraps to entry 0
  const int f = (int)(r - (k << 24));                // in [-2^23, 2^23)
  const double t = (double)f * kStep;
  const double t2 = t * t;
  const double st = fma(t * t2, fma(t2, fma(t2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), t);
  const double ct = fma(t2, fma(t2, fma(t2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
  const double sk = __ldg(tab + kBmSin + k), ck = __ldg(tab + kBmCos + k);
  s = fma(sk, ct, ck * st);
  c = fma(ck, ct, -(sk * st));
}

// Box-Muller, double precision: 4 normals from one block (tab: the tables
// above, in device memory).
__device__ __forceinline__ void box_muller4(const uint32_t r[4], double z[4],
                                            const double* __restrict__ tab) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double rad = sqrt(-2.0 * ln_u32((uint64_t)r[2 * k] + 1u, tab));
    double s, c;
    sincos_2pi_u32(r[2 * k + 1], tab, s, c);
    z[2 * k] = rad * c;
    z[2 * k + 1] = rad * s;
  }
}

// Host: the tables of the FP64 Box-Muller, from long-double library values
// rounded once to double.
inline void bm_table_fill(double* tab) {
  const long double two_pi = 2.0L * acosl(-1.0L);
  for (int j = 0; j < 97; ++j) {
    const float cj = (float)(1.0L / (1.0L + (long double)(j - 32) / 128.0L));
    tab[kBmLnC + j] = (double)cj;
    tab[kBmLnT + j] = (double)(-logl((long double)cj));
  }
  for (int k = 0; k < 256; ++k) {
    tab[kBmSin + k] = (double)sinl(two_pi * (long double)k / 256.0L);
    tab[kBmCos + k] = (double)cosl(two_pi * (long double)k / 256.0L);
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

__device__ __forceinline__ void box_muller4(const uint32_t r[4], double* out, int n,
                                            const double* __restrict__ tab) {
  double z[4];
  box_muller4(r, z, tab);
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
