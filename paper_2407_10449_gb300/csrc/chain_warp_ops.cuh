// chain_warp_ops.cuh -- warp-level pieces of the chain-step kernels that keep a
// chain's arcs in registers: the pseudo-angle buckets of the domination
// prune, warp scans, the register bitonic sort of up to kWarpSortCap arcs, and
// Alg. 3's cumulative-max sweep followed by the inverse-CDF theta draw.
#pragma once

#include <cmath>
#include <cstdint>

#include "chain_math.cuh"
#include "ess_kernels.cuh"

namespace ess {
namespace warpops {

using chainmath::kFull;
using chainmath::Lim;

constexpr int kWB = 512;                  // pseudo-angle buckets of alpha
constexpr int kCand = 256;                // candidates after the first-batch test
// Slack of pseudo-angle comparisons: far above the FP32 rounding of the
// pseudo-angles (~1e-6) and far below the bucket width (4 / kWB)
constexpr float kPhiMargin = 1e-5f;
constexpr int kCap = kWarpSortCap;        // arcs a warp sorts
constexpr int kPer = kCap / 32;           // per lane
constexpr int kWBP = kWB + kWB / 32;      // padded bucket array: bucket j at j + j / 32
constexpr int kFirst = 256;               // rows of the first batch

// Bucket j lives at j + j / 32: a lane's consecutive buckets then sit on
// different banks.
__device__ __forceinline__ int bslot(int j) { return j + (j >> 5); }

// Bucket of a pseudo-angle in [0, 4]: pa * kWB / 4 rounded to the nearest
// integer by the float add-and-round idiom (2^23 + 2^22 added, the integer
// read from the low mantissa bits), clamped to [0, kWB - 3].  Any
// non-decreasing map would do: the prune only needs bucket(a) < bucket(b) to
// imply a < b.  NaN pseudo-angles (non-finite rows) land in a valid bucket.
// The maxima of bucket j are kept in slot j + 2, so that after the prefix
// max, slot j holds the maxima of the buckets up to j - 2 (zero for j < 2).
__device__ __forceinline__ int pbucket(float pa) {
  const int k = __float_as_int(fmaf(pa, kWB / 4.0f, 12582912.0f)) - 0x4B400000;
  return min(max(k, 0), kWB - 3);
}

// A double's bits as a signed integer in the order of the values (negative
// values mirrored below zero): x < y for finite x, y exactly when
// ordered_bits(x) < ordered_bits(y), except that -0 orders below +0.
__device__ __forceinline__ long long ordered_bits(double x) {
  const long long v = __double_as_longlong(x);
  return v < 0 ? v ^ 0x7FFFFFFFFFFFFFFFll : v;
}

// In-place inclusive prefix max of kWB bucket maxima (float bits, >= 0), one warp.
__device__ __forceinline__ void prefix_max(unsigned* b, int lane) {
  unsigned run = 0u;
  unsigned* mine = b + bslot(lane * (kWB / 32));
#pragma unroll 4
  for (int k = 0; k < kWB / 32; ++k) {
    run = max(run, mine[k]);
    mine[k] = run;
  }
  unsigned incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl = max(incl, y);
  }
  unsigned before = __shfl_up_sync(kFull, incl, 1);
  if (lane == 0) before = 0u;
#pragma unroll 4
  for (int k = 0; k < kWB / 32; ++k) mine[k] = max(mine[k], before);
}

// Warp-wide min / max of a float (every lane gets the result).
__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_incl_max(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v = y > v ? y : v;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_incl_sum(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Bitonic sort of 32 P elements held as element e = lane + 32 j in key[j]
// (ascending, val travels with its key); entries j >= P are left untouched.
template <typename T, int P>
__device__ __forceinline__ void warp_bitonic(T (&key)[kPer], T (&val)[kPer], int lane) {
  constexpr int N = 32 * P;
#pragma unroll
  for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
    for (int st = kk >> 1; st > 0; st >>= 1) {
      if (st >= 32) {
        const int js = st >> 5;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const int jp = j ^ js;
          if (jp > j) {
            const int e = lane + 32 * j;
            const bool up = (e & kk) == 0;
            if ((key[j] > key[jp]) == up) {
              T tk = key[j]; key[j] = key[jp]; key[jp] = tk;
              T tv = val[j]; val[j] = val[jp]; val[jp] = tv;
            }
          }
        }
      } else {
        const bool lower = (lane & st) == 0;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const int e = lane + 32 * j;
          const bool up = (e & kk) == 0;
          const T ok = __shfl_xor_sync(kFull, key[j], st);
          const T ov = __shfl_xor_sync(kFull, val[j], st);
          // the lower element keeps the smaller key when sorting upwards
          const bool take = lower == up ? ok < key[j] : ok > key[j];
          if (take) {
            key[j] = ok;
            val[j] = ov;
          }
        }
      }
    }
  }
}

// Sorts n arcs (n <= kCap; entries past n hold key = +inf) with the smallest
// power-of-two network that holds them.
template <typename T>
__device__ __forceinline__ void warp_sort_arcs(T (&key)[kPer], T (&val)[kPer], int n, int lane) {
  if (n <= 32) warp_bitonic<T, 1>(key, val, lane);
  else if (n <= 64) warp_bitonic<T, 2>(key, val, lane);
  else warp_bitonic<T, kPer>(key, val, lane);
}

// Alg. 3 on n_roots arcs sorted by alpha (key = alpha, val = beta, element
// e = lane + 32 j): gamma = inclusive cumulative max of beta, piece e =
// [gamma_(e-1), alpha_(e)] (piece 0 starts at the glued point 0) and the tail
// [gamma_last, 2 pi]; trimming moves only constraint endpoints by eps.  Then
// theta ~ U(I_act) by the inverse CDF at u: the last positive piece starting
// at or below s = u L.  Optionally writes the positive pieces (ascending) to
// pieces_row (max_pieces pairs) and their count to *npieces.  Returns theta
// (warp-uniform; 0 when I_act has no positive length).
template <typename T>
__device__ __forceinline__ T warp_sweep_theta(const T (&key)[kPer], const T (&val)[kPer],
                                              int n_roots, T eps, double u, int lane,
                                              double* pieces_row, int max_pieces, int* npieces) {
  const T two_pi = Lim<T>::two_pi();
  T plo[kPer], phi[kPer], plen[kPer], sexcl[kPer];
  T gcarry = T(0), scarry = T(0);
  const int jn = (n_roots + 31) >> 5;  // register slots holding roots (warp-uniform)
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (j >= jn) {
      plo[j] = phi[j] = plen[j] = sexcl[j] = T(0);
      continue;
    }
    const int e = lane + 32 * j;
    const bool valid = e < n_roots;
    const T v = valid ? val[j] : T(0);
    T incl = warp_incl_max<T>(v, lane);
    incl = incl > gcarry ? incl : gcarry;
    T gprev = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) gprev = gcarry;
    gcarry = __shfl_sync(kFull, incl, 31);
    // piece e: [gamma_(e-1), alpha_(e)]; piece 0 starts at the glued point 0
    const T lo = e == 0 ? T(0) : gprev + eps;
    const T hi = key[j] - eps;
    plo[j] = lo;
    phi[j] = hi;
    plen[j] = valid && hi > lo ? hi - lo : T(0);
    const T sincl = warp_incl_sum<T>(plen[j], lane) + scarry;
    T sx = __shfl_up_sync(kFull, sincl, 1);
    sexcl[j] = lane == 0 ? scarry : sx;
    scarry = __shfl_sync(kFull, sincl, 31);
  }
  const T mid_total = scarry;
  const T tail_lo = n_roots > 0 ? gcarry + eps : T(0);
  const T tail_len = two_pi > tail_lo ? two_pi - tail_lo : T(0);
  const T total = mid_total + tail_len;

  // theta ~ U(I_act): the last positive piece starting at or below s
  const T s = (T)(u * (double)total);
  int cand = -1;
  T cand_theta = T(0);
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (plen[j] > T(0) && sexcl[j] <= s) {
      cand = lane + 32 * j;
      const T th = plo[j] + (s - sexcl[j]);
      cand_theta = th < phi[j] ? th : phi[j];
    }
  }
  if (tail_len > T(0) && mid_total <= s) {
    cand = kCap;  // the tail is the last piece
    const T th = tail_lo + (s - mid_total);
    cand_theta = th < two_pi ? th : two_pi;
  }
  int best = cand;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
  const unsigned owners = __ballot_sync(kFull, cand == best);
  T theta = __shfl_sync(kFull, cand_theta, __ffs(owners) - 1);
  if (best < 0 || !(total > T(0))) theta = T(0);

  // optional: the positive-length pieces (test/diagnostic output)
  if (pieces_row != nullptr || npieces != nullptr) {
    int at = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const bool pos = plen[j] > T(0);
      const unsigned ball = __ballot_sync(kFull, pos);
      const int k = at + __popc(ball & ((1u << lane) - 1u));
      if (pos && pieces_row && k < max_pieces) {
        pieces_row[2 * k] = (double)plo[j];
        pieces_row[2 * k + 1] = (double)phi[j];
      }
      at += __popc(ball);
    }
    if (lane == 0) {
      if (pieces_row && tail_len > T(0) && at < max_pieces) {
        pieces_row[2 * at] = (double)tail_lo;
        pieces_row[2 * at + 1] = (double)two_pi;
      }
      if (npieces) *npieces = at + (tail_len > T(0) ? 1 : 0);
    }
  }
  return theta;
}

}  // namespace warpops
}  // namespace ess
