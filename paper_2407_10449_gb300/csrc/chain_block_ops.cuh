// chain_block_ops.cuh -- block-level pieces of the CTA-per-chain step kernels:
// exclusive scans over a CTA, and the sort of a chain's arcs by alpha (Alg. 3
// sorts the arcs before its cumulative-max sweep), kept in registers in a
// blocked arrangement (thread t holds sorted positions t ITEMS .. t ITEMS +
// ITEMS - 1).
#pragma once

#include "chain_math.cuh"

namespace ess {
namespace blockops {

using chainmath::kFull;

struct OpAdd {
  template <typename V> __device__ V operator()(V a, V b) const { return a + b; }
};
struct OpMax {
  template <typename V> __device__ V operator()(V a, V b) const { return a > b ? a : b; }
};

// Exclusive block scan; returns the exclusive prefix of `v`, sets `total`.
// `tmp` holds NT/32 values.  Contains __syncthreads (call uniformly).
template <int NT, typename V, typename Op>
__device__ V block_exclusive_scan(V v, V identity, Op op, V* tmp, V& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  V x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    V y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x = op(x, y);
  }
  if (lane == 31) tmp[w] = x;
  __syncthreads();
  if (w == 0) {
    V t = lane < NW ? tmp[lane] : identity;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      V y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t = op(t, y);
    }
    if (lane < NW) tmp[lane] = t;
  }
  __syncthreads();
  V warp_prefix = w > 0 ? tmp[w - 1] : identity;
  total = tmp[NW - 1];
  // exclusive within the warp
  V incl_prev = __shfl_up_sync(kFull, x, 1);
  V excl = lane > 0 ? op(warp_prefix, incl_prev) : warp_prefix;
  __syncthreads();
  return excl;
}

// Shared-memory slot of sorted position e: one padding word per 32 keeps the
// per-thread chunks (stride ITEMS) on distinct banks.
__device__ __forceinline__ int pad_idx(int e) { return e + (e >> 5); }

// Sorts the arcs held in registers (blocked: thread t holds positions
// t ITEMS + i) by key, ascending, with val as payload.  Only the first
// n_active_slots positions (a multiple of ITEMS) hold arcs; threads past them
// hold +inf keys and take no part in the merges.  A bitonic network sorts each
// thread's ITEMS registers, then merge-path merges of sorted runs of width
// ITEMS, 2 ITEMS, ... through shared memory (s_key, s_val: padded, at least
// pad_idx(n_active_slots) entries each) until one run holds every arc.  Equal
// keys keep the order of their runs.  Contains __syncthreads (call uniformly).
template <int ITEMS, typename T>
__device__ __forceinline__ void block_sort_arcs(T (&key)[ITEMS], T (&val)[ITEMS],
                                                int n_active_slots, T* s_key, T* s_val, T inf) {
  const int base = threadIdx.x * ITEMS;
  const bool owns = base < n_active_slots;
#pragma unroll
  for (int kk = 2; kk <= ITEMS; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & kk) == 0;
          if ((key[i] > key[l]) == up) {
            T tk = key[i]; key[i] = key[l]; key[l] = tk;
            T tv = val[i]; val[i] = val[l]; val[l] = tv;
          }
        }
      }
    }
  }
  for (int w = ITEMS; w < n_active_slots; w <<= 1) {
    __syncthreads();
    if (owns) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        s_key[pad_idx(base + i)] = key[i];
        s_val[pad_idx(base + i)] = val[i];
      }
    }
    __syncthreads();
    if (owns) {
      const int start = base & ~(2 * w - 1);
      const int diag = base - start;
      // runs [start, start + w) and [start + w, start + 2w), clipped to the arcs
      const int a_end = min(w, n_active_slots - start);
      const int b_len = max(0, min(w, n_active_slots - start - w));
      int lo = diag - b_len > 0 ? diag - b_len : 0;
      int hi = diag < a_end ? diag : a_end;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!(s_key[pad_idx(start + w + diag - 1 - mid)] < s_key[pad_idx(start + mid)])) lo = mid + 1;
        else hi = mid;
      }
      int ia = lo, ib = diag - lo;
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const bool a_ok = ia < a_end;
        const bool b_ok = ib < b_len;
        const T ka = a_ok ? s_key[pad_idx(start + ia)] : inf;
        const T kb = b_ok ? s_key[pad_idx(start + w + ib)] : inf;
        const bool take_a = a_ok && (!b_ok || !(kb < ka));
        key[i] = take_a ? ka : kb;
        val[i] = take_a ? s_val[pad_idx(start + ia)] : (b_ok ? s_val[pad_idx(start + w + ib)] : T(0));
        ia += take_a ? 1 : 0;
        ib += take_a ? 0 : 1;
      }
    }
  }
}

}  // namespace blockops
}  // namespace ess
