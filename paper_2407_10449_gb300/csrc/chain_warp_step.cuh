// chain_warp_step.cuh -- one elliptical-slice step of one chain by one WARP.
//
// The same map as the CTA-per-chain step (Alg. 1 body: App. B roots, Alg. 3
// sort and cumulative-max sweep, inverse-CDF theta, move and Sec. 3.3
// safeguard), organised for the common case where few arcs matter:
//   1. classify each row (no root / near tangency / arc) and place its arc by
//      pseudo-angles of the two roots (a monotone stand-in for the angle,
//      computed without trigonometry); a first batch of 256 rows gives
//      per-bucket maxima of beta over 512 alpha buckets, then every row is
//      tested against them (and added to the full maxima): rows whose arc lies
//      inside an arc that starts at least two buckets earlier are dropped;
//   2. the remaining candidates are tested again against the full maxima (the
//      union of arcs, hence I_act and its piece endpoints, is unchanged by
//      dropping contained arcs);
//   3. exact roots for the <= 128 surviving rows, bitonic sort of alpha with
//      beta as payload in registers (4 per lane, warp shuffles), cumulative
//      max and piece lengths by warp scans, theta by the inverse CDF;
//   4. stream the rows again: p' = p cos + q sin written to P_out, rows near
//      their bound rechecked in FP64 against x' = x cos + nu sin; then x'.
// No block-wide barrier is needed.  A chain with more than 128 surviving arcs
// is left untouched and appended to prm.overflow_list for the CTA-per-chain
// step.  Used by the warp-per-chain kernel and by the persistent batched step.
#pragma once

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "chain_math.cuh"
#include "chain_warp_ops.cuh"
#include "ess_kernels.cuh"

namespace ess {
namespace {

using namespace chainmath;
using namespace warpops;

#ifndef ESS_WARP_BATCH
#define ESS_WARP_BATCH 8
#endif
#ifndef ESS_WARP_MINBLOCKS
#define ESS_WARP_MINBLOCKS 4
#endif
// FP64 chains: their double p, q and thresholds take twice the registers per
// row in flight; 4 rows per lane and trip keep them out of local memory at 4
// CTAs per SM (measured at d = 1000, m = 2000, 8192 chains: 0.516 ms per step
// against 0.551 with 8 rows, 0.551 with 4 rows at 3 CTAs, 0.586 with 8 rows
// at 2 CTAs)
#ifndef ESS_WARP_BATCH_F64
#define ESS_WARP_BATCH_F64 4
#endif
#ifndef ESS_WARP_MINBLOCKS_F64
#define ESS_WARP_MINBLOCKS_F64 4
#endif
constexpr int kBatchF32 = ESS_WARP_BATCH;  // rows per lane in flight per loop trip (float)
// Candidate codes: a kept row is 0x80000000 | i; an arc is bucket << kRowBits
// | i (buckets < kWB = 2^9 fill bits 22 .. 30), so rows up to 2^22.
constexpr int kRowBits = 22;
constexpr unsigned kRowMask = (1u << kRowBits) - 1u;
static_assert(kWB <= 512, "bucket field of the candidate code");

// Rows of one loop trip (32 kBatch rows from i0) and the lane slots that hold
// them.  Lane-strided form: slot k of a lane is row i0 + lane + 32 k, one
// 32-bit load per row.  Vector form (float rows on 16-byte boundaries, whole
// trips): a lane takes four consecutive rows per 128-bit load, slot k being
// row i0 + 4 (lane + 32 (k / 4)) + k % 4; a warp's load still covers 512
// consecutive bytes.
template <bool VEC>
__device__ __forceinline__ int slot_row(int i0, int lane, int k) {
  return VEC ? i0 + 4 * (lane + 32 * (k >> 2)) + (k & 3) : i0 + lane + 32 * k;
}

// The slots of a whole trip of float rows, 128 bits at a time (VEC) or one row
// per slot.
template <bool VEC, int N>
__device__ __forceinline__ void load_trip(const float* __restrict__ src, int i0, int lane,
                                          float (&out)[N]) {
  if constexpr (VEC) {
    static_assert(N % 4 == 0, "vector trips take four rows per load");
#pragma unroll
    for (int g = 0; g < N / 4; ++g) {
      const float4 t = *reinterpret_cast<const float4*>(src + i0 + 4 * (lane + 32 * g));
      out[4 * g] = t.x;
      out[4 * g + 1] = t.y;
      out[4 * g + 2] = t.z;
      out[4 * g + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = src[i0 + lane + 32 * k];
  }
}

template <bool VEC, int N>
__device__ __forceinline__ void store_trip(float* __restrict__ dst, int i0, int lane,
                                           const float (&in)[N]) {
  if constexpr (VEC) {
#pragma unroll
    for (int g = 0; g < N / 4; ++g)
      *reinterpret_cast<float4*>(dst + i0 + 4 * (lane + 32 * g)) =
          make_float4(in[4 * g], in[4 * g + 1], in[4 * g + 2], in[4 * g + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) dst[i0 + lane + 32 * k] = in[k];
  }
}

__device__ __forceinline__ bool aligned16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// Shared memory of one warp's chain step: two padded bucket arrays,
// candidates (code, pseudo-beta), survivor rows (16-byte aligned base).
constexpr size_t kWarpStepSmem = ((size_t)2 * kWBP + 2 * kCand + kCap) * 4;

// One step of chain c by the calling warp (all 32 lanes), with kWarpStepSmem
// bytes of shared memory at wsm.  Returns the chain's sorted keys (the same
// on every lane), or -1 if the chain was left untouched for the CTA-per-chain
// step (appended to prm.overflow_list when prm.overflow_count is set).
// LONG: compile the long-arc union (used for the chains whose view has
// long_arcs set); without it the kernel carries none of that code.
template <typename T, bool BATCH, bool LONG = false>
__device__ __forceinline__ int warp_chain_step(const ChainParams<T>& prm, int c,
                                               unsigned char* wsm, int lane) {
  constexpr int kBatch = sizeof(T) == 4 ? kBatchF32 : ESS_WARP_BATCH_F64;
  unsigned* bsub = reinterpret_cast<unsigned*>(wsm);
  unsigned* bfull = bsub + kWBP;
  unsigned* candc = bfull + kWBP;
  float* candb = reinterpret_cast<float*>(candc + kCand);
  int* surv = reinterpret_cast<int*>(candb + kCand);
  const T inf = Lim<T>::inf();
  int my_sort_keys = 0;
  const ChainView<T> v = chain_view<T, BATCH>(prm, c);
  const int m = v.m, d = v.d;
  const T* Prow = v.P;
  const T* Qrow = v.Q;
  // clear bsub and bfull (contiguous, 16-byte aligned: 2 kWBP words)
  for (int k = lane; k < 2 * kWBP / 4; k += 32)
    reinterpret_cast<uint4*>(bsub)[k] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  const T tlo = (T)(1.0 - prm.tangent_thresh);
  const T thi = (T)(1.0 + prm.tangent_thresh);
  // squared thresholds of the float classification (1e-6 relative slack)
  const float tlo_s = (float)((1.0 - prm.tangent_thresh) * 0.999999);
  const float thi_s = (float)((1.0 + prm.tangent_thresh) * 1.000001);
  const float tlo2 = tlo_s * tlo_s, thi2 = thi_s * thi_s;
  bool infeasible = false, nonfinite = false;

  // Long arcs: a row with b_i <= 0 has h_i >= pi / 2, an infeasible arc of
  // length >= pi.  Two such open arcs inside (0, 2 pi) (theta = 0 is feasible)
  // overlap, so all of them form ONE arc (min alpha, max beta); any arc inside
  // it can be dropped without changing I_act, as long as the rows holding the
  // two extremes stay.  ua / ub: min pseudo-alpha and max pseudo-beta of the
  // long arcs seen (+inf / -inf: none).
  float ua = INFINITY, ub = -INFINITY;

  // ---- 1a. a first batch of rows builds bucket maxima of beta ---------------
  // (with m <= kCand every row fits the candidate list: no first batch)
  const int m_sub = m > kCand ? min(m, kFirst) : 0;
  // float rows on 16-byte boundaries are read 128 bits at a time
  // (one problem's chains; packed batches of uneven m keep lane-strided rows)
  bool vec_rows = false;
  if constexpr (sizeof(T) == 4 && !BATCH)
    vec_rows = aligned16(Prow) && aligned16(Qrow) && aligned16(v.b) && aligned16(v.slack) &&
               aligned16(v.P_out);
  if constexpr (sizeof(T) == 4) {
    static_assert(kFirst == 32 * kBatchF32, "the first batch is one loop trip");
  }
  if (sizeof(T) == 4 && !BATCH && m_sub == kFirst && vec_rows) {
    if constexpr (sizeof(T) == 4 && !BATCH) {
      float pv[kBatch], qv[kBatch], bv[kBatch];
      load_trip<true>(Prow, 0, lane, pv);
      load_trip<true>(Qrow, 0, lane, qv);
      load_trip<true>(v.b, 0, lane, bv);
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        float pa = 0.f, pb = 0.f;
        bool zero = false, nf = false;
        const int cls = classify_phi_nb(pv[k], qv[k], bv[k], tlo2, thi2, pa, pb, zero, nf);
        if (cls == kRowApprox) atomicMax(&bsub[bslot(pbucket(pa) + 2)], __float_as_uint(pb));
        if (cls == kRowApprox && (LONG && v.long_arcs) && bv[k] <= 0.f) {
          ua = fminf(ua, pa);
          ub = fmaxf(ub, pb);
        }
      }
    }
  } else if (m_sub > 0) {
    for (int i0 = 0; i0 < m_sub; i0 += 32 * kBatch) {
      T pv[kBatch], qv[kBatch], bv[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int i = i0 + lane + 32 * k;
        pv[k] = i < m_sub ? Prow[i] : T(0);
        qv[k] = i < m_sub ? Qrow[i] : T(0);
        bv[k] = i < m_sub ? v.b[i] : T(0);
      }
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int i = i0 + lane + 32 * k;
        if (i >= m_sub) continue;
        float pa = 0.f, pb = 0.f;
        bool inf_row = false, nf = false;
        int cls;
        if constexpr (sizeof(T) == 4)
          cls = classify_phi_nb(pv[k], qv[k], bv[k], tlo2, thi2, pa, pb, inf_row, nf);
        else
          cls = classify_phi_d(pv[k], qv[k], bv[k], tlo2, thi2, pa, pb, nf);
        if (cls == kRowApprox) atomicMax(&bsub[bslot(pbucket(pa) + 2)], __float_as_uint(pb));
        if (cls == kRowApprox && (LONG && v.long_arcs) && bv[k] <= T(0)) {
          ua = fminf(ua, pa);
          ub = fmaxf(ub, pb);
        }
      }
    }
  }
  __syncwarp();
  if (m_sub > 0) prefix_max(bsub, lane);
  // the first batch's long arcs: one union (ua, ub) in pseudo-angles
  if ((LONG && v.long_arcs)) {
    ua = warp_min_f(ua);
    ub = warp_max_f(ub);
  }
  __syncwarp();

  // ---- 1b. every row: full bucket maxima, candidates not dominated by an
  //          arc of the first batch ------------------------------------------
  int n_cand = 0;
  float la = INFINITY, lb = -INFINITY;  // every long arc's union (this lane's rows)
  // candidate compaction of one row slot of the batch
  auto push = [&](bool cand, unsigned code, float pb) {
    const unsigned ball = __ballot_sync(kFull, cand);
    const int at = n_cand + __popc(ball & ((1u << lane) - 1u));
    if (cand && at < kCand) {
      candc[at] = code;
      candb[at] = pb;
    }
    n_cand += __popc(ball);
  };
  if constexpr (sizeof(T) == 4) {
    // One batch of 32 kBatch rows in straight-line form (class, bucket test
    // and candidate code by selects, so the rows interleave); FULL batches
    // skip the bounds checks.
    auto batch = [&](int i0, auto full_tag, auto vec_tag, auto union_tag) {
      constexpr bool FULL = decltype(full_tag)::value;
      constexpr bool VEC = decltype(vec_tag)::value;
      constexpr bool UNION = decltype(union_tag)::value;
      static_assert(FULL || !VEC, "vector trips are whole trips");
      float pv[kBatch], qv[kBatch], bv[kBatch];
      if constexpr (FULL) {
        load_trip<VEC>(Prow, i0, lane, pv);
        load_trip<VEC>(Qrow, i0, lane, qv);
        load_trip<VEC>(v.b, i0, lane, bv);
      } else {
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          const int i = i0 + lane + 32 * k;
          pv[k] = i < m ? Prow[i] : 0.f;
          qv[k] = i < m ? Qrow[i] : 0.f;
          bv[k] = i < m ? v.b[i] : 0.f;
        }
      }
      unsigned zmask = 0u;  // rows of the batch with r = 0 (no root)
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int i = slot_row<VEC>(i0, lane, k);
        float pa = 0.f, pb = 0.f;
        bool zero = false;
        int cls = classify_phi_nb(pv[k], qv[k], bv[k], tlo2, thi2, pa, pb, zero, nonfinite);
        if (!FULL) {
          // padding slots past the last row (p = q = 0) are no rows at all
          cls = i < m ? cls : kRowNone;
          zero = zero && i < m;
        }
        zmask |= (zero ? 1u : 0u) << k;
        const int bk = pbucket(pa);
        // bucket maxima sit two slots up: slot bk holds the maxima of the
        // arcs that start at least two buckets earlier
        const bool undominated = !(pb + 2.f * kPhiMargin <= __uint_as_float(bsub[bslot(bk)]));
        const bool approx = cls == kRowApprox;
        bool arc = approx && undominated;
        if constexpr (UNION) {
          // inside the first batch's long-arc union: covered as well
          arc = arc && !(pa >= ua + 2.f * kPhiMargin && pb <= ub - 2.f * kPhiMargin);
          if (approx && bv[k] <= 0.f) {
            la = fminf(la, pa);
            lb = fmaxf(lb, pb);
          }
        }
        // a row dominated by the first batch adds nothing to the full
        // maxima: the first-batch arc that covers it dominates every arc
        // it would dominate
        if (arc) atomicMax(&bfull[bslot(bk + 2)], __float_as_uint(pb));
        push(cls == kRowKeep || arc,
             cls == kRowKeep ? (0x80000000u | (unsigned)i) : (((unsigned)bk << kRowBits) | (unsigned)i),
             pb);
      }
      // rare: r = 0 with b_i < 0 means x violates row i (App. B)
      if (zmask) {
        for (int k = 0; k < kBatch; ++k)
          if ((zmask >> k) & 1u) infeasible |= v.b64[slot_row<VEC>(i0, lane, k)] < 0.0;
      }
    };
    auto rows = [&](auto union_tag) {
      int i0 = 0;
      if constexpr (!BATCH) {
        if (vec_rows)
          for (; i0 + 32 * kBatch <= m; i0 += 32 * kBatch)
            batch(i0, std::true_type{}, std::true_type{}, union_tag);
      }
      for (; i0 + 32 * kBatch <= m; i0 += 32 * kBatch)
        batch(i0, std::true_type{}, std::false_type{}, union_tag);
      if (i0 < m) batch(i0, std::false_type{}, std::false_type{}, union_tag);
    };
    if constexpr (LONG) {
      if (v.long_arcs)
        rows(std::true_type{});
      else
        rows(std::false_type{});
    } else {
      rows(std::false_type{});
    }
  } else {
    for (int i0 = 0; i0 < m; i0 += 32 * kBatch) {
      T pv[kBatch], qv[kBatch], bv[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int i = i0 + lane + 32 * k;
        pv[k] = i < m ? Prow[i] : T(0);
        qv[k] = i < m ? Qrow[i] : T(0);
        bv[k] = i < m ? v.b[i] : T(0);
      }
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int i = i0 + lane + 32 * k;
        bool cand = false;
        unsigned code = 0u;
        float pa = 0.f, pb = 0.f;
        if (i < m) {
          // FP32 classification (rows it cannot decide are kept; r = 0 rows
          // get their infeasibility test from the exact roots)
          const int cls = classify_phi_d(pv[k], qv[k], bv[k], tlo2, thi2, pa, pb, nonfinite);
          if (cls == kRowKeep) {
            cand = true;
            code = 0x80000000u | (unsigned)i;
          } else if (cls == kRowApprox) {
            const int bk = pbucket(pa);
            const bool in_union = (LONG && v.long_arcs) && pa >= ua + 2.f * kPhiMargin &&
                                  pb <= ub - 2.f * kPhiMargin;
            if ((LONG && v.long_arcs) && bv[k] <= T(0)) {
              la = fminf(la, pa);
              lb = fmaxf(lb, pb);
            }
            cand = !in_union && !(pb + 2.f * kPhiMargin <= __uint_as_float(bsub[bslot(bk)]));
            if (cand) atomicMax(&bfull[bslot(bk + 2)], __float_as_uint(pb));
            code = ((unsigned)bk << kRowBits) | (unsigned)i;
          }
        }
        push(cand, code, pb);
      }
    }
  }
  __syncwarp();
  // the union of every long arc, (la, lb); its arcs holding the two extremes
  // start in bucket bkl and end at pseudo-beta lb, and stay
  if ((LONG && v.long_arcs)) {
    la = warp_min_f(la);
    lb = warp_max_f(lb);
  }
  const int bkl = pbucket(la);
  int n_surv = kCap + 1;  // overflow unless the candidates fit
  if (n_cand <= kCand) {
    prefix_max(bfull, lane);
    __syncwarp();
    // ---- 2. survivors: candidates not dominated by any arc ----
    n_surv = 0;
    for (int e0 = 0; e0 < n_cand; e0 += 32) {
      const int e = e0 + lane;
      bool keep = false;
      int row = 0;
      if (e < n_cand) {
        const unsigned code = candc[e];
        row = (int)(code & kRowMask);
        if (code & 0x80000000u) {
          keep = true;
        } else {
          const int bk = (int)((code >> kRowBits) & 0x1FFu);
          // dropped if contained in an arc starting two buckets earlier, or
          // inside the long-arc union (two buckets past its start: more
          // than 2 kPhiMargin in pseudo-angle)
          keep = !(candb[e] + 2.f * kPhiMargin <= __uint_as_float(bfull[bslot(bk)]));
          if constexpr (LONG) keep = keep && !(bk >= bkl + 2 && candb[e] <= lb - 2.f * kPhiMargin);
        }
      }
      const unsigned ball = __ballot_sync(kFull, keep);
      const int at = n_surv + __popc(ball & ((1u << lane) - 1u));
      if (keep && at < kCap) surv[at] = row;
      n_surv += __popc(ball);
    }
  }
  __syncwarp();

  const bool left = n_surv > kCap;
  if (left) {
    // too many arcs for one warp: the CTA-per-chain step takes this chain
    // (listed here when the launch gives a list; else the caller takes it)
    if (lane == 0 && prm.overflow_count) {
      const int at = atomicAdd(prm.overflow_count, 1);
      prm.overflow_list[at] = c;
    }
  } else {
    // ---- 3. exact roots of the survivors, sorted in registers ----
    T key[kPer], val[kPer];
    int tangent = 0, no_root = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int e = lane + 32 * j;
      key[j] = inf;
      val[j] = T(0);
      if (e < n_surv) {
        const int i = surv[e];
        T al, be;
        bool inf_row = false;
        const bool has = roots(Prow[i], Qrow[i], v.b[i], v.b64[i], prm.tangent_thresh, al,
                               be, inf_row, tangent);
        infeasible |= inf_row;
        if (has) {
          key[j] = al;
          val[j] = be;
        } else {
          ++no_root;
        }
      }
    }
    // bitonic sort of the smallest power-of-two size that holds the arcs
    warp_sort_arcs<T>(key, val, n_surv, lane);
    // warp-wide counts
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      no_root += __shfl_xor_sync(kFull, no_root, o);
      tangent += __shfl_xor_sync(kFull, tangent, o);
    }
    const int n_roots = n_surv - no_root;
    my_sort_keys = n_roots;

    // ---- Alg. 3 sweep and theta ~ U(I_act) (inverse CDF) ----
    const double u = prm.U ? prm.U[c] : theta_uniform(prm.seed, v.chain, v.t, v.problem);
    double* pieces_row = prm.pieces_out ? prm.pieces_out + (size_t)c * prm.max_pieces * 2 : nullptr;
    const T theta = warp_sweep_theta<T>(key, val, n_roots, (T)prm.trim_eps, u, lane, pieces_row,
                                        prm.max_pieces,
                                        prm.npieces_out ? prm.npieces_out + c : nullptr);

    // ---- 4. move: p' for every row, FP64 recheck of rows near their bound ----
    T sn, cs;
    if constexpr (sizeof(T) == 8) {
      sincos((double)theta, reinterpret_cast<double*>(&sn), reinterpret_cast<double*>(&cs));
    } else {
      sincosf((float)theta, reinterpret_cast<float*>(&sn), reinterpret_cast<float*>(&cs));
    }
    const T* xrow = v.X;
    const T* nurow = v.NU;
    T* prow_out = v.P_out;
    bool bad = nonfinite || !isfinite(theta);
    bool violated = false;
    int rechecks = 0;
    double maxres = -INFINITY;
    // one loop trip of rows: p' for each, rows near their bound rechecked
    auto move_trip = [&](int i0, auto full_tag, auto vec_tag) {
      constexpr bool FULL = decltype(full_tag)::value;
      constexpr bool VEC = decltype(vec_tag)::value;
      static_assert(FULL || !VEC, "vector trips are whole trips");
      T pv[kBatch], qv[kBatch], sv[kBatch];
      if constexpr (sizeof(T) == 4 && FULL) {
        load_trip<VEC>(Prow, i0, lane, pv);
        load_trip<VEC>(Qrow, i0, lane, qv);
        load_trip<VEC>(v.slack, i0, lane, sv);  // float chains always carry the thresholds
      } else {
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          const int i = i0 + lane + 32 * k;
          pv[k] = i < m ? Prow[i] : T(0);
          qv[k] = i < m ? Qrow[i] : T(0);
          if constexpr (sizeof(T) == 4) {
            sv[k] = i < m ? v.slack[i] : T(0);
          } else {
            sv[k] = i < m ? (v.slack ? v.slack[i] : (T)(v.b64[i] - prm.margin * v.anorm[i]))
                          : T(0);
          }
        }
      }
      unsigned flags = 0u;
      T pn[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int i = slot_row<VEC>(i0, lane, k);
        pn[k] = pv[k] * cs + qv[k] * sn;
        if (FULL || i < m) {
          if constexpr (sizeof(T) == 8) {
            // pn > sv on the doubles' bits mapped to ordered integers (no
            // FP64 instruction); a NaN pn also marks the chain bad, which
            // rejects the move
            if (ordered_bits(pn[k]) > ordered_bits(sv[k])) flags |= 1u << k;
          } else {
            if (!(pn[k] <= sv[k])) flags |= 1u << k;
          }
        }
      }
      if constexpr (sizeof(T) == 4 && FULL) {
        store_trip<VEC>(prow_out, i0, lane, pn);
      } else {
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          const int i = i0 + lane + 32 * k;
          if (i < m) prow_out[i] = pn[k];
        }
      }
      // rows near their bound are rare: one vote per batch, then per slot
      if (__any_sync(kFull, flags != 0u)) {
        for (int k = 0; k < kBatch; ++k) {
          unsigned ball = __ballot_sync(kFull, (flags >> k) & 1u);
          rechecks += __popc(ball);
          while (ball) {
            const int src = __ffs(ball) - 1;
            ball &= ball - 1;
            const int row = slot_row<VEC>(i0, src, k);
            const double* arow = v.A64 + (size_t)row * d;
            double acc = 0.0;
            for (int jj = lane; jj < d; jj += 32) {
              const T xn = xrow[jj] * cs + nurow[jj] * sn;
              acc = fma(arow[jj], (double)xn, acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            const double res = acc - v.b64[row];
            maxres = fmax(maxres, res);
            violated |= res > 0.0;
          }
        }
      }
    };
    {
      int i0 = 0;
      if constexpr (sizeof(T) == 4) {
        if constexpr (!BATCH) {
          if (vec_rows)
            for (; i0 + 32 * kBatch <= m; i0 += 32 * kBatch)
              move_trip(i0, std::true_type{}, std::true_type{});
        }
        {
          for (; i0 + 32 * kBatch <= m; i0 += 32 * kBatch)
            move_trip(i0, std::true_type{}, std::false_type{});
        }
      }
      for (; i0 < m; i0 += 32 * kBatch) move_trip(i0, std::false_type{}, std::false_type{});
    }
    // x' is finite whenever theta, x and nu are (x_0 passes an FP64 check)
    const bool reject = __any_sync(kFull, violated || bad);
    bad = __any_sync(kFull, bad);
    T* xout = v.X_out;
    T* srow = v.S;
    if (!reject) {
      int j0 = 0;
      if constexpr (sizeof(T) == 4 && !BATCH) {
        // whole trips of 16-byte aligned rows: 128-bit loads and stores
        if (aligned16(xrow) && aligned16(nurow) && aligned16(xout) &&
            (srow == nullptr || aligned16(srow))) {
          for (; j0 + 32 * kBatch <= d; j0 += 32 * kBatch) {
            float xv[kBatch], nv[kBatch], xn[kBatch];
            load_trip<true>(xrow, j0, lane, xv);
            load_trip<true>(nurow, j0, lane, nv);
#pragma unroll
            for (int k = 0; k < kBatch; ++k) xn[k] = xv[k] * cs + nv[k] * sn;
            store_trip<true>(xout, j0, lane, xn);
            if (srow) store_trip<true>(srow, j0, lane, xn);
          }
        }
      }
      for (; j0 < d; j0 += 32 * kBatch) {
        T xv[kBatch], nv[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          const int jj = j0 + lane + 32 * k;
          xv[k] = jj < d ? xrow[jj] : T(0);
          nv[k] = jj < d ? nurow[jj] : T(0);
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          const int jj = j0 + lane + 32 * k;
          if (jj < d) {
            const T xn = xv[k] * cs + nv[k] * sn;
            xout[jj] = xn;
            if (srow) srow[jj] = xn;
          }
        }
      }
    } else {
      // Sec. 3.3: stay at x_t; p is restored
      for (int i = lane; i < m; i += 32) prow_out[i] = Prow[i];
      for (int jj = lane; jj < d; jj += 32) {
        if (prm.X_out != prm.X) xout[jj] = xrow[jj];
        if (srow) srow[jj] = xrow[jj];
      }
    }
    if (lane == 0) {
      if (prm.theta_out) prm.theta_out[c] = (double)theta;
      if (prm.rejected_out) prm.rejected_out[c] = reject ? 1 : 0;
      if (reject && !bad) atomicAdd(&prm.stats->rejections, 1ull);
      if (bad) {
        atomicAdd(&prm.stats->numeric_errors, 1ull);
        atomicOr(prm.status, kStatusNumeric);
      }
      if (tangent) atomicAdd(&prm.stats->tangent_fp64, (unsigned long long)tangent);
      if (rechecks) atomicAdd(&prm.stats->rechecks, (unsigned long long)rechecks);
    }
    if (rechecks && maxres > -INFINITY)
      atomicMax(&prm.stats->max_residual_bits, enc_ordered(maxres));
  }
  if (__any_sync(kFull, infeasible) && lane == 0) atomicOr(prm.status, kStatusInfeasible);
  return left ? -1 : my_sort_keys;
}

}  // namespace
}  // namespace ess
