// k_chain_stream.cu -- one elliptical-slice step per chain, one warp per chain,
// the chain's p and q rows streamed through shared memory in chunks.
//
// The same map as chain_warp_kernel (Alg. 1 body: App. B roots, the
// domination prune of contained arcs, Alg. 3 sort and cumulative-max sweep,
// inverse-CDF theta, move and the Sec. 3.3 safeguard), organised so that the
// warp neither waits on HBM nor spends instructions on bookkeeping:
//   * each warp takes chains from a work counter; it streams the p and q rows
//     of its chain through a ring of kStages chunks of kRows rows in shared
//     memory (1-D bulk copies completing on per-stage mbarriers), so a chunk's
//     rows are on chip while the previous one is classified; the move streams
//     them again (from L2) the same way;
//   * a row costs one 128-bit shared load each for p and q (four rows per
//     lane and trip) and a lean classification (classify_lean); the bucket
//     maxima are stored with the domination margin already subtracted, and a
//     candidate row costs one bit in a register mask instead of a list entry;
//   * after the pass, the candidates (a few dozen of m rows) are classified
//     again from global memory and tested against the full maxima; the <= 128
//     survivors get exact roots and the register sort of the warp kernel.
// No block-wide barrier is used; warps of a CTA are independent.  Chains with
// more than 128 surviving arcs are listed for the CTA-per-chain kernel.
// Float chains of one problem (no batch descriptors) with m and d multiples
// of 4 (16-byte rows), m <= kStreamMaxM.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "chain_math.cuh"
#include "chain_warp_ops.cuh"
#include "ess_kernels.cuh"

namespace ess {
namespace {

using namespace chainmath;
using namespace warpops;

#ifndef ESS_STREAM_WARPS
#define ESS_STREAM_WARPS 4
#endif
#ifndef ESS_STREAM_ROWS
#define ESS_STREAM_ROWS 256
#endif
#ifndef ESS_STREAM_STAGES
#define ESS_STREAM_STAGES 3
#endif
#ifndef ESS_STREAM_MINBLOCKS
#define ESS_STREAM_MINBLOCKS 5
#endif
constexpr int kSW = ESS_STREAM_WARPS;     // warps (chains in flight) per CTA
constexpr int kRows = ESS_STREAM_ROWS;    // rows per staged chunk
constexpr int kStages = ESS_STREAM_STAGES;  // chunks in flight per warp
constexpr int kTrips = kRows / 128;      // 4 rows per lane and trip
constexpr int kStreamMaxM = 4096;
constexpr int kMaxD = 1 << 20;
constexpr unsigned long long kStreamWaitNs = 2000000000ull;  // 2 s per wait
static_assert(kFirst <= kRows, "the first batch lies in the first chunk");
static_assert(kRows % 128 == 0, "four rows per lane and trip");

// ---- PTX wrappers (mbarrier and 1-D bulk copies) --------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity, at most kStreamWaitNs; false if
// it gave up.
__device__ __noinline__ bool bar_wait_slow(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (bar_test(bar, parity)) return true;
    if (now_ns() - t0 > kStreamWaitNs) return false;
  }
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  return bar_test(bar, parity) || bar_wait_slow(bar, parity);
}

// Orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned), completing as transaction bytes on bar.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<uint64_t>(p)));
}

// x' = x cos + nu sin with one explicit rounding order, so that the FP64
// recheck of a row sees exactly the x' that is written.
__device__ __forceinline__ float move1(float x, float nu, float cs, float sn) {
  return __fmaf_rn(x, cs, __fmul_rn(nu, sn));
}

// Per-warp shared memory.
struct alignas(16) WarpSmem {
  float stage[kStages][2][kRows];   // chunk rows: p, q (or x, nu)
  unsigned bsub[kWBP];              // first-batch maxima (floats after the prefix)
  unsigned bfull[kWBP];             // full maxima (floats after the prefix)
  int surv[kCap];
  unsigned long long bar[kStages];
};

// Prefix max of the bucket maxima, then the domination margin subtracted: the
// test of an arc is then pb <= slot value (floats; empty prefixes go negative).
__device__ __forceinline__ void prefix_max_margin(unsigned* b, int lane) {
  prefix_max(b, lane);
  __syncwarp();
  for (int k = lane; k < kWBP; k += 32)
    b[k] = __float_as_uint(__uint_as_float(b[k]) - 2.f * kPhiMargin);
  __syncwarp();
}

__global__ void __launch_bounds__(kSW * 32, ESS_STREAM_MINBLOCKS) chain_stream_kernel(ChainParams<float> prm) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& W = reinterpret_cast<WarpSmem*>(smem_raw)[warp];
  const int m = prm.m, d = prm.d, n = prm.n_chains;
  const int nch = (m + kRows - 1) / kRows;   // chunks of p and q rows
  const int ntot = nch + (d + kRows - 1) / kRows;  // ... then of x and nu
  const unsigned step_t = prm.t + (prm.t_dev ? *prm.t_dev : 0u);
  const float inf = INFINITY;
  // squared thresholds of the float classification (1e-6 relative slack)
  const float tlo_s = (float)((1.0 - prm.tangent_thresh) * 0.999999);
  const float thi_s = (float)((1.0 + prm.tangent_thresh) * 1.000001);
  const float tlo2 = tlo_s * tlo_s, thi2 = thi_s * thi_s;
  const float4* b4g = reinterpret_cast<const float4*>(prm.b);
  const float4* slack4 = reinterpret_cast<const float4*>(prm.slack);
  const float* bsubf = reinterpret_cast<const float*>(W.bsub);
  const float* bfullf = reinterpret_cast<const float*>(W.bfull);

  if (lane == 0) {
    for (int s = 0; s < kStages; ++s) bar_init(smem_addr(&W.bar[s]));
    bar_init_fence();
  }
  __syncwarp();
  unsigned phase = 0u;    // bit s: parity of the next wait on stage s
  unsigned pending = 0u;  // bit s: a load into stage s not yet waited for
  unsigned long long sort_keys = 0ull;

  // chunk kk of a chain's stream into stage s: for kk < nch the rows
  // [kk kRows, min(m, (kk + 1) kRows)) of p and q, beyond that the elements
  // [(kk - nch) kRows, ...) of x and nu
  auto issue = [&](const float* Pg, const float* Qg, const float* Xg, const float* Ng, int kk,
                   int s) {
    pending |= 1u << s;
    if (lane == 0) {
      const bool rows = kk < nch;
      const int e0 = (rows ? kk : kk - nch) * kRows;
      const uint32_t bytes = 4u * (uint32_t)min(kRows, (rows ? m : d) - e0);
      const uint32_t bar = smem_addr(&W.bar[s]);
      fence_async_smem();
      bar_expect(bar, 2u * bytes);
      bulk_load(smem_addr(W.stage[s][0]), (rows ? Pg : Xg) + e0, bytes, bar);
      bulk_load(smem_addr(W.stage[s][1]), (rows ? Qg : Ng) + e0, bytes, bar);
    }
  };
  // waits for stage s; on a time-out drains the other loads in flight
  auto wait = [&](int s) -> bool {
    const bool ok = __all_sync(kFull, bar_wait(smem_addr(&W.bar[s]), (phase >> s) & 1u));
    phase ^= 1u << s;
    pending &= ~(1u << s);
    if (!ok) {
      if (lane == 0) atomicOr(prm.status, kStatusTimeout);
      for (int t = 0; t < kStages; ++t)
        if ((pending >> t) & 1u) (void)bar_wait(smem_addr(&W.bar[t]), (phase >> t) & 1u);
      pending = 0u;
    }
    return ok;
  };

  for (;;) {
    int c = 0;
    if (lane == 0) c = atomicAdd(prm.work_counter, 1);
    c = __shfl_sync(kFull, c, 0);
    if (c >= n) break;
    const float* Pg = prm.P_in + (size_t)c * prm.ldp;
    const float* Qg = prm.Q + (size_t)c * prm.ldp;
    const float* Xg = prm.X + (size_t)c * prm.ldx;
    const float* Ng = prm.NU + (size_t)c * prm.ldx;
    for (int k = 0; k < min(kStages, nch); ++k) issue(Pg, Qg, Xg, Ng, k, k);
    // the theta uniform does not depend on the rows: draw it while they load
    const double u =
        prm.U ? prm.U[c] : theta_uniform(prm.seed, prm.chain0 + (unsigned)c, step_t, prm.problem);
    for (int k = lane; k < 2 * kWBP / 4; k += 32)
      reinterpret_cast<uint4*>(W.bsub)[k] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    if (!wait(0)) return;

    // ---- 1a. the first batch (rows of chunk 0) builds bucket maxima of beta ----
    // (with m <= kCand there is no first batch: every arc is a candidate)
    float nfacc = 0.f;
    const int m_sub = m > kCand ? min(m, kFirst) : 0;
#pragma unroll
    for (int t = 0; t < kTrips; ++t) {
      const int r0 = 128 * t + 4 * lane;
      if (r0 < m_sub) {
        const float4 p4 = *reinterpret_cast<const float4*>(&W.stage[0][0][r0]);
        const float4 q4 = *reinterpret_cast<const float4*>(&W.stage[0][1][r0]);
        const float4 bb = __ldg(b4g + (r0 >> 2));
        const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
        const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
        const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float pa, pb;
          if (classify_lean(pv[r], qv[r], bv[r], tlo2, thi2, pa, pb, nfacc) == kRowApprox)
            atomicMax(&W.bsub[bslot(pbucket(pa) + 2)], __float_as_uint(pb));
        }
      }
    }
    __syncwarp();
    prefix_max_margin(W.bsub, lane);

    // ---- 1b. every row: full bucket maxima; candidates (not dominated by an
    //          arc of the first batch) as bits of per-lane masks -----------------
    // bit 4 tg + r of (cm1:cm0): row 128 tg + 4 lane + r (trip tg < m / 128 <= 32)
    unsigned long long cm0 = 0ull, cm1 = 0ull;
    bool ok = true;
    for (int k = 0; k < nch; ++k) {
      const int s = k % kStages;
      if (k > 0 && !(ok = wait(s))) break;
#pragma unroll
      for (int t = 0; t < kTrips; ++t) {
        const int rl = 128 * t + 4 * lane;   // row within the chunk
        const int r0 = k * kRows + rl;
        unsigned bits = 0u;
        if (r0 < m) {
          const float4 p4 = *reinterpret_cast<const float4*>(&W.stage[s][0][rl]);
          const float4 q4 = *reinterpret_cast<const float4*>(&W.stage[s][1][rl]);
          const float4 bb = __ldg(b4g + (r0 >> 2));
          const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
          const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
          const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            float pa, pb;
            const int cls = classify_lean(pv[r], qv[r], bv[r], tlo2, thi2, pa, pb, nfacc);
            const int bk = pbucket(pa);
            // slot bk holds the maxima of the arcs that start at least two
            // buckets earlier, less the margin
            const bool undominated = !(pb <= bsubf[bslot(bk)]);
            const bool approx = cls == kRowApprox;
            if (approx && undominated) atomicMax(&W.bfull[bslot(bk + 2)], __float_as_uint(pb));
            bits |= (cls == kRowKeep || (approx && undominated) ? 1u : 0u) << r;
          }
        }
        const int tg = k * kTrips + t;       // trip index: bits 4 tg .. 4 tg + 3
        const unsigned long long wide = (unsigned long long)bits << (4 * (tg & 15));
        if (tg < 16) cm0 |= wide;
        else cm1 |= wide;
      }
      __syncwarp();
      if (k + kStages < nch) issue(Pg, Qg, Xg, Ng, k + kStages, s);
    }
    if (!ok) return;
    const bool bad_pq = __any_sync(kFull, nfacc != nfacc);
    // the move streams the rows (and then x, nu) again: its first chunks load
    // during the rest
    for (int k = 0; k < min(kStages, ntot); ++k) issue(Pg, Qg, Xg, Ng, k, k);
    // the candidates' p and q are read again below: bring them to L1 now
    {
      unsigned long long a0 = cm0, a1 = cm1;
      while (a0 | a1) {
        int bit;
        if (a0) {
          bit = __ffsll((long long)a0) - 1;
          a0 &= a0 - 1ull;
        } else {
          bit = 64 + __ffsll((long long)a1) - 1;
          a1 &= a1 - 1ull;
        }
        const int row = 128 * (bit >> 2) + 4 * lane + (bit & 3);
        prefetch_l1(Pg + row);
        prefetch_l1(Qg + row);
      }
    }
    __syncwarp();
    prefix_max_margin(W.bfull, lane);

    // ---- 2. survivors: the candidates, classified again, not dominated by any arc
    int n_surv = 0;
    bool infeasible = false;
    for (;;) {
      const bool mine = (cm0 | cm1) != 0ull;
      if (!__any_sync(kFull, mine)) break;
      bool keep = false;
      int row = 0;
      if (mine) {
        int bit;
        if (cm0) {
          bit = __ffsll((long long)cm0) - 1;
          cm0 &= cm0 - 1ull;
        } else {
          bit = 64 + __ffsll((long long)cm1) - 1;
          cm1 &= cm1 - 1ull;
        }
        const int tg = bit >> 2;
        row = 128 * tg + 4 * lane + (bit & 3);
        float pa, pb, nf = 0.f;
        const int cls = classify_lean(Pg[row], Qg[row], __ldg(prm.b + row), tlo2, thi2, pa, pb, nf);
        keep = cls == kRowKeep ||
               (cls == kRowApprox && !(pb <= bfullf[bslot(pbucket(pa))]));
      }
      const unsigned ball = __ballot_sync(kFull, keep);
      const int at = n_surv + __popc(ball & ((1u << lane) - 1u));
      if (keep && at < kCap) W.surv[at] = row;
      n_surv += __popc(ball);
    }
    __syncwarp();

    if (n_surv > kCap) {
      // too many arcs for one warp: the CTA-per-chain kernel takes this chain
      if (lane == 0) {
        const int at = atomicAdd(prm.overflow_count, 1);
        prm.overflow_list[at] = c;
      }
      for (int k = 0; k < min(kStages, ntot); ++k)
        if (!wait(k)) return;
      __syncwarp();
      continue;
    }

    // ---- 3. exact roots of the survivors, sorted in registers; Alg. 3; theta ----
    float key[kPer], val[kPer];
    int tangent = 0, no_root = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int e = lane + 32 * j;
      key[j] = inf;
      val[j] = 0.f;
      if (e < n_surv) {
        const int i = W.surv[e];
        float al = 0.f, be = 0.f;
        bool inf_row = false;
        if (roots(Pg[i], Qg[i], __ldg(prm.b + i), prm.b64[i], prm.tangent_thresh, al, be, inf_row,
                  tangent)) {
          key[j] = al;
          val[j] = be;
        } else {
          ++no_root;
        }
        infeasible |= inf_row;
      }
    }
    warp_sort_arcs<float>(key, val, n_surv, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      no_root += __shfl_xor_sync(kFull, no_root, o);
      tangent += __shfl_xor_sync(kFull, tangent, o);
    }
    const int n_roots = n_surv - no_root;
    sort_keys += (unsigned long long)n_roots;
    double* pieces_row = prm.pieces_out ? prm.pieces_out + (size_t)c * prm.max_pieces * 2 : nullptr;
    const float theta = warp_sweep_theta<float>(key, val, n_roots, (float)prm.trim_eps, u, lane,
                                                pieces_row, prm.max_pieces,
                                                prm.npieces_out ? prm.npieces_out + c : nullptr);

    // ---- 4. move: p' for every row, FP64 recheck of the rows near their bound;
    //         then x' (or, on rejection, x and p restored: Sec. 3.3).  The rows of
    //         p and q, then x and nu, are streamed again through the ring. -------
    float sn, cs;
    sincosf(theta, &sn, &cs);
    const bool bad = bad_pq || !isfinite(theta);
    float* pout = prm.P_out + (size_t)c * prm.ldp;
    float* xout = prm.X_out + (size_t)c * prm.ldx;
    float* srow = prm.samples ? prm.samples + (size_t)c * prm.sample_stride : nullptr;
    const bool svec = srow != nullptr && (reinterpret_cast<uintptr_t>(srow) & 15u) == 0u;
    const bool x_inplace = prm.X_out == prm.X;
    bool violated = false, reject = false;
    int rechecks = 0;
    double maxres = -INFINITY;
    for (int kk = 0; kk < ntot; ++kk) {
      const int s = kk % kStages;
      if (!(ok = wait(s))) break;
      if (kk < nch) {
        unsigned fl = 0u;
#pragma unroll
        for (int t = 0; t < kTrips; ++t) {
          const int rl = 128 * t + 4 * lane;
          const int r0 = kk * kRows + rl;
          if (r0 < m) {
            const float4 p4 = *reinterpret_cast<const float4*>(&W.stage[s][0][rl]);
            const float4 q4 = *reinterpret_cast<const float4*>(&W.stage[s][1][rl]);
            const float4 s4 = __ldg(slack4 + (r0 >> 2));
            float4 o;
            o.x = __fmaf_rn(p4.x, cs, __fmul_rn(q4.x, sn));
            o.y = __fmaf_rn(p4.y, cs, __fmul_rn(q4.y, sn));
            o.z = __fmaf_rn(p4.z, cs, __fmul_rn(q4.z, sn));
            o.w = __fmaf_rn(p4.w, cs, __fmul_rn(q4.w, sn));
            *reinterpret_cast<float4*>(pout + r0) = o;
            fl |= ((!(o.x <= s4.x) ? 1u : 0u) | (!(o.y <= s4.y) ? 2u : 0u) |
                   (!(o.z <= s4.z) ? 4u : 0u) | (!(o.w <= s4.w) ? 8u : 0u)) << (4 * t);
          }
        }
        __syncwarp();
        if (kk + kStages < ntot) issue(Pg, Qg, Xg, Ng, kk + kStages, s);
        // rows near their bound are rare: one vote, then row by row
        if (__any_sync(kFull, fl != 0u)) {
          for (int bit = 0; bit < 4 * kTrips; ++bit) {
            unsigned ball = __ballot_sync(kFull, (fl >> bit) & 1u);
            rechecks += __popc(ball);
            while (ball) {
              const int src = __ffs(ball) - 1;
              ball &= ball - 1;
              const int row = kk * kRows + 128 * (bit >> 2) + 4 * src + (bit & 3);
              const double* arow = prm.A64 + (size_t)row * d;
              double acc = 0.0;
              for (int j = lane; j < d; j += 32)
                acc = fma(arow[j], (double)move1(Xg[j], Ng[j], cs, sn), acc);
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
              const double res = acc - prm.b64[row];
              maxres = fmax(maxres, res);
              violated |= res > 0.0;
            }
          }
        }
      } else {
        if (kk == nch) reject = __any_sync(kFull, violated || bad);
        const int e0 = (kk - nch) * kRows;
#pragma unroll
        for (int t = 0; t < kTrips; ++t) {
          const int el = 128 * t + 4 * lane;
          const int j0 = e0 + el;
          if (j0 < d) {
            const float4 x4 = *reinterpret_cast<const float4*>(&W.stage[s][0][el]);
            const float4 v4 = *reinterpret_cast<const float4*>(&W.stage[s][1][el]);
            float4 o = x4;
            if (!reject) {
              o.x = move1(x4.x, v4.x, cs, sn);
              o.y = move1(x4.y, v4.y, cs, sn);
              o.z = move1(x4.z, v4.z, cs, sn);
              o.w = move1(x4.w, v4.w, cs, sn);
            }
            if (!reject || !x_inplace) *reinterpret_cast<float4*>(xout + j0) = o;
            if (svec) {
              *reinterpret_cast<float4*>(srow + j0) = o;
            } else if (srow) {
              srow[j0] = o.x;
              srow[j0 + 1] = o.y;
              srow[j0 + 2] = o.z;
              srow[j0 + 3] = o.w;
            }
          }
        }
        __syncwarp();
        if (kk + kStages < ntot) issue(Pg, Qg, Xg, Ng, kk + kStages, s);
      }
    }
    if (!ok) return;
    if (reject) {
      // Sec. 3.3: stay at x_t; p is restored
      for (int g = lane; g < (m >> 2); g += 32)
        reinterpret_cast<float4*>(pout)[g] = reinterpret_cast<const float4*>(Pg)[g];
    }
    const bool inf_any = __any_sync(kFull, infeasible);
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
      if (rechecks && maxres > -INFINITY)
        atomicMax(&prm.stats->max_residual_bits, enc_ordered(maxres));
      if (inf_any) atomicOr(prm.status, kStatusInfeasible);
    }
    __syncwarp();
  }
  if (lane == 0 && sort_keys) atomicAdd(&prm.stats->sort_keys, sort_keys);
}

}  // namespace

bool chain_stream_aligned(const ChainParams<float>& p) {
  auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0u; };
  return (p.ldp & 3) == 0 && (p.ldx & 3) == 0 && a16(p.P_in) && a16(p.P_out) && a16(p.Q) &&
         a16(p.X) && a16(p.X_out) && a16(p.NU) && a16(p.b) && a16(p.slack);
}

bool chain_stream_supported(int m, int d) {
  return m >= 4 && d >= 4 && (m & 3) == 0 && (d & 3) == 0 && m <= kStreamMaxM && d <= kMaxD;
}

cudaError_t launch_chain_step_stream(const ChainParams<float>& p, cudaStream_t s) {
  if (p.n_chains <= 0) return cudaSuccess;
  if (p.desc || !chain_stream_supported(p.m, p.d) || !p.work_counter || !p.overflow_list ||
      !p.overflow_count || p.P_out == p.P_in || !p.slack || !chain_stream_aligned(p))
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(WarpSmem) * kSW;
  cudaError_t e = cudaFuncSetAttribute(chain_stream_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain_stream_kernel, kSW * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min((p.n_chains + kSW - 1) / kSW, per_sm * sms);
  chain_stream_kernel<<<grid, kSW * 32, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ess
