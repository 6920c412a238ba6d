// k_chain_wide.cu -- one elliptical-slice step per chain, one CTA per chain,
// for any number of rows m: the rows are streamed, never held all at once.
//
// The map is the one of chain_step_kernel (App. B roots with the Sec. 3.2
// edge cases, Alg. 3 sort and cumulative-max sweep, inverse-CDF theta, move
// and the Sec. 3.3 safeguard); only the storage differs, so that m is bounded
// by memory instead of by one CTA's registers and shared memory:
//   1. a pass over the rows: each row's arc is placed by the pseudo-angles of
//      its two roots (a monotone stand-in for the angle, without
//      trigonometry) in one of 512 buckets, for the domination prune of the
//      warp kernel (an arc that lies inside an arc starting two buckets
//      earlier changes no piece): a first batch of rows gives bucket maxima,
//      the later rows that no first-batch arc covers become candidates;
//   2. the first batch and the candidates (or, when the candidates overflow
//      their list, all rows again) are tested against the full maxima, and
//      every row that is not dominated gets its exact roots,
//      merged into its alpha bucket (NB buckets of width 2 pi / NB): an arc
//      that reaches the end of its bucket contains that point, so all such
//      arcs of a bucket overlap and their union is [min alpha, max beta]; a
//      shorter arc (near tangency) goes to a short list, in shared memory and
//      past its capacity in the CTA's global scratch slot;
//   3. the bucket intervals and the short arcs are sorted by alpha -- in
//      registers and shared memory when they fit in kWSlots, else by a merge
//      sort in the scratch slot -- and Alg. 3 runs over them in chunks of
//      kWSlots arcs, carrying the cumulative max gamma and the summed piece
//      length from chunk to chunk: one sweep gives the total length of I_act,
//      a second finds the piece that the inverse CDF lands in;
//   4. a third pass: p' = p cos + q sin written to P_out, rows within the
//      margin of their bound collected and their residual recomputed in FP64
//      against x' (in batches, one warp per row); a violation rejects the move
//      and p is copied back from P_in.
// The union of the arcs -- hence I_act, its piece endpoints and theta -- is
// the one Alg. 3 gives on the arcs themselves.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "chain_block_ops.cuh"
#include "chain_math.cuh"
#include "chain_warp_ops.cuh"
#include "ess_kernels.cuh"

namespace ess {
namespace {

using namespace chainmath;
using namespace blockops;
using warpops::bslot;
using warpops::kPhiMargin;
using warpops::kWBP;
using warpops::pbucket;
using warpops::prefix_max;

#ifndef ESS_WIDE_THREADS
#define ESS_WIDE_THREADS 512
#endif
#ifndef ESS_WIDE_MINBLOCKS
#define ESS_WIDE_MINBLOCKS 2
#endif
#ifndef ESS_WIDE_ROWS
#define ESS_WIDE_ROWS 2
#endif
constexpr int kWT = ESS_WIDE_THREADS;          // threads per CTA
constexpr int kWW = kWT / 32;                  // warps per CTA
constexpr int kWSlots = 4096;                  // arcs sorted at once in shared memory
constexpr int kWItems = kWSlots / kWT;         // sorted arcs per thread
constexpr int kWPad = kWSlots + kWSlots / 32;  // padded shared arrays
constexpr int kWU = ESS_WIDE_ROWS;             // rows per thread per pass trip
constexpr int kWTrip = kWT * kWU;              // rows per pass trip
constexpr int kWFlag = 2 * kWTrip;             // flagged rows held before a recheck batch
constexpr int kWFirst = 2048;                  // rows of the prune's first batch
// Candidate rows held after the first batch: 2048 (float chains), 1024
// (double chains: two CTAs per SM at d = 1000).
template <typename T>
constexpr int wide_cand() { return sizeof(T) == 8 ? 1024 : 2048; }
// Candidate codes: a kept row is 0x80000000 | i; an arc is bucket << kWRowBits
// | i (buckets below 512 in bits 22 .. 30), so rows up to 2^22.
constexpr int kWRowBits = 22;
constexpr unsigned kWRowMask = (1u << kWRowBits) - 1u;

// Merge buckets: 2048 for float chains, 1024 for double chains (whose wider
// entries would otherwise cost a CTA per SM at d = 1000).
template <typename T>
constexpr int wide_buckets() { return sizeof(T) == 8 ? 1024 : 2048; }
// Short arcs kept in shared memory: the rest of the kWSlots sort slots.
template <typename T>
constexpr int wide_short_smem() { return kWSlots - wide_buckets<T>(); }
static_assert(wide_buckets<float>() % kWT == 0 && wide_buckets<double>() % kWT == 0,
              "whole buckets per thread");

template <typename T>
using BitsOf = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned>::type;

// Non-negative floating-point values compare like their bit patterns; -0
// becomes +0.
template <typename T>
__device__ __forceinline__ BitsOf<T> abs_bits(T v) {
  if constexpr (sizeof(T) == 8)
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  else
    return __float_as_uint(v) & 0x7FFFFFFFu;
}
template <typename T>
__device__ __forceinline__ T from_bits(BitsOf<T> b) {
  if constexpr (sizeof(T) == 8) return __longlong_as_double((long long)b);
  else return __uint_as_float(b);
}
template <typename T>
__device__ __forceinline__ BitsOf<T> empty_bits() {  // +inf: an empty bucket's min alpha
  if constexpr (sizeof(T) == 8) return 0x7FF0000000000000ull;
  else return 0x7F800000u;
}

// Alg. 3 over one chunk of sorted arcs held in registers (blocked: thread t
// holds positions gbase + t kWItems + i, valid below n).  Piece k is
// [gamma_(k-1) + eps, alpha_k - eps], piece 0 is [0, alpha_0 - eps] (its left
// end is the glued point 0, never trimmed), gamma_k the cumulative max of
// beta.  gamma and len carry the max beta and the summed piece length of all
// earlier chunks.  With locate, the thread's candidate becomes its last piece
// of positive length whose cumulative start is <= s (theta then lies in it),
// and the positive pieces are written from position *np on (up to max_pieces).
// Contains __syncthreads (call uniformly).
template <typename T>
__device__ void alg3_chunk(const T (&key)[kWItems], const T (&val)[kWItems], int gbase, int n,
                           T eps, T& gamma, T& len, bool locate, T s, int& cand, T& cand_theta,
                           T* s_ttmp, int* s_itmp, double* pieces, int max_pieces, int& np) {
  const int base = gbase + threadIdx.x * kWItems;
  T run = T(0);
#pragma unroll
  for (int i = 0; i < kWItems; ++i)
    if (base + i < n) run = val[i] > run ? val[i] : run;
  T gchunk;
  const T gex = block_exclusive_scan<kWT>(run, T(0), OpMax(), s_ttmp, gchunk);
  const T gstart = gamma > gex ? gamma : gex;  // gamma before this thread's first arc
  T my_len = T(0);
  int my_np = 0;
  {
    T g = gstart;
#pragma unroll
    for (int i = 0; i < kWItems; ++i) {
      const int k = base + i;
      if (k < n) {
        const T lo = k == 0 ? T(0) : g + eps;
        const T hi = key[i] - eps;
        const T l = hi > lo ? hi - lo : T(0);
        my_len += l;
        my_np += l > T(0) ? 1 : 0;
        g = val[i] > g ? val[i] : g;
      }
    }
  }
  T chunk_len;
  const T lpre = block_exclusive_scan<kWT>(my_len, T(0), OpAdd(), s_ttmp, chunk_len);
  if (locate) {
    T acc = len + lpre;
    T g = gstart;
#pragma unroll
    for (int i = 0; i < kWItems; ++i) {
      const int k = base + i;
      if (k < n) {
        const T lo = k == 0 ? T(0) : g + eps;
        const T hi = key[i] - eps;
        const T l = hi > lo ? hi - lo : T(0);
        if (l > T(0) && acc <= s) {
          cand = k;
          const T th = lo + (s - acc);
          cand_theta = th < hi ? th : hi;
        }
        acc += l;
        g = val[i] > g ? val[i] : g;
      }
    }
    if (pieces != nullptr) {
      int np_chunk;
      int at = np + block_exclusive_scan<kWT>(my_np, 0, OpAdd(), s_itmp, np_chunk);
      T g2 = gstart;
#pragma unroll
      for (int i = 0; i < kWItems; ++i) {
        const int k = base + i;
        if (k < n) {
          const T lo = k == 0 ? T(0) : g2 + eps;
          const T hi = key[i] - eps;
          if (hi > lo) {
            if (at < max_pieces) {
              pieces[2 * at] = (double)lo;
              pieces[2 * at + 1] = (double)hi;
            }
            ++at;
          }
          g2 = val[i] > g2 ? val[i] : g2;
        }
      }
      np += np_chunk;
    }
  }
  gamma = gamma > gchunk ? gamma : gchunk;
  len += chunk_len;
}

// Sorts n arcs (k0, v0) of the CTA's scratch slot by key: chunks of kWSlots
// sorted in registers and shared memory, then merge-path merges of runs of
// kWSlots, 2 kWSlots, ... between (k0, v0) and (k1, v1).  (ko, vo) receive the
// buffers that hold the result.  Contains __syncthreads (call uniformly).
template <typename T>
__device__ void global_sort_arcs(T* k0, T* v0, T* k1, T* v1, int n, T* s_key, T* s_val, T inf,
                                 T*& ko, T*& vo) {
  const int base = threadIdx.x * kWItems;
  for (int cb = 0; cb < n; cb += kWSlots) {
    const int cn = min(kWSlots, n - cb);
    T key[kWItems], val[kWItems];
#pragma unroll
    for (int i = 0; i < kWItems; ++i) {
      key[i] = base + i < cn ? k0[cb + base + i] : inf;
      val[i] = base + i < cn ? v0[cb + base + i] : T(0);
    }
    block_sort_arcs<kWItems, T>(key, val, (cn + kWItems - 1) / kWItems * kWItems, s_key, s_val,
                                inf);
#pragma unroll
    for (int i = 0; i < kWItems; ++i) {
      if (base + i < cn) {
        k0[cb + base + i] = key[i];
        v0[cb + base + i] = val[i];
      }
    }
    __syncthreads();
  }
  T *sk = k0, *sv = v0, *dk = k1, *dv = v1;
  for (int w = kWSlots; w < n; w <<= 1) {
    for (int ob = 0; ob < n; ob += kWSlots) {
      const int pos = ob + base;
      if (pos < n) {
        const int start = pos & ~(2 * w - 1);
        const int diag = pos - start;
        const int a_end = min(w, n - start);
        const int b_len = max(0, min(w, n - start - w));
        int lo = max(0, diag - b_len), hi = min(diag, a_end);
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (!(sk[start + w + diag - 1 - mid] < sk[start + mid])) lo = mid + 1;
          else hi = mid;
        }
        int ia = lo, ib = diag - lo;
#pragma unroll
        for (int i = 0; i < kWItems; ++i) {
          if (pos + i < n) {
            const bool a_ok = ia < a_end;
            const bool b_ok = ib < b_len;
            const T ka = a_ok ? sk[start + ia] : inf;
            const T kb = b_ok ? sk[start + w + ib] : inf;
            const bool take_a = a_ok && (!b_ok || !(kb < ka));
            dk[pos + i] = take_a ? ka : kb;
            dv[pos + i] = take_a ? sv[start + ia] : sv[start + w + ib];
            ia += take_a ? 1 : 0;
            ib += take_a ? 0 : 1;
          }
        }
      }
    }
    __syncthreads();
    T* t = sk; sk = dk; dk = t;
    t = sv; sv = dv; dv = t;
  }
  ko = sk;
  vo = sv;
}

template <typename T>
__global__ void __launch_bounds__(kWT, ESS_WIDE_MINBLOCKS) chain_wide_kernel(ChainParams<T> prm) {
  constexpr int NB = wide_buckets<T>();
  constexpr int NSH = wide_short_smem<T>();
  constexpr int NC = wide_cand<T>();
  static_assert(NC <= kWFlag, "candidate codes share the recheck list");
  constexpr int BPT = NB / kWT;  // buckets per thread
  using Bits = BitsOf<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_key = reinterpret_cast<T*>(smem_raw);
  T* s_val = s_key + kWPad;
  Bits* s_bmin = reinterpret_cast<Bits*>(s_val + kWPad);
  Bits* s_bmax = s_bmin + NB;
  int* s_flag = reinterpret_cast<int*>(s_bmax + NB);
  // candidate rows of the prune (codes in the recheck list's space, which is
  // free until the move) and their pseudo-beta
  unsigned* s_ccode = reinterpret_cast<unsigned*>(s_flag);
  float* s_cpb = reinterpret_cast<float*>(s_flag + kWFlag);
  T* s_x = reinterpret_cast<T*>(s_cpb + NC);

  // prune buckets: the max pseudo-beta (bits) of the arcs of pseudo-alpha
  // bucket j sits in slot bslot(j + 2); after the prefix max, slot bslot(j)
  // holds the max over the buckets <= j - 2
  __shared__ __align__(16) unsigned s_pbk[kWBP];
  __shared__ __align__(16) unsigned s_pbf[kWBP];  // the later rows' maxima, then the full ones
  __shared__ int s_itmp[kWW];
  __shared__ T s_ttmp[kWW];
  __shared__ int s_ncand, s_nshort, s_nflag, s_reject, s_bad, s_tangent, s_best, s_infeasible;
  __shared__ T s_theta;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T two_pi = Lim<T>::two_pi();
  const T inf = Lim<T>::inf();
  const long long cap = prm.wide_cap;
  T* gk0 = prm.wide_scratch + (size_t)blockIdx.x * 4 * cap;
  T* gv0 = gk0 + cap;
  T* gk1 = gv0 + cap;
  T* gv1 = gk1 + cap;

  const int n_work = prm.chain_list ? *prm.list_count : prm.n_chains;
  for (int work = blockIdx.x; work < n_work; work += gridDim.x) {
    const int c = prm.chain_list ? prm.chain_list[work] : work;
    const ChainView<T> v = chain_view<T, false>(prm, c);
    const int m = v.m, d = v.d;
    const T* Prow = v.P;
    const T* Qrow = v.Q;
    __syncthreads();
    if (tid == 0) {
      s_ncand = 0;
      s_nshort = 0;
      s_nflag = 0;
      s_reject = 0;
      s_bad = 0;
      s_tangent = 0;
      s_best = -1;
      s_infeasible = 0;
    }
    for (int k = tid; k < kWBP; k += kWT) {
      s_pbk[k] = 0u;
      s_pbf[k] = 0u;
    }
    for (int k = tid; k < NB; k += kWT) {
      s_bmin[k] = empty_bits<T>();
      s_bmax[k] = 0;
    }
    __syncthreads();

    // squared thresholds of the float classification (1e-6 relative slack
    // around the exact test of roots())
    const float tlo_s = (float)((1.0 - prm.tangent_thresh) * 0.999999);
    const float thi_s = (float)((1.0 + prm.tangent_thresh) * 1.000001);
    const float tlo2 = tlo_s * tlo_s, thi2 = thi_s * thi_s;
    bool infeasible = false, nonfinite = false;
    // class and pseudo-angles of one row (a row with r = 0 has no root; x
    // violates it iff b_i < 0, read from the exact b in that rare case)
    auto classify = [&](T p, T q, T b, int i, float& pa, float& pb, bool& inf_row) {
      if constexpr (sizeof(T) == 4) {
        bool zero = false;
        const int cls = classify_phi_nb(p, q, b, tlo2, thi2, pa, pb, zero, nonfinite);
        if (zero) inf_row |= v.b64[i] < 0.0;
        return cls;
      } else {
        (void)i;
        (void)inf_row;
        return classify_phi_d(p, q, b, tlo2, thi2, pa, pb, nonfinite);
      }
    };

    // ---- 1. pseudo-angle arcs: the domination prune ----------------------------
    // A first batch of rows gives per-bucket maxima (s_pbk, then prefix-maxed);
    // every later row is tested against them: a row whose arc lies inside a
    // first-batch arc starting two buckets earlier is dropped, the others add
    // to the full maxima (s_pbf) and join the candidate list.  (A dropped row
    // adds nothing to the full maxima: the first-batch arc that covers it
    // dominates every arc it would dominate.)
    const int m_first = min(m, kWFirst);
    for (int i0 = 0; i0 < m_first; i0 += kWTrip) {
      T pv[kWU], qv[kWU], bv[kWU];
#pragma unroll
      for (int k = 0; k < kWU; ++k) {
        const int i = i0 + tid + k * kWT;
        pv[k] = i < m_first ? Prow[i] : T(0);
        qv[k] = i < m_first ? Qrow[i] : T(0);
        bv[k] = i < m_first ? v.b[i] : T(0);
      }
#pragma unroll
      for (int k = 0; k < kWU; ++k) {
        const int i = i0 + tid + k * kWT;
        if (i < m_first) {
          float pa = 0.f, pb = 0.f;
          const int cls = classify(pv[k], qv[k], bv[k], i, pa, pb, infeasible);
          if (cls == kRowApprox) atomicMax(&s_pbk[bslot(pbucket(pa) + 2)], __float_as_uint(pb));
        }
      }
    }
    __syncthreads();
    if (warp == 0) prefix_max(s_pbk, lane);
    __syncthreads();
    for (int i0 = m_first; i0 < m; i0 += kWTrip) {
      T pv[kWU], qv[kWU], bv[kWU];
#pragma unroll
      for (int k = 0; k < kWU; ++k) {
        const int i = i0 + tid + k * kWT;
        pv[k] = i < m ? Prow[i] : T(0);
        qv[k] = i < m ? Qrow[i] : T(0);
        bv[k] = i < m ? v.b[i] : T(0);
      }
#pragma unroll
      for (int k = 0; k < kWU; ++k) {
        const int i = i0 + tid + k * kWT;
        bool cand = false;
        unsigned code = 0u;
        float pb = 0.f;
        if (i < m) {
          float pa = 0.f;
          const int cls = classify(pv[k], qv[k], bv[k], i, pa, pb, infeasible);
          const int bk = pbucket(pa);
          const bool undominated =
              !(pb + 2.f * kPhiMargin <= __uint_as_float(s_pbk[bslot(bk)]));
          if (cls == kRowApprox && undominated)
            atomicMax(&s_pbf[bslot(bk + 2)], __float_as_uint(pb));
          cand = cls == kRowKeep || (cls == kRowApprox && undominated);
          code = cls == kRowKeep ? (0x80000000u | (unsigned)i)
                                 : (((unsigned)bk << kWRowBits) | (unsigned)i);
        }
        // candidate list: one shared atomic per warp
        const unsigned ball = __ballot_sync(kFull, cand);
        if (ball) {
          const int leader = __ffs(ball) - 1;
          int base = 0;
          if (lane == leader) base = atomicAdd(&s_ncand, __popc(ball));
          base = __shfl_sync(kFull, base, leader);
          const int at = base + __popc(ball & ((1u << lane) - 1u));
          if (cand && at < NC) {
            s_ccode[at] = code;
            s_cpb[at] = pb;
          }
        }
      }
    }
    __syncthreads();
    // full maxima: prefix max of the later rows' maxima, joined with the first batch's
    if (warp == 0) prefix_max(s_pbf, lane);
    __syncthreads();
    for (int k = tid; k < kWBP; k += kWT) s_pbf[k] = max(s_pbf[k], s_pbk[k]);
    __syncthreads();

    // ---- 2. exact roots of the rows not dominated, merged per bucket -----------
    int tangent = 0;
    const T bucket_w = two_pi / (T)NB;
    const T to_slot = (T)NB / two_pi;
    // exact roots of one kept row (App. B, Sec. 3.2), merged into its bucket
    auto exact_merge = [&](T p, T q, T b, double b64) {
      T al, be;
      bool inf_root = false;
      const bool has = roots(p, q, b, b64, prm.tangent_thresh, al, be, inf_root, tangent);
      infeasible |= inf_root;
      if (!has) return;
      // bucket j = [lo_j, hi_j], lo_j = j w, hi_j = (j + 1) w (2 pi for the
      // last); the same expressions for every arc, so hi_j == lo_(j+1)
      int j = min(max((int)(al * to_slot), 0), NB - 1);
      auto lo_of = [&](int bb) { return (T)bb * bucket_w; };
      auto hi_of = [&](int bb) { return bb + 1 == NB ? two_pi : (T)(bb + 1) * bucket_w; };
      if (j > 0 && al < lo_of(j)) --j;
      else if (j + 1 < NB && al > hi_of(j)) ++j;
      if (al >= lo_of(j) && al <= hi_of(j) && be >= hi_of(j)) {
        atomicMin(&s_bmin[j], abs_bits<T>(al));
        atomicMax(&s_bmax[j], abs_bits<T>(be));
      } else {
        // shorter than its bucket: to the short list
        const int at = atomicAdd(&s_nshort, 1);
        if (at < NSH) {
          s_key[pad_idx(at)] = al;
          s_val[pad_idx(at)] = be;
        } else {
          gk0[at - NSH] = al;
          gv0[at - NSH] = be;
        }
      }
    };
    // rows [r0, r1) streamed: classified again and tested against the full maxima
    auto stream_rows = [&](int r0, int r1) {
      for (int i0 = r0; i0 < r1; i0 += kWTrip) {
        // every operand of the trip's rows is loaded up front (exact b too:
        // the near-tangent roots take it), so that the loads overlap
        T pv[kWU], qv[kWU], bv[kWU];
        double b64v[kWU];
#pragma unroll
        for (int k = 0; k < kWU; ++k) {
          const int i = i0 + tid + k * kWT;
          pv[k] = i < r1 ? Prow[i] : T(0);
          qv[k] = i < r1 ? Qrow[i] : T(0);
          bv[k] = i < r1 ? v.b[i] : T(0);
          if constexpr (sizeof(T) == 8) b64v[k] = bv[k];  // double chains: b is exact b
          else b64v[k] = i < r1 ? v.b64[i] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < kWU; ++k) {
          const int i = i0 + tid + k * kWT;
          if (i >= r1) continue;
          float pa = 0.f, pb = 0.f;
          const int cls = classify(pv[k], qv[k], bv[k], i, pa, pb, infeasible);
          // dominated: inside an arc of a bucket at least two earlier
          const bool keep =
              cls == kRowKeep ||
              (cls == kRowApprox &&
               !(pb + 2.f * kPhiMargin <= __uint_as_float(s_pbf[bslot(pbucket(pa))])));
          if (keep) exact_merge(pv[k], qv[k], bv[k], b64v[k]);
        }
      }
    };
    const int n_cand = s_ncand;
    if (n_cand <= NC) {
      // the first batch, then the candidates (rows read where they lie)
      stream_rows(0, m_first);
      for (int e = tid; e < n_cand; e += kWT) {
        const unsigned code = s_ccode[e];
        const int i = (int)(code & kWRowMask);
        const bool keep =
            (code & 0x80000000u) != 0u ||
            !(s_cpb[e] + 2.f * kPhiMargin <=
              __uint_as_float(s_pbf[bslot((int)((code >> kWRowBits) & 0x1FFu))]));
        if (keep) exact_merge(Prow[i], Qrow[i], v.b[i], v.b64[i]);
      }
    } else {
      stream_rows(0, m);
    }
    if (tangent) atomicAdd(&s_tangent, tangent);
    if (infeasible) s_infeasible = 1;
    if (nonfinite) s_bad = 1;
    __syncthreads();

    // ---- 3. the arcs of Alg. 3: bucket intervals (in bucket order) + short arcs --
    const int ns = s_nshort;
    const bool in_smem = ns <= NSH;
    Bits lo_b[BPT], hi_b[BPT];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      lo_b[k] = s_bmin[tid * BPT + k];
      hi_b[k] = s_bmax[tid * BPT + k];
      cnt += lo_b[k] != empty_bits<T>() ? 1 : 0;
    }
    int nb;
    int at = ns + block_exclusive_scan<kWT>(cnt, 0, OpAdd(), s_itmp, nb);
    const int n = ns + nb;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      if (lo_b[k] != empty_bits<T>()) {
        if (in_smem) {
          s_key[pad_idx(at)] = from_bits<T>(lo_b[k]);
          s_val[pad_idx(at)] = from_bits<T>(hi_b[k]);
        } else {
          gk0[at] = from_bits<T>(lo_b[k]);
          gv0[at] = from_bits<T>(hi_b[k]);
        }
        ++at;
      }
    }
    if (!in_smem) {
      // the short arcs held in shared memory follow the spilled ones
      for (int e = tid; e < NSH; e += kWT) {
        gk0[ns - NSH + e] = s_key[pad_idx(e)];
        gv0[ns - NSH + e] = s_val[pad_idx(e)];
      }
    }
    __syncthreads();

    const T eps = (T)prm.trim_eps;
    const double u = prm.U ? prm.U[c] : theta_uniform(prm.seed, v.chain, v.t, v.problem);
    double* pieces_row = prm.pieces_out ? prm.pieces_out + (size_t)c * prm.max_pieces * 2 : nullptr;
    T gamma = T(0), mid_total = T(0);
    int cand = -1;
    T cand_theta = T(0);
    int np = 0;
    T tail_lo, tail_len, total, s;
    auto finish_total = [&]() {
      // tail piece [gamma_(n) + eps, 2 pi] (the whole circle when no row has roots)
      tail_lo = n > 0 ? gamma + eps : T(0);
      tail_len = two_pi > tail_lo ? two_pi - tail_lo : T(0);
      total = mid_total + tail_len;
      s = (T)(u * (double)total);
    };
    if (in_smem) {
      const int base = tid * kWItems;
      T key[kWItems], val[kWItems];
#pragma unroll
      for (int i = 0; i < kWItems; ++i) {
        key[i] = base + i < n ? s_key[pad_idx(base + i)] : inf;
        val[i] = base + i < n ? s_val[pad_idx(base + i)] : T(0);
      }
      // the bucket intervals alone are already in ascending order of alpha
      if (ns > 0)
        block_sort_arcs<kWItems, T>(key, val, (n + kWItems - 1) / kWItems * kWItems, s_key, s_val,
                                    inf);
      alg3_chunk<T>(key, val, 0, n, eps, gamma, mid_total, false, T(0), cand, cand_theta, s_ttmp,
                    s_itmp, nullptr, 0, np);
      finish_total();
      T g2 = T(0), l2 = T(0);
      alg3_chunk<T>(key, val, 0, n, eps, g2, l2, true, s, cand, cand_theta, s_ttmp, s_itmp,
                    pieces_row, prm.max_pieces, np);
    } else {
      T *ko, *vo;
      global_sort_arcs<T>(gk0, gv0, gk1, gv1, n, s_key, s_val, inf, ko, vo);
      for (int pass = 0; pass < 2; ++pass) {
        T g2 = T(0), l2 = T(0);
        for (int cb = 0; cb < n; cb += kWSlots) {
          const int base = cb + tid * kWItems;
          T key[kWItems], val[kWItems];
#pragma unroll
          for (int i = 0; i < kWItems; ++i) {
            key[i] = base + i < n ? ko[base + i] : inf;
            val[i] = base + i < n ? vo[base + i] : T(0);
          }
          if (pass == 0)
            alg3_chunk<T>(key, val, cb, n, eps, gamma, mid_total, false, T(0), cand, cand_theta,
                          s_ttmp, s_itmp, nullptr, 0, np);
          else
            alg3_chunk<T>(key, val, cb, n, eps, g2, l2, true, s, cand, cand_theta, s_ttmp, s_itmp,
                          pieces_row, prm.max_pieces, np);
        }
        if (pass == 0) finish_total();
      }
    }
    // ---- theta ~ U(I_act): the inverse CDF landed in piece cand (or the tail) ---
    if (tid == 0 && tail_len > T(0) && mid_total <= s) {
      // the tail is the last piece; it wins over every middle piece
      cand = n;
      const T th = tail_lo + (s - mid_total);
      cand_theta = th < two_pi ? th : two_pi;
    }
    if (cand >= 0) atomicMax(&s_best, cand);
    __syncthreads();
    if (cand >= 0 && cand == s_best) s_theta = cand_theta;
    if (tid == 0 && (s_best < 0 || !(total > T(0)))) s_theta = T(0);
    if (tid == 0 && prm.npieces_out) prm.npieces_out[c] = np + (tail_len > T(0) ? 1 : 0);
    if (tid == 0 && pieces_row && tail_len > T(0) && np < prm.max_pieces) {
      pieces_row[2 * np] = (double)tail_lo;
      pieces_row[2 * np + 1] = (double)two_pi;
    }
    __syncthreads();
    const T theta = s_theta;

    // ---- 4. move: x' into shared memory, p' streamed to P_out, rechecks --------
    T sn, cs;
    if constexpr (sizeof(T) == 8) {
      sincos((double)theta, reinterpret_cast<double*>(&sn), reinterpret_cast<double*>(&cs));
    } else {
      sincosf((float)theta, reinterpret_cast<float*>(&sn), reinterpret_cast<float*>(&cs));
    }
    const T* xrow = v.X;
    const T* nurow = v.NU;
    bool bad = !isfinite(theta);
    for (int j = tid; j < d; j += kWT) {
      const T xn = xrow[j] * cs + nurow[j] * sn;
      bad |= !isfinite(xn);
      s_x[j] = xn;
    }
    if (bad) s_bad = 1;
    __syncthreads();
    double my_maxres = -INFINITY;
    bool violated = false;
    int n_rechecks = 0;
    // FP64 residuals of the flagged rows (Sec. 3.3), one warp per row
    auto recheck = [&](int nf) {
      for (int f = warp; f < nf; f += kWW) {
        const int i = s_flag[f];
        const double* arow = v.A64 + (size_t)i * d;
        double acc = 0.0;
        for (int j = lane; j < d; j += 32) acc = fma(arow[j], (double)s_x[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        const double res = acc - v.b64[i];
        my_maxres = fmax(my_maxres, res);
        violated |= res > 0.0;
      }
      n_rechecks += nf;
      __syncthreads();
      if (tid == 0) s_nflag = 0;
      __syncthreads();
    };
    T* prow_out = v.P_out;
    for (int i0 = 0; i0 < m; i0 += kWTrip) {
      T pv[kWU], qv[kWU], sv[kWU];
#pragma unroll
      for (int k = 0; k < kWU; ++k) {
        const int i = i0 + tid + k * kWT;
        pv[k] = i < m ? Prow[i] : T(0);
        qv[k] = i < m ? Qrow[i] : T(0);
        sv[k] = i < m ? (v.slack ? v.slack[i] : (T)(v.b64[i] - prm.margin * v.anorm[i])) : T(0);
      }
#pragma unroll
      for (int k = 0; k < kWU; ++k) {
        const int i = i0 + tid + k * kWT;
        if (i < m) {
          const T pn = pv[k] * cs + qv[k] * sn;
          prow_out[i] = pn;
          if (!(pn <= sv[k])) s_flag[atomicAdd(&s_nflag, 1)] = i;  // within the margin, or NaN
        }
      }
      __syncthreads();
      const int nf = s_nflag;
      __syncthreads();  // every thread has read the count before the next trip adds to it
      // at most kWTrip rows join per trip: a batch is checked before the list can overflow
      if (nf > kWFlag - kWTrip) recheck(nf);
    }
    {
      const int nf = s_nflag;
      if (nf > 0) recheck(nf);
    }
    if (violated) s_reject = 1;
    __syncthreads();
    const bool reject = s_reject != 0 || s_bad != 0;

    // ---- write back ----------------------------------------------------------
    T* xout = v.X_out;
    if (!reject) {
      for (int j = tid; j < d; j += kWT) {
        xout[j] = s_x[j];
        if (v.S) v.S[j] = s_x[j];
      }
    } else {
      // Sec. 3.3: stay at x_t; p is restored
      for (int i = tid; i < m; i += kWT) prow_out[i] = Prow[i];
      for (int j = tid; j < d; j += kWT) {
        if (prm.X_out != prm.X) xout[j] = xrow[j];
        if (v.S) v.S[j] = xrow[j];
      }
    }

    // ---- statistics ----------------------------------------------------------
    double wmax = my_maxres;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(kFull, wmax, o));
    if (lane == 0 && wmax > -INFINITY) atomicMax(&prm.stats->max_residual_bits, enc_ordered(wmax));
    if (tid == 0) {
      if (prm.theta_out) prm.theta_out[c] = (double)theta;
      if (prm.rejected_out) prm.rejected_out[c] = reject ? 1 : 0;
      if (reject && s_bad == 0) atomicAdd(&prm.stats->rejections, 1ull);
      if (s_bad) {
        atomicAdd(&prm.stats->numeric_errors, 1ull);
        atomicOr(prm.status, kStatusNumeric);
      }
      if (s_tangent) atomicAdd(&prm.stats->tangent_fp64, (unsigned long long)s_tangent);
      atomicAdd(&prm.stats->sort_keys, (unsigned long long)n);
      if (n_rechecks) atomicAdd(&prm.stats->rechecks, (unsigned long long)n_rechecks);
      if (s_infeasible) atomicOr(prm.status, kStatusInfeasible);
    }
  }  // chains of this CTA
}

}  // namespace

template <typename T>
size_t chain_wide_smem_bytes(int d) {
  using Bits = BitsOf<T>;
  return 2 * (size_t)kWPad * sizeof(T) + 2 * (size_t)wide_buckets<T>() * sizeof(Bits) +
         (size_t)kWFlag * sizeof(int) + (size_t)wide_cand<T>() * sizeof(float) +
         (size_t)((d + 1) & ~1) * sizeof(T);
}

template <typename T>
long long chain_wide_cap(int m) {
  const long long n = (long long)m + wide_buckets<T>();
  return (n + kWSlots - 1) / kWSlots * kWSlots;
}

int chain_wide_slots(int device) {
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return 2 * sms;
}

template <typename T>
cudaError_t launch_chain_step_wide(const ChainParams<T>& p, int slots, cudaStream_t s) {
  if (p.n_chains <= 0) return cudaSuccess;
  if (p.P_out == p.P_in || !p.wide_scratch || p.wide_cap < chain_wide_cap<T>(p.m) || slots < 1 ||
      p.desc != nullptr || (p.chain_list && !p.list_count))
    return cudaErrorInvalidValue;
  const size_t smem = chain_wide_smem_bytes<T>(p.d);
  auto k = chain_wide_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // list mode: the list length is known on the device only; idle CTAs return
  const unsigned grid = (unsigned)(p.chain_list ? slots : std::min(slots, p.n_chains));
  k<<<grid, kWT, smem, s>>>(p);
  return cudaGetLastError();
}

template size_t chain_wide_smem_bytes<float>(int);
template size_t chain_wide_smem_bytes<double>(int);
template long long chain_wide_cap<float>(int);
template long long chain_wide_cap<double>(int);
template cudaError_t launch_chain_step_wide<float>(const ChainParams<float>&, int, cudaStream_t);
template cudaError_t launch_chain_step_wide<double>(const ChainParams<double>&, int,
                                                   cudaStream_t);

}  // namespace ess
