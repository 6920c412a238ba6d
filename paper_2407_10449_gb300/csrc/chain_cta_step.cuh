// chain_cta_step.cuh -- one elliptical-slice step of one chain by one CTA.
//
// For chain c (Alg. 1 body, arXiv 2407.10449):
//   1. roots of p_i cos(theta) + q_i sin(theta) = b_i for every row
//      (Eq. trigonometry-equation; closed form of App. B:
//      tau = atan2(q, p), h = arccos(b / r), open infeasible arc
//      (tau - h, tau + h) with tau shifted into [0, 2 pi)); rows with
//      b/r >= 1 or r = 0 are dropped instead of padded (Sec. 3.2: such a
//      constraint "can be simply ignored").
//   2. Alg. 3 on the kept arcs, sorted by alpha.  The arcs are first merged
//      per bucket of alpha (up to 2048 buckets of width w, 512 for double): an arc in bucket j = [j w, (j + 1) w] that reaches (j + 1) w
//      contains that point, so all such arcs of one bucket overlap and their
//      union is the single interval [min alpha, max beta]; the bucket
//      intervals are already in ascending order of alpha, and Alg. 3 on them
//      gives the same union of arcs (hence I_act) as on the arcs themselves,
//      without a sort.  If any kept arc is shorter than its bucket, the arcs
//      are sorted instead (register bitonic network per thread, then
//      merge-path merges in shared memory).  Then the cumulative max gamma_k
//      of beta (warp-shuffle scan), and the pieces [0, alpha_(1)],
//      [gamma_(k-1), alpha_(k)], [gamma_(n), 2 pi] of Prop. 1.
//   3. theta ~ U(I_act) by the inverse CDF over the piece lengths (prefix sum).
//   4. x' = x cos(theta) + nu sin(theta) (Alg. 1), p' = p cos(theta) +
//      q sin(theta) (A x carried forward), and the Sec. 3.3 safeguard: rows
//      with p'_i within margin * ||a_i|| of b_i get a_i.x' recomputed in
//      FP64; any violation rejects the move (x and p stay).
//
// T = double gives the plain FP64 form.  T = float gives the mixed form: the
// roots run in float except near tangency (|b/r| > 1 - tangent_thresh), where
// r, b/r, atan2 and arccos are evaluated in double (Sec. 3.2 discusses why
// b/r ~ +-1 is the delicate case).
#pragma once

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "chain_block_ops.cuh"
#include "chain_math.cuh"
#include "ess_kernels.cuh"

namespace ess {
namespace {

using namespace chainmath;
using namespace blockops;

// ---- the step ---------------------------------------------------------------
constexpr int kBuckets = 64;  // alpha buckets of the domination prune
// Alpha buckets of the interval merge (at most): 2048 for float chains; 512
// for double chains, whose larger arrays would otherwise cost the CTA kernel
// half its residency at m = 2000.
template <typename T>
constexpr int merge_buckets() { return sizeof(T) == 8 ? 512 : 2048; }

// One step of chain c by the whole CTA (NT threads, every thread calls it),
// with the dynamic shared memory at smem_raw (dyn_smem bytes: keys, values,
// x', flags, and the merge buckets when they fit).
template <typename T, int NT, int ITEMS, bool BATCH>
__device__ __forceinline__ void cta_chain_step(const ChainParams<T>& prm, int c,
                                               unsigned char* smem_raw, uint32_t dyn_smem) {
  constexpr int NSLOT = NT * ITEMS;
  constexpr int NPAD = NSLOT + NSLOT / 32;
  constexpr int NW = NT / 32;
  constexpr int NB = NSLOT < merge_buckets<T>() ? NSLOT : merge_buckets<T>();  // merge buckets
  T* s_key = reinterpret_cast<T*>(smem_raw);
  T* s_val = s_key + NPAD;
  T* s_x = s_val + NPAD;
  int* s_flag = reinterpret_cast<int*>(s_x + ((prm.d + 1) & ~1));
  // per alpha bucket: min alpha and max beta as ordered bit patterns
  // (non-negative floating-point values compare like their bits)
  using Bits = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned>::type;
  Bits* s_bmin = reinterpret_cast<Bits*>(s_flag + NSLOT);
  Bits* s_bmaxb = s_bmin + NB;

  __shared__ int s_itmp[NW];
  __shared__ T s_ttmp[NW];
  __shared__ unsigned int s_bmax[kBuckets];  // max approximate beta (bits) per alpha bucket
  __shared__ float s_gearly[kBuckets];       // max approximate beta over buckets <= j - 2
  __shared__ int s_nflag, s_reject, s_best, s_bad, s_tangent, s_noroot, s_slow;
  __shared__ T s_theta;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const T two_pi = Lim<T>::two_pi();
  const T inf = Lim<T>::inf();
  // the bucket arrays exist only if the launch provided their shared memory
  const bool can_merge =
      (size_t)dyn_smem >= 2 * NPAD * sizeof(T) + (size_t)((prm.d + 1) & ~1) * sizeof(T) +
                              NSLOT * sizeof(int) + 2 * NB * sizeof(T);
  const ChainView<T> v = chain_view<T, BATCH>(prm, c);
  const int m = v.m, d = v.d;
  __syncthreads();
  if (tid == 0) {
    s_nflag = 0;
    s_reject = 0;
    s_best = -1;
    s_bad = 0;
    s_tangent = 0;
    s_noroot = 0;
    s_slow = can_merge ? 0 : 1;
  }
  for (int k = tid; k < kBuckets; k += NT) s_bmax[k] = 0;
  for (int k = tid; k < NB && can_merge; k += NT) {
    s_bmin[k] = sizeof(T) == 8 ? (Bits)0x7FF0000000000000ull : (Bits)0x7F800000u;  // +inf
    s_bmaxb[k] = 0;
  }
  __syncthreads();

  // ---- 1. p, q of every row (kept in registers) and approximate arcs --------
  const T* Prow = v.P;
  const T* Qrow = v.Q;
  T p[ITEMS], q[ITEMS];
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int i = tid + r * NT;
    p[r] = i < m ? Prow[i] : T(0);
    q[r] = i < m ? Qrow[i] : T(0);
  }
  const T tlo = (T)(1.0 - prm.tangent_thresh);
  const T thi = (T)(1.0 + prm.tangent_thresh);
  int cls[ITEMS];
  float a_ap[ITEMS], b_ap[ITEMS];
  bool infeasible = false, nonfinite = false;
  const float to_bucket = (float)(kBuckets / kTwoPi);
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int i = tid + r * NT;
    cls[r] = kRowNone;
    a_ap[r] = 0.f;
    b_ap[r] = 0.f;
    if (i < m) {
      nonfinite |= !isfinite(p[r]) || !isfinite(q[r]);
      bool inf_row = false;
      cls[r] = classify_row<T>(p[r], q[r], v.b[i], v.b64[i], tlo, thi, a_ap[r], b_ap[r],
                               inf_row);
      infeasible |= inf_row;
      if (cls[r] == kRowApprox) {
        const int bk = min(kBuckets - 1, (int)(a_ap[r] * to_bucket));
        atomicMax(&s_bmax[bk], __float_as_uint(b_ap[r]));
      }
    }
  }
  __syncthreads();

  // ---- domination prune ------------------------------------------------------
  // Arc i (alpha_i in bucket j) lies inside an arc D from a bucket <= j - 2
  // whenever beta_i <= beta_D: then alpha_D < alpha_i (buckets are wider than
  // twice the approximation error) and D covers arc i, so dropping arc i
  // leaves the union of arcs -- I_act and its piece endpoints -- unchanged.
  // With approximate angles the test is b_ap_i + 2 margin <= max b_ap over
  // the buckets <= j - 2.
  if (warp == 0) {
    // lane l holds buckets 2l and 2l + 1; incl = max over buckets <= 2l + 1
    const float b0 = __uint_as_float(s_bmax[2 * lane]);
    const float b1 = __uint_as_float(s_bmax[2 * lane + 1]);
    float incl = fmaxf(b0, b1);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl = fmaxf(y, incl);
    }
    const float incl1 = __shfl_up_sync(kFull, incl, 1);  // buckets <= 2l - 1
    const float incl2 = __shfl_up_sync(kFull, incl, 2);  // buckets <= 2l - 3
    const float b0_prev = __shfl_up_sync(kFull, b0, 1);  // bucket 2l - 2
    // max over buckets <= j - 2 for j = 2l and j = 2l + 1 (-1: no such bucket)
    s_gearly[2 * lane] = lane == 0 ? -1.f : (lane == 1 ? b0_prev : fmaxf(incl2, b0_prev));
    s_gearly[2 * lane + 1] = lane == 0 ? -1.f : incl1;
  }
  __syncthreads();
  // Long arcs (b_i <= 0: half a circle or more) overlap pairwise when x is
  // feasible, so together they are one arc (min alpha, max beta): an arc
  // inside it changes no piece, and the rows holding the two extremes stay.
  float ua = INFINITY, ub = -INFINITY;
  if (v.long_arcs) {
    __shared__ float s_utmp[NW];
    float my_na = -INFINITY, my_b = -INFINITY;
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const int i = tid + r * NT;
      if (cls[r] == kRowApprox && v.b[i] <= T(0)) {
        my_na = fmaxf(my_na, -a_ap[r]);
        my_b = fmaxf(my_b, b_ap[r]);
      }
    }
    float tot;
    (void)block_exclusive_scan<NT>(my_na, -INFINITY, OpMax(), s_utmp, tot);
    ua = -tot;
    (void)block_exclusive_scan<NT>(my_b, -INFINITY, OpMax(), s_utmp, tot);
    ub = tot;
  }
  int my_count = 0;
  bool keep[ITEMS];
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    keep[r] = cls[r] == kRowKeep;
    if (cls[r] == kRowApprox) {
      const int bk = min(kBuckets - 1, (int)(a_ap[r] * to_bucket));
      keep[r] = !(b_ap[r] + 2.f * kPruneMargin <= s_gearly[bk]) &&
                !(a_ap[r] >= ua + 2.f * kPruneMargin && b_ap[r] <= ub - 2.f * kPruneMargin);
    }
    my_count += keep[r] ? 1 : 0;
  }
  int n_keep;
  int offset = block_exclusive_scan<NT>(my_count, 0, OpAdd(), s_itmp, n_keep);
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    if (keep[r]) s_flag[offset++] = tid + r * NT;  // kept row indices (s_flag is free until step 5)
  }
  __syncthreads();

  // ---- exact roots of the kept rows (App. B, Sec. 3.2), merged per bucket ----
  int tangent = 0, no_root = 0;
  const T bucket_w = two_pi / (T)NB;
  const T to_slot = (T)NB / two_pi;
  bool slow = false;
  for (int k = tid; k < n_keep; k += NT) {
    const int i = s_flag[k];
    T al, be;
    bool inf_row = false;
    const bool has = roots(Prow[i], Qrow[i], v.b[i], v.b64[i], prm.tangent_thresh, al, be,
                           inf_row, tangent);
    infeasible |= inf_row;
    s_key[pad_idx(k)] = has ? al : inf;
    s_val[pad_idx(k)] = has ? be : T(0);
    no_root += has ? 0 : 1;
    if (has && can_merge) {
      // bucket j = [lo_j, hi_j], lo_j = j w, hi_j = (j + 1) w (2 pi for the
      // last); the same expressions for every arc, so hi_j == lo_(j+1)
      int j = min(max((int)(al * to_slot), 0), NB - 1);
      auto lo_of = [&](int b) { return (T)b * bucket_w; };
      auto hi_of = [&](int b) { return b + 1 == NB ? two_pi : (T)(b + 1) * bucket_w; };
      if (j > 0 && al < lo_of(j)) --j;
      else if (j + 1 < NB && al > hi_of(j)) ++j;
      if (al >= lo_of(j) && al <= hi_of(j) && be >= hi_of(j)) {
        Bits ab, bb;
        if constexpr (sizeof(T) == 8) {
          ab = (Bits)__double_as_longlong((double)al) & 0x7FFFFFFFFFFFFFFFull;  // +0 for -0
          bb = (Bits)__double_as_longlong((double)be) & 0x7FFFFFFFFFFFFFFFull;
        } else {
          ab = (Bits)__float_as_uint((float)al) & 0x7FFFFFFFu;
          bb = (Bits)__float_as_uint((float)be) & 0x7FFFFFFFu;
        }
        atomicMin(&s_bmin[j], ab);
        atomicMax(&s_bmaxb[j], bb);
      } else {
        slow = true;  // shorter than its bucket: this chain's arcs are sorted
      }
    }
  }
  if (slow) s_slow = 1;
  if (tangent) atomicAdd(&s_tangent, tangent);
  if (no_root) atomicAdd(&s_noroot, no_root);
  const int n_active_slots = ((n_keep + ITEMS - 1) / ITEMS) * ITEMS;
  for (int k = n_keep + tid; k < n_active_slots; k += NT) {
    s_key[pad_idx(k)] = inf;
    s_val[pad_idx(k)] = T(0);
  }
  __syncthreads();
  int n_roots = n_keep - s_noroot;  // rows without roots sort to the end (+inf)
  const int base = tid * ITEMS;
  T key[ITEMS], val[ITEMS];
  if (!s_slow) {
    // ---- 2a. bucket intervals in ascending order of alpha -------------------
    int my_n = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      key[i] = inf;
      val[i] = T(0);
      if (base + i < NB) {
        const Bits ab = s_bmin[base + i];
        key[i] = sizeof(T) == 8 ? (T)__longlong_as_double((long long)ab)
                                : (T)__uint_as_float((unsigned)ab);
        const Bits bb = s_bmaxb[base + i];
        val[i] = sizeof(T) == 8 ? (T)__longlong_as_double((long long)bb)
                                : (T)__uint_as_float((unsigned)bb);
      }
      my_n += key[i] < inf ? 1 : 0;
    }
    int n_int;
    int at = block_exclusive_scan<NT>(my_n, 0, OpAdd(), s_itmp, n_int);
    // compact the non-empty buckets to the front, in bucket order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (key[i] < inf) {
        s_key[pad_idx(at)] = key[i];
        s_val[pad_idx(at)] = val[i];
        ++at;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool in = base + i < n_int;
      key[i] = in ? s_key[pad_idx(base + i)] : inf;
      val[i] = in ? s_val[pad_idx(base + i)] : T(0);
    }
    n_roots = n_int;
  } else {
  // ---- 2b. Alg. 3: sort alpha ascending, beta as payload -----------------
  // Only the first n_active_slots positions hold arcs; the rest is padding
  // (+inf keys) that the sort never needs to touch.
  const bool owns = base < n_active_slots;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    key[i] = owns ? s_key[pad_idx(base + i)] : inf;
    val[i] = owns ? s_val[pad_idx(base + i)] : T(0);
  }
  block_sort_arcs<ITEMS, T>(key, val, n_active_slots, s_key, s_val, inf);
  }  // sorted arcs

  // ---- 3. Alg. 3: gamma_k = cumulative max of beta ----------------------
  T g[ITEMS];
  T run = T(0);
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (base + i < n_roots) run = val[i] > run ? val[i] : run;
    g[i] = run;
  }
  T gamma_total;
  const T gamma_excl = block_exclusive_scan<NT>(run, T(0), OpMax(), s_ttmp, gamma_total);

  // ---- Alg. 3 / Prop. 1: pieces and their lengths ----------------------
  const T eps = (T)prm.trim_eps;
  T plo[ITEMS], phi[ITEMS], plen[ITEMS];
  T my_len = T(0);
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int k = base + i;
    plo[i] = T(0);
    phi[i] = T(0);
    plen[i] = T(0);
    if (k < n_roots) {
      // piece k is [gamma_(k-1), alpha_(k)]; piece 0 is [0, alpha_(1)] and
      // its left end is the glued point 0, which is never trimmed
      // gamma_(k-1) = max(beta of all earlier threads, this thread's earlier items)
      const T gprev = i == 0 ? gamma_excl : (g[i - 1] > gamma_excl ? g[i - 1] : gamma_excl);
      const T lo_k = k == 0 ? T(0) : gprev + eps;
      const T hi_k = key[i] - eps;
      plo[i] = lo_k;
      phi[i] = hi_k;
      plen[i] = hi_k > lo_k ? hi_k - lo_k : T(0);
      my_len += plen[i];
    }
  }
  T mid_total;
  const T len_prefix = block_exclusive_scan<NT>(my_len, T(0), OpAdd(), s_ttmp, mid_total);
  // tail piece [gamma_(n), 2 pi] (the whole circle when no row has roots)
  const T tail_lo = n_roots > 0 ? gamma_total + eps : T(0);
  const T tail_len = two_pi > tail_lo ? two_pi - tail_lo : T(0);
  const T total = mid_total + tail_len;

  // ---- 4. theta ~ U(I_act): inverse CDF ------------------------------------
  const double u = prm.U ? prm.U[c] : theta_uniform(prm.seed, v.chain, v.t, v.problem);
  const T s = (T)(u * (double)total);
  int cand = -1;
  T cand_theta = T(0);
  {
    T acc = len_prefix;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (plen[i] > T(0) && acc <= s) {
        cand = base + i;
        const T th = plo[i] + (s - acc);
        cand_theta = th < phi[i] ? th : phi[i];
      }
      acc += plen[i];
    }
  }
  if (tid == 0 && tail_len > T(0) && mid_total <= s) {
    // the tail is the last piece; it wins over every middle piece
    cand = NSLOT;
    const T th = tail_lo + (s - mid_total);
    cand_theta = th < two_pi ? th : two_pi;
  }
  if (cand >= 0) atomicMax(&s_best, cand);
  __syncthreads();
  if (cand >= 0 && cand == s_best) s_theta = cand_theta;
  if (tid == 0 && (s_best < 0 || !(total > T(0)))) s_theta = T(0);
  __syncthreads();
  const T theta = s_theta;

  // optional: the positive-length pieces (test/diagnostic output)
  if (prm.pieces_out != nullptr || prm.npieces_out != nullptr) {
    int my_np = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) my_np += plen[i] > T(0) ? 1 : 0;
    int np_total;
    int at = block_exclusive_scan<NT>(my_np, 0, OpAdd(), s_itmp, np_total);
    double* out = prm.pieces_out ? prm.pieces_out + (size_t)c * prm.max_pieces * 2 : nullptr;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (plen[i] > T(0)) {
        if (out && at < prm.max_pieces) {
          out[2 * at] = (double)plo[i];
          out[2 * at + 1] = (double)phi[i];
        }
        ++at;
      }
    }
    if (tid == 0) {
      int np = np_total + (tail_len > T(0) ? 1 : 0);
      if (out && tail_len > T(0) && np_total < prm.max_pieces) {
        out[2 * np_total] = (double)tail_lo;
        out[2 * np_total + 1] = (double)two_pi;
      }
      if (prm.npieces_out) prm.npieces_out[c] = np;
    }
  }

  // ---- 5. move: x' = x cos(theta) + nu sin(theta), p' likewise -----------
  T sn, cs;
  if constexpr (sizeof(T) == 8) {
    sincos((double)theta, reinterpret_cast<double*>(&sn), reinterpret_cast<double*>(&cs));
  } else {
    sincosf((float)theta, reinterpret_cast<float*>(&sn), reinterpret_cast<float*>(&cs));
  }
  const bool theta_ok = isfinite(theta);
  const T* xrow = v.X;
  const T* nurow = v.NU;
  bool bad = !theta_ok || nonfinite;
  for (int j = tid; j < d; j += NT) {
    const T xn = xrow[j] * cs + nurow[j] * sn;
    bad |= !isfinite(xn);
    s_x[j] = xn;
  }
  T pn[ITEMS];
  int my_flags = 0;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int i = tid + r * NT;
    pn[r] = p[r] * cs + q[r] * sn;
    if (i < m) {
      const T slack_bound = v.slack ? v.slack[i] : (T)(v.b64[i] - prm.margin * v.anorm[i]);
      if (!(pn[r] <= slack_bound)) {  // within the margin (or NaN)
        const int at = atomicAdd(&s_nflag, 1);
        s_flag[at] = i;
        ++my_flags;
      }
    }
  }
  if (bad) s_bad = 1;
  __syncthreads();

  // ---- 6. Sec. 3.3 safeguard: exact FP64 residual of the flagged rows -----
  const int nflag = s_nflag;
  double my_maxres = -INFINITY;
  bool violated = false;
  for (int f = warp; f < nflag; f += NW) {
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
  if (violated) s_reject = 1;
  __syncthreads();
  const bool reject = s_reject != 0 || s_bad != 0;

  // ---- 7. write back ------------------------------------------------------
  T* xout = v.X_out;
  if (!reject) {
    for (int j = tid; j < d; j += NT) xout[j] = s_x[j];
  } else if (prm.X_out != prm.X) {
    for (int j = tid; j < d; j += NT) xout[j] = xrow[j];
  }
  T* prow_out = v.P_out;
  if (!reject) {
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const int i = tid + r * NT;
      if (i < m) prow_out[i] = pn[r];
    }
  } else if (prm.P_out != prm.P_in) {
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const int i = tid + r * NT;
      if (i < m) prow_out[i] = p[r];
    }
  }
  if (v.S) {
    T* srow = v.S;
    for (int j = tid; j < d; j += NT) srow[j] = reject ? xrow[j] : s_x[j];
  }

  // ---- statistics ----------------------------------------------------------
  const int blk_tangent = s_tangent;
  const int blk_flags = nflag;
  // max residual across warps
  double wmax = my_maxres;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(kFull, wmax, o));
  if (lane == 0 && wmax > -INFINITY)
    atomicMax(&prm.stats->max_residual_bits, enc_ordered(wmax));
  if (tid == 0) {
    if (prm.theta_out) prm.theta_out[c] = (double)theta;
    if (prm.rejected_out) prm.rejected_out[c] = reject ? 1 : 0;
    if (reject && s_bad == 0) atomicAdd(&prm.stats->rejections, 1ull);
    if (s_bad) {
      atomicAdd(&prm.stats->numeric_errors, 1ull);
      atomicOr(prm.status, kStatusNumeric);
    }
    if (blk_tangent) atomicAdd(&prm.stats->tangent_fp64, (unsigned long long)blk_tangent);
    atomicAdd(&prm.stats->sort_keys, (unsigned long long)n_roots);
    if (blk_flags) atomicAdd(&prm.stats->rechecks, (unsigned long long)blk_flags);
  }
  if (infeasible) atomicOr(prm.status, kStatusInfeasible);
}

}  // namespace
}  // namespace ess
