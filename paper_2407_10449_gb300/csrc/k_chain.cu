// k_chain.cu -- one elliptical-slice step per chain, one CTA per chain.
//
// For chain c (Alg. 1 body, arXiv 2407.10449):
//   1. roots of p_i cos(theta) + q_i sin(theta) = b_i for every row
//      (Eq. trigonometry-equation; closed form of App. B:
//      tau = atan2(q, p), h = arccos(b / r), open infeasible arc
//      (tau - h, tau + h) with tau shifted into [0, 2 pi)); rows with
//      b/r >= 1 or r = 0 are dropped instead of padded (Sec. 3.2: such a
//      constraint "can be simply ignored").
//   2. Alg. 3: sort the left endpoints alpha with beta as payload (register
//      bitonic network per thread, then merge-path merges in shared memory),
//      cumulative max gamma_k of beta (warp-shuffle scan), and the pieces
//      [0, alpha_(1)], [gamma_(k-1), alpha_(k)], [gamma_(n), 2 pi] of Prop. 1.
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
#include <cfloat>
#include <cmath>

#include "ess_kernels.cuh"

namespace ess {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct Lim;
template <> struct Lim<float> {
  __device__ static float inf() { return INFINITY; }
  __device__ static float two_pi() { return kTwoPiF; }
};
template <> struct Lim<double> {
  __device__ static double inf() { return INFINITY; }
  __device__ static double two_pi() { return kTwoPi; }
};

// ---- roots (App. B, Sec. 3.2) ------------------------------------------
__device__ __forceinline__ bool roots_dp(double p, double q, double b, double& al, double& be,
                                         bool& infeasible) {
  double r = sqrt(p * p + q * q);
  if (r == 0.0) {
    infeasible = b < 0.0;
    return false;
  }
  double ratio = b / r;
  if (ratio >= 1.0) return false;
  if (ratio < -1.0) ratio = -1.0;
  double tau = atan2(q, p);
  if (tau < 0.0) tau += kTwoPi;
  double h = acos(ratio);
  al = fmax(0.0, tau - h);
  be = fmin(kTwoPi, tau + h);
  return true;
}

__device__ __forceinline__ bool roots(double p, double q, double b, double b64, double,
                                      double& al, double& be, bool& infeasible, int& tangent) {
  (void)b;
  (void)tangent;
  return roots_dp(p, q, b64, al, be, infeasible);
}

__device__ __forceinline__ bool roots(float p, float q, float b, double b64, double thresh,
                                      float& al, float& be, bool& infeasible, int& tangent) {
  float r2 = fmaf(p, p, q * q);
  if (r2 == 0.0f) {
    infeasible = b64 < 0.0;
    return false;
  }
  float ratio = b / sqrtf(r2);
  if (ratio >= (float)(1.0 + thresh)) return false;  // clearly no root
  if (fabsf(ratio) > (float)(1.0 - thresh)) {
    // near tangency: the arccos argument and the angles in double
    ++tangent;
    double ad, bd;
    bool has = roots_dp((double)p, (double)q, b64, ad, bd, infeasible);
    if (has) {
      al = (float)ad;
      be = fminf((float)bd, kTwoPiF);
    }
    return has;
  }
  float tau = atan2f(q, p);
  if (tau < 0.0f) tau += kTwoPiF;
  float h = acosf(ratio);
  al = fmaxf(0.0f, tau - h);
  be = fminf(kTwoPiF, tau + h);
  return true;
}

// ---- block scans ---------------------------------------------------------
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

// ---- kernel ----------------------------------------------------------------
template <typename T> struct BitsOf;
template <> struct BitsOf<float> {
  typedef unsigned int type;
  __device__ static type get(float v) { return __float_as_uint(v); }
  __device__ static float put(type v) { return __uint_as_float(v); }
};
template <> struct BitsOf<double> {
  typedef unsigned long long type;
  __device__ static type get(double v) { return (unsigned long long)__double_as_longlong(v); }
  __device__ static double put(type v) { return __longlong_as_double((long long)v); }
};

// Shared-memory slot of sorted position e: one padding word per 32 keeps the
// per-thread chunks (stride ITEMS) on distinct banks.
__device__ __forceinline__ int pad_idx(int e) { return e + (e >> 5); }

constexpr int kBuckets = 64;  // alpha buckets of the domination prune

template <typename T, int NT, int ITEMS>
__global__ void __launch_bounds__(NT, (768 / NT > 0 ? 768 / NT : 1)) chain_step_kernel(ChainParams<T> prm) {
  constexpr int NSLOT = NT * ITEMS;
  constexpr int NPAD = NSLOT + NSLOT / 32;
  constexpr int NW = NT / 32;
  typedef typename BitsOf<T>::type Bits;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_key = reinterpret_cast<T*>(smem_raw);
  T* s_val = s_key + NPAD;
  T* s_x = s_val + NPAD;
  int* s_flag = reinterpret_cast<int*>(s_x + ((prm.d + 1) & ~1));

  __shared__ int s_itmp[NW];
  __shared__ T s_ttmp[NW];
  __shared__ Bits s_bmax[kBuckets];   // max beta (bits) of the arcs whose alpha falls in a bucket
  __shared__ T s_gearly[kBuckets];    // max beta of the arcs in all earlier buckets
  __shared__ int s_nflag, s_reject, s_best, s_bad, s_tangent;
  __shared__ T s_theta;

  const int c = blockIdx.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int m = prm.m, d = prm.d;
  const T two_pi = Lim<T>::two_pi();
  const T inf = Lim<T>::inf();

  if (tid == 0) {
    s_nflag = 0;
    s_reject = 0;
    s_best = -1;
    s_bad = 0;
    s_tangent = 0;
  }
  for (int k = tid; k < kBuckets; k += NT) s_bmax[k] = 0;
  __syncthreads();

  // ---- 1. roots of every row, kept in registers --------------------------
  const T* Prow = prm.P_in + (size_t)c * prm.ldp;
  const T* Qrow = prm.Q + (size_t)c * prm.ldp;
  T p[ITEMS], q[ITEMS], al[ITEMS], be[ITEMS];
  bool has[ITEMS];
  int tangent = 0;
  bool infeasible = false, nonfinite = false;
  const T to_bucket = (T)(kBuckets / kTwoPi);
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int i = tid + r * NT;
    has[r] = false;
    p[r] = T(0);
    q[r] = T(0);
    if (i < m) {
      p[r] = Prow[i];
      q[r] = Qrow[i];
      nonfinite |= !isfinite((double)p[r]) || !isfinite((double)q[r]);
      bool inf_row = false;
      has[r] = roots(p[r], q[r], prm.b[i], prm.b64[i], prm.tangent_thresh, al[r], be[r], inf_row,
                     tangent);
      infeasible |= inf_row;
      if (has[r]) {
        const int bk = min(kBuckets - 1, (int)(al[r] * to_bucket));
        atomicMax(&s_bmax[bk], BitsOf<T>::get(be[r]));
      }
    }
  }
  if (tangent) atomicAdd(&s_tangent, tangent);
  __syncthreads();

  // ---- domination prune ------------------------------------------------------
  // An arc (alpha_i, beta_i) lies inside an arc that starts in an earlier
  // alpha bucket whenever beta_i <= max beta of the earlier buckets (bucket
  // indices are monotone in alpha), so it cannot change the union of arcs:
  // I_act and its piece endpoints are unchanged when it is dropped.
  if (warp == 0) {
    // exclusive prefix max over the buckets, two buckets per lane
    const T b0 = BitsOf<T>::put(s_bmax[2 * lane]);
    const T b1 = BitsOf<T>::put(s_bmax[2 * lane + 1]);
    T incl = b0 > b1 ? b0 : b1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl = y > incl ? y : incl;
    }
    T excl = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) excl = T(-1);
    s_gearly[2 * lane] = excl;
    s_gearly[2 * lane + 1] = b0 > excl ? b0 : excl;
  }
  __syncthreads();
  int my_count = 0;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    if (has[r]) {
      const int bk = min(kBuckets - 1, (int)(al[r] * to_bucket));
      has[r] = be[r] > s_gearly[bk];
      my_count += has[r] ? 1 : 0;
    }
  }
  int n_roots;
  int offset = block_exclusive_scan<NT>(my_count, 0, OpAdd(), s_itmp, n_roots);
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    if (has[r]) {
      s_key[pad_idx(offset)] = al[r];
      s_val[pad_idx(offset)] = be[r];
      ++offset;
    }
  }
  const int n_active_slots = ((n_roots + ITEMS - 1) / ITEMS) * ITEMS;
  for (int k = n_roots + tid; k < n_active_slots; k += NT) {
    s_key[pad_idx(k)] = inf;
    s_val[pad_idx(k)] = T(0);
  }
  __syncthreads();

  // ---- 2. Alg. 3: sort alpha ascending, beta as payload -----------------
  // Only the first n_active_slots positions hold arcs; the rest is padding
  // (+inf keys) that the sort never needs to touch.
  const int base = tid * ITEMS;
  const bool owns = base < n_active_slots;
  T key[ITEMS], val[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    key[i] = owns ? s_key[pad_idx(base + i)] : inf;
    val[i] = owns ? s_val[pad_idx(base + i)] : T(0);
  }
  // bitonic network over the thread's ITEMS registers
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
  // merge-path merges of sorted runs of width ITEMS, 2 ITEMS, ... until one
  // run holds every arc
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
  const double u = prm.U ? prm.U[c]
                         : theta_uniform(prm.seed, prm.chain0 + (uint32_t)c, prm.t, prm.problem);
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
  const bool theta_ok = isfinite((double)theta);
  const T* xrow = prm.X + (size_t)c * prm.ldx;
  const T* nurow = prm.NU + (size_t)c * prm.ldx;
  bool bad = !theta_ok || nonfinite;
  for (int j = tid; j < d; j += NT) {
    const T xn = xrow[j] * cs + nurow[j] * sn;
    bad |= !isfinite((double)xn);
    s_x[j] = xn;
  }
  T pn[ITEMS];
  int my_flags = 0;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int i = tid + r * NT;
    pn[r] = p[r] * cs + q[r] * sn;
    if (i < m) {
      const double slack_bound = prm.b64[i] - prm.margin * prm.anorm[i];
      if (!((double)pn[r] <= slack_bound)) {  // within the margin (or NaN)
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
    const double* arow = prm.A64 + (size_t)i * d;
    double acc = 0.0;
    for (int j = lane; j < d; j += 32) acc = fma(arow[j], (double)s_x[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    const double res = acc - prm.b64[i];
    my_maxres = fmax(my_maxres, res);
    violated |= res > 0.0;
  }
  if (violated) s_reject = 1;
  __syncthreads();
  const bool reject = s_reject != 0 || s_bad != 0;

  // ---- 7. write back ------------------------------------------------------
  T* xout = prm.X_out + (size_t)c * prm.ldx;
  if (!reject) {
    for (int j = tid; j < d; j += NT) xout[j] = s_x[j];
  } else if (prm.X_out != prm.X) {
    for (int j = tid; j < d; j += NT) xout[j] = xrow[j];
  }
  T* prow_out = prm.P_out + (size_t)c * prm.ldp;
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
  if (prm.samples) {
    T* srow = prm.samples + (size_t)c * prm.sample_stride;
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
    if (blk_flags) atomicAdd(&prm.stats->rechecks, (unsigned long long)blk_flags);
  }
  if (infeasible) atomicOr(prm.status, kStatusInfeasible);
}

}  // namespace

int chain_threads_for(int m) {
  int t = 32;
  while (t * kChainItems < m) t <<= 1;
  return t <= kChainMaxThreads ? t : 0;
}

template <typename T>
size_t chain_smem_bytes(int threads, int d) {
  const size_t nslot = (size_t)threads * kChainItems;
  const size_t npad = nslot + nslot / 32;
  return 2 * npad * sizeof(T) + (size_t)((d + 1) & ~1) * sizeof(T) + nslot * sizeof(int);
}

template <typename T>
cudaError_t launch_chain_step(const ChainParams<T>& p, int threads, cudaStream_t s) {
  const size_t smem = chain_smem_bytes<T>(threads, p.d);
  dim3 grid(p.n_chains);
#define ESS_CHAIN_CASE(NT)                                                              \
  case NT: {                                                                            \
    auto k = chain_step_kernel<T, NT, kChainItems>;                                     \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                    \
    if (e != cudaSuccess) return e;                                                     \
    k<<<grid, NT, smem, s>>>(p);                                                        \
    return cudaGetLastError();                                                          \
  }
  switch (threads) {
    ESS_CHAIN_CASE(32)
    ESS_CHAIN_CASE(64)
    ESS_CHAIN_CASE(128)
    ESS_CHAIN_CASE(256)
    ESS_CHAIN_CASE(512)
    ESS_CHAIN_CASE(1024)
    default:
      return cudaErrorInvalidValue;
  }
#undef ESS_CHAIN_CASE
}

template size_t chain_smem_bytes<float>(int, int);
template size_t chain_smem_bytes<double>(int, int);
template cudaError_t launch_chain_step<float>(const ChainParams<float>&, int, cudaStream_t);
template cudaError_t launch_chain_step<double>(const ChainParams<double>&, int, cudaStream_t);

}  // namespace ess
