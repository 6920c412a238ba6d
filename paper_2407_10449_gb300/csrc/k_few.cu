// k_few.cu -- FP64 chains of one polytope, a few at a time (1 to 16 chains):
// all steps of a run in one persistent cooperative kernel.
//
// With so few chains the generic path is a string of nearly empty launches:
// a GEMM with one to sixteen columns, one warp per chain for the roots and the
// sort.  Here every SM works on every step, and the phases of a step are
// separated by grid barriers (cooperative launch; every wait is bounded):
//   B  the rows of A are split over the CTAs; each CTA streams its rows once
//      per step, with nu (and x on refresh steps) of all chains staged in
//      shared memory, giving q = A nu (Sec. 2.2; p = A x on refresh steps, else
//      p is carried).  Every (chain, row) gets its exact FP64 roots (App. B);
//      the arc (alpha, beta) is merged into its chain's bucket of alpha
//      (kFewB buckets of width w over [0, 2 pi]) by atomic min of alpha and max
//      of beta.  An arc that reaches the end of its bucket contains that point,
//      so all such arcs of a bucket overlap and their union is [min alpha, max
//      beta]; an arc shorter than that (near tangency) goes to a short list.
//   D  one CTA per chain collects the non-empty buckets in ascending order (and
//      the short arcs, sorted with them by a bitonic sort when there are any),
//      runs Alg. 3 (cumulative max of beta, piece lengths, prefix sums) and
//      draws theta by the inverse CDF.  The union of the arcs, hence I_act, is
//      that of the arcs themselves.  With one chain every CTA runs D for it
//      (the same data and code give the same theta everywhere), so E needs no
//      grid barrier after D.  Buckets, short lists and flags come in two sets
//      by step parity: step t + 1 clears the set step t read.
//   E  x' = x cos + nu sin and p' = p cos + q sin into the other buffer of
//      each chain; rows with p' above b - margin ||a|| get their residual
//      recomputed in FP64 (Sec. 3.3: a positive one rejects the move); nu of
//      the next step is drawn.
// A chain's state lives in one of two buffers; a step that is not rejected
// flips which one.  The map is the one of ess_run in the FP64 form (the same
// draws: Philox counters (chain, step); the same roots and Alg. 3).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "chain_math.cuh"
#include "chain_warp_ops.cuh"
#include "ess_kernels.cuh"
#include "grid_sync.cuh"

namespace ess {
namespace {

using namespace chainmath;
using namespace warpops;

constexpr int kFT = 512;            // threads per CTA
constexpr int kFW = kFT / 32;       // warps per CTA
constexpr int kFB = kFewBuckets;    // angle buckets per chain
constexpr double kFewW = kTwoPi / kFB;  // their width
constexpr int kDW = 4;              // phase D: warps of the FP64 sweep
constexpr int kDT = kDW * 32;
constexpr int kFSlots = 256;        // phase B: (row, chain) pairs of a round (RW kFW CM)

// x cos + nu sin with one explicit rounding order (the FP64 recheck of a row
// evaluates exactly the x' that is written).
__device__ __forceinline__ double move_d(double x, double nu, double cs, double sn) {
  return __fma_rn(x, cs, __dmul_rn(nu, sn));
}

template <int CM>
__global__ void __launch_bounds__(kFT, 1) few_chains_kernel(FewArgs a) {
  // CM: chains the registers are sized for (C <= CM); rows per warp and round
  constexpr int RW = CM <= 4 ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sd = reinterpret_cast<double*>(smem_raw);
  __shared__ double s_cs[kMaxFew], s_sn[kMaxFew];  // cos, sin of each chain's theta
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int C = a.C, d = a.d, m = a.m;
  const int G = gridDim.x;
  const long long gtid = (long long)blockIdx.x * kFT + tid;
  const long long gthreads = (long long)G * kFT;
  const int gwarps = G * kFW;
  // the same index sets dealt CTA by CTA (thread tid of every CTA before
  // thread tid + 1): short FP64 loops (draws, the move, the rows of E) then
  // spread over all SMs instead of filling the first CTAs
  const long long sgtid = (long long)tid * G + blockIdx.x;
  const int sgwarp = warp * G + blockIdx.x;
  // rows of this CTA in phases B and C
  const int R = (m + G - 1) / G;
  const int r0 = min(m, blockIdx.x * R), r1 = min(m, r0 + R);
  const int nblk = (d + 3) >> 2;  // Philox blocks of nu per chain

  // ---- start: x0 into buffer 0, nu of the first step, per-step state cleared --
  for (long long k = gtid; k < (long long)C * kFB; k += gthreads) {
    a.bmin[0][k] = a.bmin[1][k] = kEmptyBucket;
    a.bmax[0][k] = a.bmax[1][k] = 0ull;
  }
  for (long long k = gtid; k < (long long)C * d; k += gthreads) {
    const int c = (int)(k / d), j = (int)(k % d);
    a.X[0][(size_t)c * d + j] = a.X_user[(size_t)c * d + j];
  }
  for (long long k = sgtid; k < (long long)C * nblk; k += gthreads) {
    const int c = (int)(k / nblk), n = (int)(k % nblk);
    uint32_t r[4];
    rng_block(a.seed, (uint32_t)n, (uint32_t)c, (uint32_t)a.t0, 0u, 0u, r);
    box_muller4(r, a.NU[a.t0 & 1] + (size_t)c * d + 4 * n, min(4, d - 4 * n), a.bm_tab);
  }
  if (!grid_barrier(a.bar, a.abort_flag, a.status, a.wait_ns, a.hold != 0 && blockIdx.x == 0))
    return;

  long long rejections = 0, rechecks = 0, sort_keys = 0;
  for (int t = a.t0; t < a.t0 + a.n_iter; ++t) {
    const int par = t & 1;
    const bool refresh = t == a.t0 || (t % a.refresh_k) == 0;
    // the buffer holding each chain's state: flipped after an accepted step
    // (read from the previous step's arrays, which no thread writes during
    // this step; thread 0 stores the result for the next step)
    auto xbuf = [&](int c) { return a.cur[par ^ 1][c] ^ (a.rej[par ^ 1][c] ? 0 : 1); };
    if (gtid == 0) {
      for (int c = 0; c < C; ++c) {
        if (t > a.t0 && a.rej[par ^ 1][c] && !a.bad_prev[c]) ++rejections;
        a.cur[par][c] = xbuf(c);
        a.rej[par][c] = 0;
      }
    }
    // record the state after the previous step
    if (a.samples && t > a.t0 && (t - a.t0) % a.record_every == 0) {
      const int rec = (t - a.t0) / a.record_every - 1;
      for (long long k = gtid; k < (long long)C * d; k += gthreads) {
        const int c = (int)(k / d), j = (int)(k % d);
        a.samples[((size_t)c * a.n_rec + rec) * d + j] = a.X[xbuf(c)][(size_t)c * d + j];
      }
    }

    // the other parity's arcs, short lists and flags were read in D of the
    // previous step, which every CTA has finished: cleared for the next step
    for (long long k = gtid; k < (long long)C * kFB; k += gthreads) {
      a.bmin[par ^ 1][k] = kEmptyBucket;
      a.bmax[par ^ 1][k] = 0ull;
    }
    if (gtid < C) {
      a.nshort[par ^ 1][gtid] = 0;
      a.bad[par ^ 1][gtid] = 0;
    }

    // ---- B: q = A nu (p = A x on refresh steps), float classification ----------
    {
      const double* NU = a.NU[par];
      const int chunk = a.chunk;
      double* nu_s = sd;                          // C x chunk
      double* x_s = sd + (size_t)C * chunk;       // C x chunk (refresh)
      // a round's (row, chain) pairs for the roots: slot (h kFW + warp) CM + c
      __shared__ double s_rp[kFSlots], s_rq[kFSlots];
      __shared__ int s_ri[kFSlots];  // the row, or -1
      static_assert(RW * kFW * CM <= kFSlots, "root slots of a round");
      // each warp: RW rows of this CTA per round, all chains
      for (int base = r0; base < r1; base += RW * kFW) {
        double qs[RW][CM], ps[RW][CM];
#pragma unroll
        for (int h = 0; h < RW; ++h)
#pragma unroll
          for (int c = 0; c < CM; ++c) qs[h][c] = ps[h][c] = 0.0;
        for (int j0 = 0; j0 < d; j0 += chunk) {
          const int len = min(chunk, d - j0);
          __syncthreads();
          for (int k = tid; k < C * len; k += kFT) {
            const int c = k / len, j = k - c * len;
            nu_s[(size_t)c * chunk + j] = NU[(size_t)c * d + j0 + j];
            if (refresh)
              x_s[(size_t)c * chunk + j] = a.X[xbuf(c)][(size_t)c * d + j0 + j];
          }
          __syncthreads();
          for (int j = lane; j < len; j += 32) {
            double av[RW];
#pragma unroll
            for (int h = 0; h < RW; ++h) {
              const int i = base + h * kFW + warp;
              av[h] = i < r1 ? a.A[(size_t)i * d + j0 + j] : 0.0;
            }
#pragma unroll
            for (int c = 0; c < CM; ++c) {
              if (c < C) {
                const double nu = nu_s[(size_t)c * chunk + j];
                const double x = refresh ? x_s[(size_t)c * chunk + j] : 0.0;
#pragma unroll
                for (int h = 0; h < RW; ++h) {
                  qs[h][c] = fma(av[h], nu, qs[h][c]);
                  if (refresh) ps[h][c] = fma(av[h], x, ps[h][c]);
                }
              }
            }
          }
        }
        // sums over the lanes; lane c keeps chain c's values
        double myq[RW], myp[RW];
#pragma unroll
        for (int h = 0; h < RW; ++h) myq[h] = myp[h] = 0.0;
#pragma unroll
        for (int c = 0; c < CM; ++c) {
          if (c < C) {
#pragma unroll
            for (int h = 0; h < RW; ++h) {
              double v = qs[h][c], w = ps[h][c];
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_xor_sync(kFull, v, o);
                if (refresh) w += __shfl_xor_sync(kFull, w, o);
              }
              if (lane == c) {
                myq[h] = v;
                myp[h] = w;
              }
            }
          }
        }
        if (lane < C) {
          const int c = lane;
          const int xbc = xbuf(c);
#pragma unroll
          for (int h = 0; h < RW; ++h) {
            const int i = base + h * kFW + warp;
            const int slot = (h * kFW + warp) * CM + c;
            s_ri[slot] = i < r1 ? i : -1;
            if (i >= r1) continue;
            double* Pc = a.P[xbc] + (size_t)c * m;
            double p;
            if (refresh) {
              p = myp[h];
              Pc[i] = p;
              if (t == a.t0 && p > a.b[i]) atomicOr(a.status, kStatusInfeasible);
            } else {
              p = Pc[i];
            }
            const double q = myq[h];
            a.Q[(size_t)c * m + i] = q;
            if (!(isfinite(p) && isfinite(q))) a.bad[par][c] = 1;
            s_rp[slot] = p;
            s_rq[slot] = q;
          }
        }
        __syncthreads();
        // the exact roots of the round's (row, chain) pairs, 32 to a warp: an
        // FP64 instruction costs the SM the same with one lane as with 32
        for (int slot = tid; slot < RW * kFW * CM; slot += kFT) {
          const int c = slot % CM;
          const int i = c < C ? s_ri[slot] : -1;
          if (i < 0) continue;
          double al, be;
          bool inf_row = false;
          if (roots_dp(s_rp[slot], s_rq[slot], a.b[i], al, be, inf_row)) {
            const int j = min(kFB - 1, (int)(al * (1.0 / kFewW)));
            if (be >= (j + 1) * kFewW) {
              atomicMin(&a.bmin[par][(size_t)c * kFB + j],
                        (unsigned long long)__double_as_longlong(al));
              atomicMax(&a.bmax[par][(size_t)c * kFB + j],
                        (unsigned long long)__double_as_longlong(be));
            } else {
              const int at = atomicAdd(&a.nshort[par][c], 1);
              a.shorts[par][((size_t)c * m + at) * 2] = al;
              a.shorts[par][((size_t)c * m + at) * 2 + 1] = be;
            }
          }
          if (inf_row) atomicOr(a.status, kStatusInfeasible);
        }
      }
    }
    if (!grid_barrier(a.bar, a.abort_flag, a.status, a.wait_ns)) return;
    if (t == a.t0 && (*reinterpret_cast<volatile int*>(a.status) & kStatusInfeasible)) return;

    // ---- D: one CTA per chain: sort the arcs, Alg. 3 sweep, theta ----------------
    // with one chain every CTA runs D itself (the same theta everywhere), so
    // E follows without a grid barrier; otherwise CTA c takes chain c
    const bool d_all = C == 1;
    for (int c = d_all ? 0 : blockIdx.x; c < C; c += d_all ? 1 : G) {
      __shared__ int s_part[kFW];
      // the non-empty buckets, in ascending order, as merged arcs
      const int ns = a.nshort[par][c];
      const unsigned long long* bmin = a.bmin[par] + (size_t)c * kFB;
      const unsigned long long* bmax = a.bmax[par] + (size_t)c * kFB;
      constexpr int kPer = kFB / kFT;  // buckets per thread
      static_assert(kFB % kFT == 0, "whole buckets per thread");
      unsigned long long lo_b[kPer], hi_b[kPer];
      int cnt = 0;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        lo_b[k] = bmin[tid * kPer + k];
        hi_b[k] = bmax[tid * kPer + k];
        cnt += lo_b[k] != kEmptyBucket ? 1 : 0;
      }
      const int incl_c = warp_incl_sum<int>(cnt, lane);
      if (lane == 31) s_part[warp] = incl_c;
      __syncthreads();
      int off = incl_c - cnt;
      int nb = 0;
      for (int w = 0; w < kFW; ++w) {
        if (w < warp) off += s_part[w];
        nb += s_part[w];
      }
      const int n = nb + ns;
      int N = 1;
      while (N < n) N <<= 1;
      double* key = sd;
      double* val = sd + (ns > 0 ? N : n);
      __shared__ double s_red[kFW];
      __shared__ int s_best;
      __shared__ double s_theta, s_mid, s_tail_lo, s_total;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        if (lo_b[k] != kEmptyBucket) {
          key[off] = __longlong_as_double((long long)lo_b[k]);
          val[off] = __longlong_as_double((long long)hi_b[k]);
          ++off;
        }
      }
      if (ns > 0) {
        // the short arcs join the list; then one bitonic sort of all of them
        for (int k = tid; k < N - nb; k += kFT) {
          key[nb + k] = k < ns ? a.shorts[par][((size_t)c * m + k) * 2] : INFINITY;
          val[nb + k] = k < ns ? a.shorts[par][((size_t)c * m + k) * 2 + 1] : 0.0;
        }
        __syncthreads();
        for (int kk = 2; kk <= N; kk <<= 1) {
          for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = tid; i < N; i += kFT) {
              const int ix = i ^ jj;
              if (ix > i) {
                const bool up = (i & kk) == 0;
                if ((key[i] > key[ix]) == up) {
                  const double tk = key[i]; key[i] = key[ix]; key[ix] = tk;
                  const double tv = val[i]; val[i] = val[ix]; val[ix] = tv;
                }
              }
            }
            __syncthreads();
          }
        }
      }
      __syncthreads();
      // Alg. 3 over the n merged arcs by the first kDW warps only: an FP64
      // instruction costs the SM the same with any number of lanes, so the
      // sweep runs on few warps with longer segments (E consecutive arcs per
      // thread) while the others wait at the block barriers
      const bool dw = warp < kDW;
      const int E = (n + kDT - 1) / kDT;
      const int lo = dw ? min(n, tid * E) : n, hi = dw ? min(n, lo + E) : n;
      const double eps = a.trim_eps;
      double before = 0.0, gall = 0.0, sloc = 0.0, soff = 0.0, mid = 0.0;
      if (dw) {
        double mloc = 0.0;
        for (int k = lo; k < hi; ++k) mloc = fmax(mloc, val[k]);
        // exclusive max scan of mloc over the threads (gamma before the segment)
        const double incl = warp_incl_max<double>(mloc, lane);
        if (lane == 31) s_red[warp] = incl;
        before = __shfl_up_sync(kFull, incl, 1);
        if (lane == 0) before = 0.0;
      }
      __syncthreads();
      if (dw) {
        for (int w = 0; w < warp; ++w) before = fmax(before, s_red[w]);
        for (int w = 0; w < kDW; ++w) gall = fmax(gall, s_red[w]);
        double g = before;
        for (int k = lo; k < hi; ++k) {
          const double plo = k == 0 ? 0.0 : g + eps, phi = key[k] - eps;
          sloc += phi > plo ? phi - plo : 0.0;
          g = fmax(g, val[k]);
        }
      }
      __syncthreads();
      if (dw) {
        const double sincl = warp_incl_sum<double>(sloc, lane);
        if (lane == 31) s_red[warp] = sincl;
        soff = __shfl_up_sync(kFull, sincl, 1);
        if (lane == 0) soff = 0.0;
      }
      __syncthreads();
      double s = 0.0, tail_len = 0.0;
      if (dw) {
        for (int w = 0; w < kDW; ++w) {
          if (w < warp) soff += s_red[w];
          mid += s_red[w];
        }
        const double tail_lo = n > 0 ? gall + eps : 0.0;
        tail_len = kTwoPi > tail_lo ? kTwoPi - tail_lo : 0.0;
        const double total = mid + tail_len;
        const double u = theta_uniform(a.seed, (uint32_t)c, (uint32_t)t, 0u);
        s = u * total;
        if (tid == 0) {
          s_best = -1;
          s_theta = 0.0;
          s_mid = mid;
          s_tail_lo = tail_lo;
          s_total = total;
        }
      }
      __syncthreads();
      // the last positive piece starting at or below s (the tail is the last)
      if (dw) {
        int cand = -1;
        double gg = before, cum = soff;
        for (int k = lo; k < hi; ++k) {
          const double plo = k == 0 ? 0.0 : gg + eps, phi = key[k] - eps;
          const double len = phi > plo ? phi - plo : 0.0;
          if (len > 0.0 && cum <= s) cand = k;
          cum += len;
          gg = fmax(gg, val[k]);
        }
        if (tid == 0 && tail_len > 0.0 && mid <= s) cand = max(cand, n);
        if (cand >= 0) atomicMax(&s_best, cand);
      }
      __syncthreads();
      const int best = s_best;
      if (dw && best >= 0 && best < n && best >= lo && best < hi) {
        double gg = before, cum = soff;
        for (int k = lo; k <= best; ++k) {
          const double plo = k == 0 ? 0.0 : gg + eps, phi = key[k] - eps;
          const double len = phi > plo ? phi - plo : 0.0;
          if (k == best) {
            const double th = plo + (s - cum);
            s_theta = th < phi ? th : phi;
          }
          cum += len;
          gg = fmax(gg, val[k]);
        }
      }
      if (tid == 0 && best == n) {
        const double th = s_tail_lo + (s - s_mid);
        s_theta = th < kTwoPi ? th : kTwoPi;
      }
      __syncthreads();
      if (tid == 0) {
        double theta = (best < 0 || !(s_total > 0.0)) ? 0.0 : s_theta;
        const bool bad = a.bad[par][c] != 0 || !isfinite(theta);
        if (bad) theta = 0.0;
        double sn, cs;
        sincos(theta, &sn, &cs);
        s_cs[c] = cs;
        s_sn[c] = sn;
        // the outputs: written once (by CTA 0 when every CTA runs D)
        if (!d_all || blockIdx.x == 0) {
          if (bad) {
            a.rej[par][c] = 1;
            atomicAdd(&a.stats->numeric_errors, 1ull);
            atomicOr(a.status, kStatusNumeric);
          }
          a.bad_prev[c] = bad ? 1 : 0;
          a.theta[c] = theta;
          a.cth[c] = cs;
          a.sth[c] = sn;
          sort_keys += n;
        }
      }
      __syncthreads();
    }
    if (!d_all && !grid_barrier(a.bar, a.abort_flag, a.status, a.wait_ns)) return;

    // ---- E: move, FP64 recheck, nu of the next step, per-step state cleared ------
    {
      const double* NU = a.NU[par];
      // cos and sin of each chain's theta: this CTA's own (d_all) or chain c's CTA's
      auto cth = [&](int c) { return d_all ? s_cs[c] : a.cth[c]; };
      auto sth = [&](int c) { return d_all ? s_sn[c] : a.sth[c]; };
      for (long long k = sgtid; k < (long long)C * d; k += gthreads) {
        const int c = (int)(k / d), j = (int)(k % d);
        const size_t o = (size_t)c * d + j;
        const int xbc = xbuf(c);
        a.X[xbc ^ 1][o] = move_d(a.X[xbc][o], NU[o], cth(c), sth(c));
      }
      for (int i = sgwarp; i < m; i += gwarps) {
        const double slack = a.b[i] - a.margin * a.anorm[i];
        bool flag = false;
        if (lane < C) {
          const int c = lane;
          const int xbc = xbuf(c);
          const double pn = fma(a.P[xbc][(size_t)c * m + i], cth(c),
                                a.Q[(size_t)c * m + i] * sth(c));
          a.P[xbc ^ 1][(size_t)c * m + i] = pn;
          flag = !(pn <= slack);
        }
        unsigned ball = __ballot_sync(kFull, flag);
        while (ball) {
          const int c = __ffs(ball) - 1;
          ball &= ball - 1;
          const double* arow = a.A + (size_t)i * d;
          const double* xr = a.X[xbuf(c)] + (size_t)c * d;
          const double* vr = NU + (size_t)c * d;
          const double cs = cth(c), sn = sth(c);
          double acc = 0.0;
          for (int j = lane; j < d; j += 32) acc = fma(arow[j], move_d(xr[j], vr[j], cs, sn), acc);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
          ++rechecks;
          const double res = acc - a.b[i];
          if (lane == 0) {
            atomicMax(&a.stats->max_residual_bits, enc_ordered(res));
            if (res > 0.0) a.rej[par][c] = 1;
          }
        }
      }
      if (t + 1 < a.t0 + a.n_iter) {
        for (long long k = sgtid; k < (long long)C * nblk; k += gthreads) {
          const int c = (int)(k / nblk), n = (int)(k % nblk);
          uint32_t r[4];
          rng_block(a.seed, (uint32_t)n, (uint32_t)c, (uint32_t)(t + 1), 0u, 0u, r);
          box_muller4(r, a.NU[par ^ 1] + (size_t)c * d + 4 * n, min(4, d - 4 * n), a.bm_tab);
        }
      }
    }
    if (!grid_barrier(a.bar, a.abort_flag, a.status, a.wait_ns)) return;
  }

  // ---- end: the final states (and the last record) ------------------------------
  {
    const int par = (a.t0 + a.n_iter) & 1;
    for (long long k = gtid; k < (long long)C * d; k += gthreads) {
      const int c = (int)(k / d), j = (int)(k % d);
      const int xbf = a.cur[par ^ 1][c] ^ (a.rej[par ^ 1][c] ? 0 : 1);
      const double v = a.X[xbf][(size_t)c * d + j];
      a.X_user[(size_t)c * d + j] = v;
      if (a.samples && a.n_iter % a.record_every == 0 && a.n_iter > 0)
        a.samples[((size_t)c * a.n_rec + a.n_iter / a.record_every - 1) * d + j] = v;
    }
    if (gtid == 0) {
      for (int c = 0; c < C; ++c)
        if (a.n_iter > 0 && a.rej[par ^ 1][c] && !a.bad_prev[c]) ++rejections;
    }
  }
  // rechecks were counted by every lane of the warp that did them, rejections
  // by thread 0 of the grid, sort keys by thread 0 of the CTAs of phase D
  if (lane == 0 && rechecks) atomicAdd(&a.stats->rechecks, (unsigned long long)rechecks);
  if (gtid == 0 && rejections) atomicAdd(&a.stats->rejections, (unsigned long long)rejections);
  if (tid == 0 && sort_keys) atomicAdd(&a.stats->sort_keys, (unsigned long long)sort_keys);
}

}  // namespace

size_t few_chains_smem(int C, int m, int chunk) {
  // phase B: nu and x chunks; phase D: the merged buckets and short arcs,
  // padded to a power of two for the sort
  int N = 1;
  while (N < kFB + m) N <<= 1;
  const size_t gemv = (size_t)2 * C * chunk * sizeof(double);
  const size_t sort = (size_t)2 * N * sizeof(double);
  return std::max(gemv, sort);
}

int few_chains_chunk(int C, int d) {
  int chunk = (8192 / std::max(1, C)) / 32 * 32;
  return std::max(32, std::min(chunk, ((d + 31) / 32) * 32));
}

template <int CM>
cudaError_t launch_few_cm(const FewArgs& args, size_t smem, cudaStream_t s) {
  auto k = few_chains_kernel<CM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return cudaErrorNotSupported;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  FewArgs a = args;
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)k, dim3(sms), dim3(kFT), params, smem, s);
}

cudaError_t launch_few_chains(const FewArgs& args, cudaStream_t s) {
  if (args.C < 1 || args.C > kMaxFew || args.m < 1 || args.d < 1 || args.m > kFewMaxM ||
      args.refresh_k < 1 || args.chunk < 32 || (args.samples && args.record_every < 1))
    return cudaErrorInvalidValue;
  const size_t smem = few_chains_smem(args.C, args.m, args.chunk);
  if (args.C <= 1) return launch_few_cm<1>(args, smem, s);
  if (args.C <= 2) return launch_few_cm<2>(args, smem, s);
  if (args.C <= 4) return launch_few_cm<4>(args, smem, s);
  if (args.C <= 8) return launch_few_cm<8>(args, smem, s);
  return launch_few_cm<16>(args, smem, s);
}

}  // namespace ess
