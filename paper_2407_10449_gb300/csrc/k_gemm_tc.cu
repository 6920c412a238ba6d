// k_gemm_tc.cu -- q = A nu on the GB300 tensor cores (tcgen05 + TMA).
//
// The products q_i = a_i . nu of Sec. 2.2 for all chains form one GEMM
// Q (chains x m) = NU (chains x d) . A^T (A: m x d), both operands K-major.
// The mixed form evaluates it with two-way fp16 splits of the float values,
// each scaled by a power of two into the top of the fp16 range (per chain
// t_c for nu, per row s_i for A): nu t_c = h0 + h1 + r, a s_i = a0 + a1 + r',
// |r| <= 2^-22 |nu t_c| + 2^-25.  Three products are kept ("FP16x3"):
//     q ~= (h0.a0 + (h1.a0 + h0.a1)) / (s_i t_c),
// the leading product and the two smaller ones in two FP32 accumulators in
// tensor memory; the dropped h1.a1 is below 2^-22 |a s_i| |nu t_c|.  The same
// kernel, in "pairs" mode, evaluates the exact fixed-point refresh of p = A x
// (see tc_refresh) on bf16 integer slices.
//
// Kernel structure (one 128 x BN output tile per CTA, 6 warps):
//   warp 0 / lane 0   TMA producer: for every (K block, pass) loads the
//                     128 x 64 nu tile and the BN x 64 A tile of that pass
//                     into a ring of shared-memory stages (128-byte swizzle),
//                     completion signalled on the stage's "full" mbarrier;
//   warp 1 / lane 0   MMA issuer: waits "full", issues four
//                     tcgen05.mma.kind::f16 (K = 16 each) into the TMEM
//                     accumulator and commits to the stage's "empty"
//                     mbarrier so the producer can refill it;
//   warps 2..5        epilogue: tcgen05.ld of the accumulator rows (TMEM lane
//                     = chain row, warp w reads lanes 32 (w % 4) ..), the
//                     power-of-two unscaling and 16-byte stores to Q; in pairs
//                     mode they consume each slice pair's accumulator while
//                     the next pair runs in the other TMEM buffer.
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the kernel
// sets kStatusTimeout, drains its own copies, frees TMEM and returns.
#include <cuda.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ess_common.cuh"
#include "ess_gemm_tc.cuh"
#include "tc_ptx.cuh"

namespace ess {
namespace {

constexpr int BM = 128;             // chains per tile (MMA M)
constexpr int BK = 64;              // 16-bit elements per 128-byte swizzle row
constexpr int kThreads = 192;       // producer warp, MMA warp, 4 epilogue warps
constexpr int kRefreshBN = 64;      // tile width of the exact refresh
constexpr int kMaxSlices = 12;      // operand slices of the exact products
constexpr int kMaxRounds = 16;      // rounds of the exact products (<= 8 slice pairs each)
// shared memory of one refresh stage: the x and A slice tiles of one round.
// 64 KB packs the 15 slice pairs of K = 5 into rounds of 5, 7 and 3 pairs and
// leaves room for three stages (the same bytes per tile as two rounds of up
// to 112 KB in two stages, with more of them in flight: 0.73 -> 0.67 ms per
// refresh at 8192 x 2000 x 1000).
constexpr uint32_t kRefreshStage = 64u * 1024u;
// kModeSum: q = A nu (FP16x3).  A stage holds one K block of the two nu
//   slices and the two A slices; three products go into two accumulators.
// kModePairs: exact refresh in rounds of up to 8 slice pairs, each pair in its
//   own 64-column TMEM accumulator; a stage holds one K block of every slice
//   tile the round needs.
enum { kModeSum = 0, kModePairs = 1 };

// Pairs mode: one MMA of x slice tile xs with the na A slice tiles a0 ..
// a0 + na - 1 stacked as one N = 64 na operand, into accumulator blocks
// col .. col + na - 1 (64 columns each; one block per slice pair).
struct RefreshGroup {
  unsigned char xs, a0, na, col;
};
struct RefreshRound {
  unsigned char nx, na, ngroups, npairs;  // x tiles, A tiles, groups, pairs
  unsigned char x[kMaxSlices];            // x slice of each loaded x tile
  unsigned char a[kMaxSlices];            // A slice of each loaded A tile
  RefreshGroup g[8];
  unsigned char shift[8];                 // accumulator block j holds a pair of weight 2^-shift
};

struct TcMaps {
  CUtensorMap x[kMaxSlices];  // chain-side operand slices (M = chains)
  CUtensorMap b[kMaxSlices];  // constraint-side operand slices (N = rows of A)
  CUtensorMap q;              // Q, 32 x 32 fp32 blocks (persistent pair form)
};

struct TcArgs {
  int n_rows, n_cols, kblocks, ngroups;
  int nrounds;                // pairs mode
  RefreshRound round[kMaxRounds];
  float* Q;                   // sum mode output
  int ldq;
  const float* row_scale;     // t_c per chain (sum mode: 1 / t_c, or nullptr: row_const)
  const float* col_scale;     // s_i per constraint (sum mode: 1 / s_i)
  float row_const;            // sum mode: 1 / t_c of every chain when row_scale is null
  float* P32;                 // pairs mode outputs (either may be null)
  double* P64;
  int ldp;
  const float* inv_anorm;     // drift normalisation: 1 / ||a_i|| (0 for a zero row)
  unsigned long long* drift_bits;
  int* status;
};
using namespace tcptx;

// Error-free sum: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// The float f times 2^sh as a double, built from f's bits (exact; no FP64
// instruction): f must be zero or normal and f 2^sh inside double's normal
// range.
__device__ __forceinline__ double f2d_shifted(float f, int sh) {
  const unsigned u = __float_as_uint(f);
  if ((u & 0x7FFFFFFFu) == 0u) return 0.0;
  const unsigned dexp = ((u >> 23) & 0xFFu) + 896u + (unsigned)sh;
  const unsigned hiw = (u & 0x80000000u) | (dexp << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hiw, (int)(u << 29));
}

// (hi + lo) rs cs rounded once to double, where rs and cs are powers of two
// (or zero) and hi, lo the error-free float pair of an exact product: every
// nonzero hi, lo is a multiple of 2^-63 (integers times 2^-shift), hence a
// normal float.  With normal rs and cs the scales go into the exponents by
// integer operations and one FP64 addition rounds (the same double as
// ((double)hi + (double)lo) * rs * cs, whose multiplications are exact);
// otherwise that expression is evaluated as written.  The FP64 pipe of
// GB300 is narrow, and this runs for every entry of an FP64 product.
__device__ __forceinline__ double scaled_pair_sum(float hi, float lo, float rs, float cs) {
  const unsigned ur = __float_as_uint(rs), uc = __float_as_uint(cs);
  const unsigned er = (ur >> 23) & 0xFFu, ec = (uc >> 23) & 0xFFu;
  if (er == 0u || ec == 0u || er == 0xFFu || ec == 0xFFu || (ur & 0x7FFFFFu) != 0u ||
      (uc & 0x7FFFFFu) != 0u)
    return ((double)hi + (double)lo) * (double)rs * (double)cs;
  const int sh = (int)er + (int)ec - 254;  // log2 |rs cs|
  const double v = f2d_shifted(hi, sh) + f2d_shifted(lo, sh);
  return ((ur ^ uc) & 0x80000000u) ? -v : v;
}

template <int BN>
constexpr uint32_t tmem_cols_for(int groups) {
  return groups * BN <= 32 ? 32u : groups * BN <= 64 ? 64u : groups * BN <= 128 ? 128u
         : groups * BN <= 256 ? 256u : 512u;
}

template <int BN, int MODE>
constexpr uint32_t stage_bytes() {
  return MODE == kModeSum ? 2u * (uint32_t)(BM + BN) * BK * 2u : kRefreshStage;
}

template <int BN, int STAGES, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(const __grid_constant__ TcMaps maps, const __grid_constant__ TcArgs args) {
  constexpr uint32_t A_BYTES = BM * BK * 2;
  constexpr uint32_t B_BYTES = BN * BK * 2;
  constexpr uint32_t STAGE_BYTES = stage_bytes<BN, MODE>();
  // sum mode: 2 accumulators of BN columns; pairs mode: 8 blocks of 64 columns
  constexpr uint32_t TMEM_COLS = MODE == kModeSum ? tmem_cols_for<BN>(2) : 512u;
  static_assert(B_BYTES % 1024 == 0, "BN must be a multiple of 8");
  static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "BN in {32, ..., 256}, multiple of 32");

  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars: [0, S) full, [S, 2S) empty, 2S + {0, 1} accumulator full, 2S + {2, 3} accumulator empty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto accf_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto acce_bar = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN;
  const int m0 = blockIdx.y * BM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), 4);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;
  const int kblocks = args.kblocks;

  if (warp == 0 && lane == 0 && MODE == kModeSum) {
    // ---------------- TMA producer (sum mode): 4 tiles per K block ----------------
    bool loaded[STAGES];
    uint32_t last_phase[STAGES];
#pragma unroll
    for (int s = 0; s < STAGES; ++s) loaded[s] = false;
    int s = 0;
    uint32_t phase = 0;
    for (int kb = 0; kb < kblocks; ++kb) {
      if (kb >= STAGES && !mbar_wait(empty_bar(s), phase ^ 1u)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const uint32_t sa = sbase + s * STAGE_BYTES;
      mbar_expect_tx(full_bar(s), STAGE_BYTES);
      tma_load_2d(sa, &maps.x[0], kb * BK, m0, full_bar(s));
      tma_load_2d(sa + A_BYTES, &maps.x[1], kb * BK, m0, full_bar(s));
      tma_load_2d(sa + 2 * A_BYTES, &maps.b[0], kb * BK, n0, full_bar(s));
      tma_load_2d(sa + 2 * A_BYTES + B_BYTES, &maps.b[1], kb * BK, n0, full_bar(s));
      loaded[s] = true;
      last_phase[s] = phase;
      if (++s == STAGES) {
        s = 0;
        phase ^= 1u;
      }
    }
    if (*abort_flag) {
      // let every copy this thread issued land before the CTA exits
#pragma unroll
      for (int j = 0; j < STAGES; ++j)
        if (loaded[j]) (void)mbar_wait(full_bar(j), last_phase[j]);
    }
  } else if (warp == 1 && lane == 0 && MODE == kModeSum) {
    // ---------------- MMA issuer (sum mode) ----------------
    // acc 0 (columns 0 .. BN-1): h0.a0; acc 1 (BN .. 2BN-1): h1.a0 + h0.a1
    constexpr uint32_t idesc = idesc_f16(BM, BN, false);
    int s = 0;
    uint32_t phase = 0;
    for (int kb = 0; kb < kblocks; ++kb) {
      if (!mbar_wait(full_bar(s), phase)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sa = sbase + s * STAGE_BYTES;
      const uint64_t x0 = smem_desc_sw128(sa);
      const uint64_t x1 = smem_desc_sw128(sa + A_BYTES);
      const uint64_t b0 = smem_desc_sw128(sa + 2 * A_BYTES);
      const uint64_t b1 = smem_desc_sw128(sa + 2 * A_BYTES + B_BYTES);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)  // each K = 16 step advances 32 bytes
        umma_bf16(tmem_d, x0 + 2 * k, b0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)
        umma_bf16(tmem_d + BN, x1 + 2 * k, b0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)
        umma_bf16(tmem_d + BN, x0 + 2 * k, b1 + 2 * k, idesc, 1u);
      umma_commit(empty_bar(s));
      if (++s == STAGES) {
        s = 0;
        phase ^= 1u;
      }
    }
    umma_commit(accf_bar(0));
  } else if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (pairs mode): one round after another ----------------
    bool loaded[STAGES];
    uint32_t last_phase[STAGES];
#pragma unroll
    for (int j = 0; j < STAGES; ++j) loaded[j] = false;
    int s = 0, count = 0;
    uint32_t phase = 0;
    for (int r = 0; r < args.nrounds && !*abort_flag; ++r) {
      const RefreshRound& R = args.round[r];
      const uint32_t bytes = R.nx * A_BYTES + R.na * B_BYTES;
      for (int kb = 0; kb < kblocks; ++kb, ++count) {
        if (count >= STAGES && !mbar_wait(empty_bar(s), phase ^ 1u)) {
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        const uint32_t sa = sbase + s * STAGE_BYTES;
        mbar_expect_tx(full_bar(s), bytes);
        for (int i = 0; i < R.nx; ++i)
          tma_load_2d(sa + i * A_BYTES, &maps.x[R.x[i]], kb * BK, m0, full_bar(s));
        for (int j = 0; j < R.na; ++j)
          tma_load_2d(sa + R.nx * A_BYTES + j * B_BYTES, &maps.b[R.a[j]], kb * BK, n0,
                      full_bar(s));
        loaded[s] = true;
        last_phase[s] = phase;
        if (++s == STAGES) {
          s = 0;
          phase ^= 1u;
        }
      }
    }
    if (*abort_flag) {
      // let every copy this thread issued land before the CTA exits
#pragma unroll
      for (int j = 0; j < STAGES; ++j)
        if (loaded[j]) (void)mbar_wait(full_bar(j), last_phase[j]);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer (pairs mode) ----------------
    int s = 0;
    uint32_t phase = 0;
    for (int r = 0; r < args.nrounds; ++r) {
      const RefreshRound& R = args.round[r];
      // the epilogue must have read round r - 1 out of TMEM
      if (r > 0 && !mbar_wait(acce_bar(0), (uint32_t)((r - 1) & 1))) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      bool ok = true;
      for (int kb = 0; kb < kblocks; ++kb) {
        if (!mbar_wait(full_bar(s), phase)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = sbase + s * STAGE_BYTES;
        for (int g = 0; g < R.ngroups; ++g) {
          const RefreshGroup G = R.g[g];
          const uint64_t adesc = smem_desc_sw128(sa + G.xs * A_BYTES);
          const uint64_t bdesc = smem_desc_sw128(sa + R.nx * A_BYTES + G.a0 * B_BYTES);
          const uint32_t idesc = idesc_f16(BM, BN * G.na, true);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)  // each K = 16 step advances 32 bytes
            umma_bf16(tmem_d + (uint32_t)(G.col * BN), adesc + (uint64_t)(2 * k),
                      bdesc + (uint64_t)(2 * k), idesc, (kb == 0 && k == 0) ? 0u : 1u);
        }
        umma_commit(empty_bar(s));
        if (++s == STAGES) {
          s = 0;
          phase ^= 1u;
        }
      }
      if (!ok) {
        *abort_flag = 1;
        break;
      }
      umma_commit(accf_bar(0));
    }
  } else if (warp >= 2) {
    // ---------------- epilogue warps 2..5: TMEM lane quarter warp % 4 ----------------
    const int quarter = warp & 3;
    const int row = m0 + quarter * 32 + lane;
    const uint32_t lane_base = tmem_d + ((uint32_t)(quarter * 32) << 16);
    if constexpr (MODE == kModeSum) {
      const bool ready = mbar_wait(accf_bar(0), 0);
      tc_fence_after();
      if (!ready) *abort_flag = 1;
      const bool row_ok = row < args.n_rows && ready && !*abort_flag;
      float* qrow = args.Q + (size_t)(row_ok ? row : 0) * args.ldq;
      const bool vec_ok = (args.ldq & 3) == 0 && ((reinterpret_cast<uintptr_t>(args.Q) & 15) == 0);
      const float rsc = args.row_scale ? args.row_scale[row_ok ? row : 0] : args.row_const;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        tmem_ld_32cols(lane_base + (uint32_t)c0, v);
        tmem_ld_wait();
        float f[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]);
        if (args.ngroups > 1) {
          tmem_ld_32cols(lane_base + (uint32_t)(BN + c0), v);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 32; ++j) f[j] += __uint_as_float(v[j]);
        }
        if (!row_ok) continue;
        const int col = n0 + c0;
        if (vec_ok && col + 32 <= args.n_cols) {
          // unscale by powers of two (exact): 1 / s_i per column, 1 / t_c per row
          const float4* cs4 = reinterpret_cast<const float4*>(args.col_scale + col);
          float4* dst = reinterpret_cast<float4*>(qrow + col);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 cs = __ldg(cs4 + j);
            dst[j] = make_float4(f[4 * j] * cs.x * rsc, f[4 * j + 1] * cs.y * rsc,
                                 f[4 * j + 2] * cs.z * rsc, f[4 * j + 3] * cs.w * rsc);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col + j < args.n_cols) qrow[col + j] = f[j] * args.col_scale[col + j] * rsc;
        }
      }
    } else {
      // exact integer products of the slice pairs, one 64-column block each,
      // accumulated error-free into (hi, lo) float pairs with the pair's
      // power-of-two weight, round by round
      float hi[BN], lo[BN];
#pragma unroll
      for (int j = 0; j < BN; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
      bool ok = true;
      for (int r = 0; r < args.nrounds; ++r) {
        if (*abort_flag || !mbar_wait(accf_bar(0), (uint32_t)(r & 1))) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const RefreshRound& R = args.round[r];
        for (int pj = 0; pj < R.npairs; ++pj) {
          // 2^-shift as a float (shift <= 126)
          const float w = __uint_as_float((uint32_t)(127 - R.shift[pj]) << 23);
#pragma unroll
          for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            tmem_ld_32cols(lane_base + (uint32_t)(pj * BN + c0), v);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float sum, err;
              two_sum(hi[c0 + j], __uint_as_float(v[j]) * w, sum, err);
              hi[c0 + j] = sum;
              lo[c0 + j] += err;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce_bar(0));
      }
      if (ok && row < args.n_rows) {
        const float rs = args.row_scale[row];
        const size_t base = (size_t)row * args.ldp;
        const bool full = n0 + BN <= args.n_cols;
        if (args.P64) {
          // FP64 product (hi + lo exact in double, scales are powers of two);
          // without a float copy the drift statistic compares the FP64 values,
          // 16 columns at a time (old values loaded before the stores)
          const bool d64 = args.drift_bits != nullptr && args.P32 == nullptr;
          double* prow64 = args.P64 + base + n0;
          double drift64 = 0.0;
#pragma unroll
          for (int j0 = 0; j0 < BN; j0 += 16) {
            double old[16];
            if (d64) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) old[jj] = n0 + j0 + jj < args.n_cols ? prow64[j0 + jj] : 0.0;
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int col = n0 + j0 + jj;
              if (col < args.n_cols) {
                const double v = scaled_pair_sum(hi[j0 + jj], lo[j0 + jj], rs, args.col_scale[col]);
                if (d64) drift64 = fmax(drift64, fabs(v - old[jj]) * (double)args.inv_anorm[col]);
                prow64[j0 + jj] = v;
              }
            }
          }
          if (d64 && drift64 > 0.0)
            atomicMax(args.drift_bits, (unsigned long long)__double_as_longlong(drift64));
        }
        if (args.P32) {
          // p rounded once to float (the scales are powers of two), kept in hi
#pragma unroll
          for (int j = 0; j < BN; ++j) {
            const int col = n0 + j;
            hi[j] = (hi[j] + lo[j]) * rs * (col < args.n_cols ? args.col_scale[col] : 0.f);
          }
          // the drift statistic in FP32 (a diagnostic, far coarser than FP32);
          // every old value is loaded before the first store, so the loads
          // are in flight together
          float* prow = args.P32 + base + n0;
          const bool vec = full && (args.ldp & 3) == 0 && (n0 & 3) == 0 &&
                           (reinterpret_cast<uintptr_t>(args.P32) & 15) == 0;
          float drift = 0.f;
          if (vec) {
            float4* p4 = reinterpret_cast<float4*>(prow);
            if (args.drift_bits) {
              float4 old[BN / 4];
#pragma unroll
              for (int j = 0; j < BN / 4; ++j) old[j] = p4[j];
#pragma unroll
              for (int j = 0; j < BN / 4; ++j) {
                const float* ia = args.inv_anorm + n0 + 4 * j;
                drift = fmaxf(drift, fabsf(hi[4 * j] - old[j].x) * ia[0]);
                drift = fmaxf(drift, fabsf(hi[4 * j + 1] - old[j].y) * ia[1]);
                drift = fmaxf(drift, fabsf(hi[4 * j + 2] - old[j].z) * ia[2]);
                drift = fmaxf(drift, fabsf(hi[4 * j + 3] - old[j].w) * ia[3]);
              }
            }
#pragma unroll
            for (int j = 0; j < BN / 4; ++j)
              p4[j] = make_float4(hi[4 * j], hi[4 * j + 1], hi[4 * j + 2], hi[4 * j + 3]);
          } else {
            if (args.drift_bits) {
#pragma unroll
              for (int j = 0; j < BN; ++j)
                lo[j] = n0 + j < args.n_cols ? prow[j] : 0.f;
#pragma unroll
              for (int j = 0; j < BN; ++j)
                if (n0 + j < args.n_cols)
                  drift = fmaxf(drift, fabsf(hi[j] - lo[j]) * args.inv_anorm[n0 + j]);
            }
#pragma unroll
            for (int j = 0; j < BN; ++j)
              if (n0 + j < args.n_cols) prow[j] = hi[j];
          }
          if (args.drift_bits && drift > 0.f)
            atomicMax(args.drift_bits, (unsigned long long)__double_as_longlong((double)drift));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(args.status, kStatusTimeout);
  if (warp == 0) tmem_dealloc(tmem_d, TMEM_COLS);
}


// ---- q = A nu on SM pairs (tcgen05 cta_group::2) --------------------------------
// The same FP16x3 sum as tc_gemm_kernel's sum mode, with one 256 x BN output
// tile per cluster of two CTAs on two SMs.  CTA rank r holds chains
// m0 + 128 r .. m0 + 128 r + 127 (its half of the MMA's M = 256) and rows
// n0 + (BN / 2) r .. of A (its half of N); the leader (rank 0) issues
// tcgen05.mma.cta_group::2, which reads both CTAs' shared memory at the same
// offsets and writes each CTA's 128 accumulator lanes to its own TMEM.  Per
// SM this loads (2 x 128 + BN) x 64 x 2 bytes per K block for a 128 x BN
// output, against (2 x 128 + 2 BN) x 64 x 2 in the one-SM form: the L2 reads
// and the tensor core's shared-memory reads of A fall by half.
//   both CTAs, warp 0 / lane 0: TMA producer of the CTA's own tiles; every
//     copy signals the leader's "full" barrier (the leader arms it with the
//     bytes of both CTAs); a stage is refilled after the MMA's commit has
//     arrived on the CTA's own "empty" barrier (multicast to both CTAs);
//   leader, warp 1 / lane 0: MMA issuer; commits multicast to both CTAs;
//   both CTAs, warps 2..5: epilogue of the CTA's 128 chains (as in the
//     one-SM form).
// Waits are bounded as in tc_gemm_kernel; on expiry the CTA sets
// kStatusTimeout, the leader waits (bounded) for the copies it armed, and both
// CTAs meet at a cluster barrier before TMEM is freed.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(local), "r"(rank));
  return a;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

// TMA load into this CTA's shared memory, completion counted on the barrier at
// cluster address bar (the leader's, for cta_group::2 consumers).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x,
                                                 int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void umma_f16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on the barrier at the same shared-memory offset in both CTAs of
// the pair when this thread's earlier MMAs have completed.
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .b16 m;\n\tmov.b16 m, 3;\n\t"
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], m;\n\t}\n" ::"r"(bar)
      : "memory");
}

template <int BN>
constexpr uint32_t pair_stage_bytes() {
  return 2u * (uint32_t)BM * BK * 2u + 2u * (uint32_t)(BN / 2) * BK * 2u;
}

template <int BN, int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
tc_gemm_pair_kernel(const __grid_constant__ TcMaps maps, const __grid_constant__ TcArgs args) {
  constexpr uint32_t A_BYTES = BM * BK * 2;                 // one chain-side slice tile
  constexpr uint32_t B_BYTES = (BN / 2) * BK * 2;           // this CTA's half of an A slice tile
  constexpr uint32_t STAGE_BYTES = pair_stage_bytes<BN>();
  constexpr uint32_t TMEM_COLS = tmem_cols_for<BN>(2);
  static_assert(B_BYTES % 1024 == 0, "BN / 2 must be a multiple of 8");
  static_assert(BN % 32 == 0 && BN >= 64 && BN <= 256, "BN in {64, ..., 256}, multiple of 32");

  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  // a spare half tile after the stages keeps every operand read of the last
  // stage inside the tile area
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + B_BYTES);
  // bars: [0, S) full (used in the leader), [S, 2S) empty, 2S accumulator full
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  const uint32_t accf = smem_u32(bars + 2 * STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int n0 = (blockIdx.x >> 1) * BN;
  const int m0 = blockIdx.y * (2 * BM) + (int)rank * BM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(accf, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    // one warp of each CTA of the pair allocates (the same columns in both)
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync_all();  // barriers of both CTAs initialised, TMEM address visible
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;
  const int kblocks = args.kblocks;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    const uint32_t full0 = cluster_addr(full_bar(0), 0);  // the leader's barriers
    bool armed[STAGES];
    uint32_t armed_phase[STAGES];
#pragma unroll
    for (int s = 0; s < STAGES; ++s) armed[s] = false;
    int s = 0;
    uint32_t phase = 0;
    for (int kb = 0; kb < kblocks; ++kb) {
      if (kb >= STAGES && !mbar_wait(empty_bar(s), phase ^ 1u)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const uint32_t sa = sbase + s * STAGE_BYTES;
      const uint32_t fb = full0 + (uint32_t)s * 8u;
      if (leader) {
        mbar_expect_tx(full_bar(s), 2u * STAGE_BYTES);
        armed[s] = true;
        armed_phase[s] = phase;
      }
      tma_load_2d_pair(sa, &maps.x[0], kb * BK, m0, fb);
      tma_load_2d_pair(sa + A_BYTES, &maps.x[1], kb * BK, m0, fb);
      tma_load_2d_pair(sa + 2 * A_BYTES, &maps.b[0], kb * BK, n0 + (int)rank * (BN / 2), fb);
      tma_load_2d_pair(sa + 2 * A_BYTES + B_BYTES, &maps.b[1], kb * BK, n0 + (int)rank * (BN / 2),
                       fb);
      if (++s == STAGES) {
        s = 0;
        phase ^= 1u;
      }
    }
    if (*abort_flag && leader) {
      // the copies of both CTAs complete on the leader's barriers
#pragma unroll
      for (int j = 0; j < STAGES; ++j)
        if (armed[j]) (void)mbar_wait(full_bar(j), armed_phase[j]);
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (leader) ----------------
    // acc 0 (columns 0 .. BN-1): h0.a0; acc 1 (BN .. 2BN-1): h1.a0 + h0.a1
    constexpr uint32_t idesc = idesc_f16(2 * BM, BN, false);
    int s = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int kb = 0; kb < kblocks; ++kb) {
      if (!mbar_wait(full_bar(s), phase)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = sbase + s * STAGE_BYTES;
      const uint64_t x0 = smem_desc_sw128(sa);
      const uint64_t x1 = smem_desc_sw128(sa + A_BYTES);
      const uint64_t b0 = smem_desc_sw128(sa + 2 * A_BYTES);
      const uint64_t b1 = smem_desc_sw128(sa + 2 * A_BYTES + B_BYTES);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)  // each K = 16 step advances 32 bytes
        umma_f16_pair(tmem_d, x0 + 2 * k, b0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)
        umma_f16_pair(tmem_d + BN, x1 + 2 * k, b0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)
        umma_f16_pair(tmem_d + BN, x0 + 2 * k, b1 + 2 * k, idesc, 1u);
      umma_commit_pair(empty_bar(s));
      if (++s == STAGES) {
        s = 0;
        phase ^= 1u;
      }
    }
    if (ok) umma_commit_pair(accf);
    else *abort_flag = 1;
  } else if (warp >= 2) {
    // ---------------- epilogue warps 2..5: TMEM lane quarter warp % 4 ----------------
    const int quarter = warp & 3;
    const int row = m0 + quarter * 32 + lane;
    const uint32_t lane_base = tmem_d + ((uint32_t)(quarter * 32) << 16);
    const bool ready = mbar_wait(accf, 0);
    tc_fence_after();
    if (!ready) *abort_flag = 1;
    const bool row_ok = row < args.n_rows && ready && !*abort_flag;
    float* qrow = args.Q + (size_t)(row_ok ? row : 0) * args.ldq;
    const bool vec_ok = (args.ldq & 3) == 0 && ((reinterpret_cast<uintptr_t>(args.Q) & 15) == 0);
    const float rsc = args.row_scale ? args.row_scale[row_ok ? row : 0] : args.row_const;
    if (ready) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        tmem_ld_32cols(lane_base + (uint32_t)c0, v);
        tmem_ld_wait();
        float f[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]);
        tmem_ld_32cols(lane_base + (uint32_t)(BN + c0), v);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) f[j] += __uint_as_float(v[j]);
        if (!row_ok) continue;
        const int col = n0 + c0;
        if (vec_ok && col + 32 <= args.n_cols) {
          // unscale by powers of two (exact): 1 / s_i per column, 1 / t_c per row
          const float4* cs4 = reinterpret_cast<const float4*>(args.col_scale + col);
          float4* dst = reinterpret_cast<float4*>(qrow + col);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 cs = __ldg(cs4 + j);
            dst[j] = make_float4(f[4 * j] * cs.x * rsc, f[4 * j + 1] * cs.y * rsc,
                                 f[4 * j + 2] * cs.z * rsc, f[4 * j + 3] * cs.w * rsc);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col + j < args.n_cols) qrow[col + j] = f[j] * args.col_scale[col + j] * rsc;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    // a copy of this CTA may still target its shared memory (the leader's
    // drain above covers only the stages it armed): give it time to land
    if (threadIdx.x == 0) atomicOr(args.status, kStatusTimeout);
    for (int i = 0; i < 1000; ++i) __nanosleep(1000);
  }
  cluster_sync_all();  // the leader's MMAs no longer read the peer's shared memory
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_d),
                 "r"(TMEM_COLS)
                 : "memory");
}

// ---- q = A nu on SM pairs, persistent ---------------------------------------------
// The SM-pair form of tc_gemm_pair_kernel with one cluster per SM pair looping
// over the 256 x BN output tiles (tile cid, cid + nclusters, ...).  The
// producers stream the K blocks of consecutive tiles through the stage ring
// without a break; the MMA issuer starts a tile as soon as both CTAs'
// epilogues have read the previous accumulators out of TMEM (the leader's
// "accumulator empty" barrier, one arrival per epilogue warp of either CTA);
// the epilogue writes each 32 x 32 block of Q through a 128-byte-swizzled
// shared staging buffer (two per warp) and a TMA store, so that its global
// writes overlap the next tile's loads and MMAs.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar)
               : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(src)
      : "memory");
}

constexpr uint32_t kStageQ = 32u * 32u * 4u;  // one 32 x 32 fp32 block of Q

template <int BN, int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
tc_gemm_pair_persistent_kernel(const __grid_constant__ TcMaps maps,
                               const __grid_constant__ TcArgs args) {
  constexpr uint32_t A_BYTES = BM * BK * 2;
  constexpr uint32_t B_BYTES = (BN / 2) * BK * 2;
  constexpr uint32_t STAGE_BYTES = pair_stage_bytes<BN>();
  constexpr uint32_t TMEM_COLS = tmem_cols_for<BN>(2);
  static_assert(B_BYTES % 1024 == 0, "BN / 2 must be a multiple of 8");
  static_assert(BN % 32 == 0 && BN >= 64 && BN <= 256, "BN in {64, ..., 256}, multiple of 32");

  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  // [stages][4 warps x 2 Q staging blocks][barriers]
  const uint32_t qstage = sbase + STAGES * STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + 8 * kStageQ);
  // bars: [0, S) full (leader), [S, 2S) empty, 2S accumulator full, 2S + 1 accumulator empty (leader)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  const uint32_t accf = smem_u32(bars + 2 * STAGES);
  const uint32_t acce = smem_u32(bars + 2 * STAGES + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int cid = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
  const int ncol = (args.n_cols + BN - 1) / BN;
  const int ntiles = ncol * ((args.n_rows + 2 * BM - 1) / (2 * BM));
  const int kblocks = args.kblocks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 8);  // 4 epilogue warps in each CTA of the pair
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs), K blocks of every tile ----------------
    const uint32_t full0 = cluster_addr(full_bar(0), 0);
    bool armed[STAGES];
    uint32_t armed_phase[STAGES];
#pragma unroll
    for (int s = 0; s < STAGES; ++s) armed[s] = false;
    int s = 0, count = 0;
    uint32_t phase = 0;
    for (int t = cid; t < ntiles && !*abort_flag; t += nclusters) {
      const int m0 = (t / ncol) * (2 * BM) + (int)rank * BM;
      const int nb = (t % ncol) * BN + (int)rank * (BN / 2);
      for (int kb = 0; kb < kblocks; ++kb, ++count) {
        if (count >= STAGES && !mbar_wait(empty_bar(s), phase ^ 1u)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t sa = sbase + s * STAGE_BYTES;
        const uint32_t fb = full0 + (uint32_t)s * 8u;
        if (leader) {
          mbar_expect_tx(full_bar(s), 2u * STAGE_BYTES);
          armed[s] = true;
          armed_phase[s] = phase;
        }
        tma_load_2d_pair(sa, &maps.x[0], kb * BK, m0, fb);
        tma_load_2d_pair(sa + A_BYTES, &maps.x[1], kb * BK, m0, fb);
        tma_load_2d_pair(sa + 2 * A_BYTES, &maps.b[0], kb * BK, nb, fb);
        tma_load_2d_pair(sa + 2 * A_BYTES + B_BYTES, &maps.b[1], kb * BK, nb, fb);
        if (++s == STAGES) {
          s = 0;
          phase ^= 1u;
        }
      }
    }
    if (*abort_flag && leader) {
#pragma unroll
      for (int j = 0; j < STAGES; ++j)
        if (armed[j]) (void)mbar_wait(full_bar(j), armed_phase[j]);
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (leader) ----------------
    constexpr uint32_t idesc = idesc_f16(2 * BM, BN, false);
    int s = 0, j = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += nclusters, ++j) {
      // both epilogues have read tile j - 1 out of TMEM
      if (j > 0 && !mbar_wait(acce, (uint32_t)((j - 1) & 1))) {
        ok = false;
        break;
      }
      tc_fence_after();
      for (int kb = 0; kb < kblocks; ++kb) {
        if (!mbar_wait(full_bar(s), phase)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = sbase + s * STAGE_BYTES;
        const uint64_t x0 = smem_desc_sw128(sa);
        const uint64_t x1 = smem_desc_sw128(sa + A_BYTES);
        const uint64_t b0 = smem_desc_sw128(sa + 2 * A_BYTES);
        const uint64_t b1 = smem_desc_sw128(sa + 2 * A_BYTES + B_BYTES);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          umma_f16_pair(tmem_d, x0 + 2 * k, b0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          umma_f16_pair(tmem_d + BN, x1 + 2 * k, b0 + 2 * k, idesc,
                        (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          umma_f16_pair(tmem_d + BN, x0 + 2 * k, b1 + 2 * k, idesc, 1u);
        umma_commit_pair(empty_bar(s));
        if (++s == STAGES) {
          s = 0;
          phase ^= 1u;
        }
      }
      if (ok) umma_commit_pair(accf);
    }
    if (!ok) *abort_flag = 1;
  } else if (warp >= 2) {
    // ---------------- epilogue warps 2..5: TMEM lane quarter warp % 4 ----------------
    const int quarter = warp & 3;
    const uint32_t lane_base = tmem_d + ((uint32_t)(quarter * 32) << 16);
    const uint32_t acce0 = cluster_addr(acce, 0);
    const uint32_t my_q = qstage + (uint32_t)(warp - 2) * 2u * kStageQ;
    const uint32_t sw = (uint32_t)(lane & 7);  // 128-byte swizzle of row `lane`
    int j = 0, buf = 0;
    for (int t = cid; t < ntiles; t += nclusters, ++j) {
      const bool ready = !*abort_flag && mbar_wait(accf, (uint32_t)(j & 1));
      tc_fence_after();
      if (!ready) {
        *abort_flag = 1;
        break;
      }
      const int r0 = (t / ncol) * (2 * BM) + (int)rank * BM + quarter * 32;
      const int n0 = (t % ncol) * BN;
      const int row = r0 + lane;
      const float rsc = args.row_scale ? args.row_scale[row < args.n_rows ? row : 0]
                                       : args.row_const;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32], w[32];
        tmem_ld_32cols(lane_base + (uint32_t)c0, v);
        tmem_ld_32cols(lane_base + (uint32_t)(BN + c0), w);
        tmem_ld_wait();
        if (c0 + 32 >= BN) {
          // the accumulators of this tile are in registers: release TMEM
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(acce0);
        }
        // the staging block written two chunks ago has been read by its TMA store
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
        const uint32_t dst = my_q + (uint32_t)buf * kStageQ + (uint32_t)lane * 128u;
        const int col = n0 + c0;
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4) {
          // 1 / s_i per column (zero past the last row of A), 1 / t_c per row:
          // powers of two, so the scaling is exact
          float4 cs;
          const int cq = col + 4 * q4;
          if (cq + 4 <= args.n_cols) {
            cs = __ldg(reinterpret_cast<const float4*>(args.col_scale + col) + q4);
          } else {
            cs.x = cq < args.n_cols ? args.col_scale[cq] : 0.f;
            cs.y = cq + 1 < args.n_cols ? args.col_scale[cq + 1] : 0.f;
            cs.z = cq + 2 < args.n_cols ? args.col_scale[cq + 2] : 0.f;
            cs.w = cq + 3 < args.n_cols ? args.col_scale[cq + 3] : 0.f;
          }
          const float o0 = (__uint_as_float(v[4 * q4]) + __uint_as_float(w[4 * q4])) * cs.x * rsc;
          const float o1 =
              (__uint_as_float(v[4 * q4 + 1]) + __uint_as_float(w[4 * q4 + 1])) * cs.y * rsc;
          const float o2 =
              (__uint_as_float(v[4 * q4 + 2]) + __uint_as_float(w[4 * q4 + 2])) * cs.z * rsc;
          const float o3 =
              (__uint_as_float(v[4 * q4 + 3]) + __uint_as_float(w[4 * q4 + 3])) * cs.w * rsc;
          const uint32_t a = dst + (((uint32_t)q4 ^ sw) << 4);
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(o0), "f"(o1),
                       "f"(o2), "f"(o3)
                       : "memory");
        }
        // make the generic-proxy writes visible to the TMA engine, then store
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&maps.q, col, r0, my_q + (uint32_t)buf * kStageQ);
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        buf ^= 1;
      }
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicOr(args.status, kStatusTimeout);
    for (int i = 0; i < 1000; ++i) __nanosleep(1000);
  }
  cluster_sync_all();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_d),
                 "r"(TMEM_COLS)
                 : "memory");
}

// ---- q = A_p nu for a batch of problems (tcgen05, one SM per work item) --------
// Work item: rows row0 .. row0 + 127 of one problem's A_p against one group of
// up to 64 of its chains (N = the group's chain count rounded up to 16).  The
// FP16x3 products of the one-problem form (h0.a0 into one accumulator,
// h1.a0 + h0.a1 into a second) with the roles swapped: the MMA's M side is the
// rows of A_p (TMEM lane = row), its N side the chains, so that the epilogue
// writes each chain's q as 32 consecutive floats per warp.  One persistent CTA
// per SM walks the items b, b + G, b + 2G, ... (the host sorts them largest
// first); the producer streams the K blocks of consecutive items through a
// ring of stages without a break, and two TMEM accumulator pairs let the
// epilogue of one item overlap the MMAs of the next.  Operand tiles come from
// per-problem tensor maps (128-byte swizzle, zero fill past d_p, m_p and the
// chain count).
constexpr int kBqStageBytes = 2 * 128 * 64 * 2 + 2 * 64 * 64 * 2;  // two A and two nu tiles
constexpr int kBqStages = 4;

__global__ void __launch_bounds__(kThreads, 1)
tc_batch_q_kernel(const TcBatchItem* __restrict__ items, int n_items,
                  const CUtensorMap* __restrict__ maps, const float* __restrict__ arow_unscale,
                  const float* __restrict__ chain_unscale, float* __restrict__ Q, int* status) {
  constexpr uint32_t A_BYTES = 128 * 64 * 2;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kBqStages * kBqStageBytes);
  // bars: [0, S) full, [S, 2S) empty, 2S + {0, 1} accumulator full, 2S + {2, 3} accumulator empty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kBqStages + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + kBqStages + s); };
  auto accf_bar = [&](int b) { return smem_u32(bars + 2 * kBqStages + b); };
  auto acce_bar = [&](int b) { return smem_u32(bars + 2 * kBqStages + 2 + b); };
  constexpr uint32_t TMEM_COLS = 256;  // two buffers x (two accumulators x 64 columns)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kBqStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), 4);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    bool loaded[kBqStages];
    uint32_t last_phase[kBqStages];
#pragma unroll
    for (int j = 0; j < kBqStages; ++j) loaded[j] = false;
    int s = 0, count = 0;
    uint32_t phase = 0;
    for (int it = blockIdx.x; it < n_items && !*abort_flag; it += gridDim.x) {
      const TcBatchItem I = items[it];
      const CUtensorMap* mp = maps + 4 * I.problem;
      const uint32_t bytes = 2u * A_BYTES + 2u * (uint32_t)I.ntile * 128u;
      for (int kb = 0; kb < I.kblocks; ++kb, ++count) {
        if (count >= kBqStages && !mbar_wait(empty_bar(s), phase ^ 1u)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t sa = sbase + s * kBqStageBytes;
        mbar_expect_tx(full_bar(s), bytes);
        tma_load_2d(sa, mp + 0, kb * BK, I.row0, full_bar(s));
        tma_load_2d(sa + A_BYTES, mp + 1, kb * BK, I.row0, full_bar(s));
        tma_load_2d(sa + 2 * A_BYTES, mp + 2, kb * BK, I.chain0, full_bar(s));
        tma_load_2d(sa + 2 * A_BYTES + (uint32_t)I.ntile * 128u, mp + 3, kb * BK, I.chain0,
                    full_bar(s));
        loaded[s] = true;
        last_phase[s] = phase;
        if (++s == kBqStages) {
          s = 0;
          phase ^= 1u;
        }
      }
    }
    if (*abort_flag) {
#pragma unroll
      for (int j = 0; j < kBqStages; ++j)
        if (loaded[j]) (void)mbar_wait(full_bar(j), last_phase[j]);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int s = 0, j = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++j) {
      const TcBatchItem I = items[it];
      const int buf = j & 1;
      // the epilogue has read this buffer's previous item (item j - 2)
      if (j >= 2 && !mbar_wait(acce_bar(buf), (uint32_t)(((j - 2) >> 1) & 1))) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t idesc = idesc_f16(128, I.ntile, false);
      const uint32_t acc0 = tmem_d + (uint32_t)(buf * 128), acc1 = acc0 + 64;
      for (int kb = 0; kb < I.kblocks; ++kb) {
        if (!mbar_wait(full_bar(s), phase)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = sbase + s * kBqStageBytes;
        const uint64_t a0 = smem_desc_sw128(sa);
        const uint64_t a1 = smem_desc_sw128(sa + A_BYTES);
        const uint64_t h0 = smem_desc_sw128(sa + 2 * A_BYTES);
        const uint64_t h1 = smem_desc_sw128(sa + 2 * A_BYTES + (uint32_t)I.ntile * 128u);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          umma_bf16(acc0, a0 + 2 * k, h0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          umma_bf16(acc1, a1 + 2 * k, h0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          umma_bf16(acc1, a0 + 2 * k, h1 + 2 * k, idesc, 1u);
        umma_commit(empty_bar(s));
        if (++s == kBqStages) {
          s = 0;
          phase ^= 1u;
        }
      }
      if (ok) umma_commit(accf_bar(buf));
    }
    if (!ok) *abort_flag = 1;
  } else if (warp >= 2) {
    // ---------------- epilogue warps 2..5: TMEM lane quarter warp % 4 ----------------
    const int quarter = warp & 3;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    int j = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x, ++j) {
      const int buf = j & 1;
      const bool ready = !*abort_flag && mbar_wait(accf_bar(buf), (uint32_t)((j >> 1) & 1));
      tc_fence_after();
      if (!ready) {
        *abort_flag = 1;
        break;
      }
      const TcBatchItem I = items[it];
      const int r = quarter * 32 + lane;  // row within the item
      const bool row_ok = r < I.rows;
      const float ru = row_ok ? arow_unscale[I.urow + r] : 0.f;
      const uint32_t acc0 = tmem_d + lane_off + (uint32_t)(buf * 128), acc1 = acc0 + 64;
      // all of this item's accumulators in registers first (<= 64 columns)
      float qv[64];
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 32) {
        if (c0 < I.ntile) {
          uint32_t v[32], w[32];
          tmem_ld_32cols(acc0 + (uint32_t)c0, v);
          tmem_ld_32cols(acc1 + (uint32_t)c0, w);
          tmem_ld_wait();
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) qv[c0 + jj] = __uint_as_float(v[jj]) + __uint_as_float(w[jj]);
        }
      }
      // TMEM buffer free for the item after next
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce_bar(buf));
      if (row_ok) {
        float* qrow = Q + I.q_off + I.row0 + r;  // chain c of the item at qrow[c * m]
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          if (c < I.chains) {
            const float cu = chain_unscale ? chain_unscale[I.c_first + c] : 1.f / kNuSplitScale;
            qrow[(size_t)c * I.m] = qv[c] * ru * cu;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, kStatusTimeout);
  if (warp == 0) tmem_dealloc(tmem_d, TMEM_COLS);
}

// Fixed-point slices of the chain states for the exact refresh: per row c,
// t_c = 2^e with max_j |x_cj| < t_c, and x_cj / t_c = sum_l e_l 2^(-w l) + r,
// e_l integers in (-2^w, 2^w) stored exactly as bf16.  One warp per row.
template <typename TI>
__global__ void slice_rows_kernel(const TI* __restrict__ X, int ldx, int rows, int d, int w,
                                  int K, __nv_bfloat16* __restrict__ slices, int ld_bf,
                                  size_t slice_stride, float* __restrict__ row_scale) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const TI* x = X + (size_t)row * ldx;
  TI mx = TI(0);
  bool nonfinite = false;
  for (int j = lane; j < d; j += 32) {
    mx = fmax(mx, fabs(x[j]));
    nonfinite |= !isfinite(x[j]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  nonfinite = __any_sync(0xffffffffu, nonfinite);
  int e = 0;
  if (mx > TI(0) && !nonfinite) (void)frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1): mx < 2^e
  const TI inv_t = ldexp(TI(1), -e);
  // a row with NaN or Inf gets a NaN scale: its slices carry no meaning, and
  // every product of the row comes out NaN (the epilogue multiplies by it)
  if (lane == 0) row_scale[row] = nonfinite ? __int_as_float(0x7FC00000) : mx > TI(0) ? ldexpf(1.f, e) : 0.f;
  if constexpr (sizeof(TI) == 8) {
    if (w * K <= 63) {
      // FP64 rows: |y| < 1, so |y| 2^63 converts exactly to an integer in its
      // top 60 bits (the bits below 2^-63 are below every slice), and slice l
      // is the bit field [63 - w (l + 1), 63 - w l) of it with the sign of y:
      // the same integers as the loop below, with one FP64 conversion per
      // entry instead of three FP64 operations per slice
      const unsigned long long mask = (1ull << w) - 1ull;
      for (int j = lane; j < d; j += 32) {
        const double y = x[j] * inv_t;  // exact: power-of-two scaling
        const unsigned long long Y = (unsigned long long)(fabs(y) * 9223372036854775808.0);
        const bool neg = y < 0.0;
        for (int l = 0; l < K; ++l) {
          const int v = (int)((Y >> (63 - w * (l + 1))) & mask);
          slices[(size_t)l * slice_stride + (size_t)row * ld_bf + j] =
              __float2bfloat16_rn((float)(neg ? -v : v));
        }
      }
      return;
    }
  }
  const TI up = ldexp(TI(1), w);
  for (int j = lane; j < d; j += 32) {
    TI y = x[j] * inv_t;  // exact: power-of-two scaling
    for (int l = 0; l < K; ++l) {
      y *= up;
      const TI c = trunc(y);  // an integer of at most w bits: exact in bf16
      y -= c;
      slices[(size_t)l * slice_stride + (size_t)row * ld_bf + j] = __float2bfloat16_rn((float)c);
    }
  }
}

// Scaled two-way fp16 split of float rows, one warp per row: t = 2^(15 - e)
// with max_j |v_j| in [2^(e-1), 2^e), so every v_j t lies below 2^15, and
// v_j t = h0 + h1 + r with h0 = fp16(v_j t), h1 = fp16(v_j t - h0) (the
// subtraction is exact).  unscale[row] = 1 / t (0 for an all-zero row).
__global__ void split2_rows_kernel(const float* __restrict__ src, int ld, int rows, int cols,
                                   __half* __restrict__ h0, __half* __restrict__ h1, int ld_h,
                                   float* __restrict__ unscale) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float* v = src + (size_t)row * ld;
  float mx = 0.f;
  for (int j = lane; j < cols; j += 32) mx = fmaxf(mx, fabsf(v[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int e = 0;
  if (mx > 0.f) (void)frexpf(mx, &e);
  const float t = mx > 0.f ? ldexpf(1.f, 15 - e) : 1.f;
  if (lane == 0) unscale[row] = mx > 0.f ? ldexpf(1.f, e - 15) : 0.f;
  const size_t o = (size_t)row * ld_h;
  for (int j = lane; j < cols; j += 32) {
    const float y = v[j] * t;
    const __half a = __float2half_rn(y);
    h0[o + j] = a;
    h1[o + j] = __float2half_rn(y - __half2float(a));
  }
}

// ---- host side ---------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D tensor map of 16-bit elements (bf16 or fp16) over a rows x cols matrix
// (row stride ld elements), box = box_rows x 64 columns, 128-byte swizzle,
// zero fill out of bounds.
cudaError_t make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld,
                     int box_rows, bool bf16 = true) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 2) % 16 != 0)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                  2, const_cast<void*>(base), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 2-D tensor map of a float matrix (rows x cols, row stride ld elements) for
// TMA stores of 32 x 32 blocks with the 128-byte swizzle.
cudaError_t make_map_q(CUtensorMap* map, void* base, int rows, int cols, int ld) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 4) % 16 != 0)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kSmemLimit = 227 * 1024;

template <int BN, int MODE = kModeSum>
constexpr int stages_for() {
  constexpr int stage = (int)stage_bytes<BN, MODE>();
  constexpr int s = (kSmemLimit - 1024 - 256) / stage;
  return s > 6 ? 6 : s;
}

template <int BN, int MODE>
size_t smem_for() {
  return (size_t)stages_for<BN, MODE>() * stage_bytes<BN, MODE>() + 1024 + 256;
}

template <int BN, int MODE>
cudaError_t launch_bn(const TcMaps& maps, const TcArgs& args, cudaStream_t s) {
  constexpr int ST = stages_for<BN, MODE>();
  auto k = tc_gemm_kernel<BN, ST, MODE>;
  const size_t smem = smem_for<BN, MODE>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((args.n_cols + BN - 1) / BN, (args.n_rows + BM - 1) / BM);
  k<<<grid, kThreads, smem, s>>>(maps, args);
  return cudaGetLastError();
}

const int kWidths[6] = {64, 128, 160, 192, 224, 256};
// SM-pair tiles: 256 chains x BN rows of A, reported as kPairCode + BN
constexpr int kPairCode = 2000;
const int kPairWidths[5] = {128, 160, 192, 224, 256};

// Shared memory of the pair kernel: the stages, then one spare half tile of A
// (BN / 2 rows), then the barriers.
template <int BN>
constexpr size_t pair_smem_bytes(int stages) {
  return (size_t)stages * pair_stage_bytes<BN>() + (size_t)(BN / 2) * BK * 2 + 1024 + 256;
}

template <int BN>
constexpr int pair_stages() {
  constexpr int s = (kSmemLimit - 1024 - 256 - (BN / 2) * BK * 2) / (int)pair_stage_bytes<BN>();
  return s > 6 ? 6 : s;
}

template <int BN>
cudaError_t launch_pair_bn(const TcMaps& maps, const TcArgs& args, cudaStream_t s) {
  constexpr int ST = pair_stages<BN>();
  auto k = tc_gemm_pair_kernel<BN, ST>;
  const size_t smem = pair_smem_bytes<BN>(ST);
  static_assert(pair_smem_bytes<BN>(ST) <= (size_t)kSmemLimit, "pair kernel shared memory");
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // x: two CTAs (one cluster) per column tile; y: 256 chains per cluster
  dim3 grid(2 * ((args.n_cols + BN - 1) / BN), (args.n_rows + 2 * BM - 1) / (2 * BM));
  k<<<grid, kThreads, smem, s>>>(maps, args);
  return cudaGetLastError();
}

int num_sms();

// Persistent SM-pair form: one cluster of two CTAs per co-resident slot.
constexpr int kPersistCode = 3000;

template <int BN>
constexpr int persist_stages() {
  constexpr int s = (kSmemLimit - 1024 - 256 - 8 * (int)kStageQ) / (int)pair_stage_bytes<BN>();
  return s > 6 ? 6 : s;
}

template <int BN>
constexpr size_t persist_smem_bytes() {
  return (size_t)persist_stages<BN>() * pair_stage_bytes<BN>() + 8 * kStageQ + 1024 + 256;
}

template <int BN>
cudaError_t launch_persist_bn(const TcMaps& maps, const TcArgs& args, cudaStream_t s) {
  constexpr int ST = persist_stages<BN>();
  static_assert(persist_smem_bytes<BN>() <= (size_t)kSmemLimit, "persistent pair shared memory");
  auto k = tc_gemm_pair_persistent_kernel<BN, ST>;
  const size_t smem = persist_smem_bytes<BN>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ntiles = ((args.n_cols + BN - 1) / BN) * ((args.n_rows + 2 * BM - 1) / (2 * BM));
  // co-resident clusters of this configuration (cached per width)
  static int max_clusters = 0;
  if (max_clusters == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess || n < 1) {
      (void)cudaGetLastError();
      n = std::max(1, num_sms() / 2);
    }
    max_clusters = n;
  }
  const int nclusters = std::max(1, std::min(ntiles, max_clusters));
  k<<<dim3(2 * nclusters), kThreads, smem, s>>>(maps, args);
  return cudaGetLastError();
}

cudaError_t launch_persist(int bn, const TcMaps& maps, const TcArgs& args, cudaStream_t s) {
  switch (bn) {
    case 128: return launch_persist_bn<128>(maps, args, s);
    case 160: return launch_persist_bn<160>(maps, args, s);
    case 192: return launch_persist_bn<192>(maps, args, s);
    case 224: return launch_persist_bn<224>(maps, args, s);
    case 256: return launch_persist_bn<256>(maps, args, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pair(int bn, const TcMaps& maps, const TcArgs& args, cudaStream_t s) {
  switch (bn) {
    case 128: return launch_pair_bn<128>(maps, args, s);
    case 160: return launch_pair_bn<160>(maps, args, s);
    case 192: return launch_pair_bn<192>(maps, args, s);
    case 224: return launch_pair_bn<224>(maps, args, s);
    case 256: return launch_pair_bn<256>(maps, args, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sum(int bn, const TcMaps& maps, const TcArgs& args, cudaStream_t s) {
  switch (bn) {
    case 64: return launch_bn<64, kModeSum>(maps, args, s);
    case 128: return launch_bn<128, kModeSum>(maps, args, s);
    case 160: return launch_bn<160, kModeSum>(maps, args, s);
    case 192: return launch_bn<192, kModeSum>(maps, args, s);
    case 224: return launch_bn<224, kModeSum>(maps, args, s);
    case 256: return launch_bn<256, kModeSum>(maps, args, s);
    default: return cudaErrorInvalidValue;
  }
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

struct TcGemmPlan {
  int ld16 = 0, m = 0, d = 0;
  // q = A nu (FP16x3): scaled 2-way fp16 split of A rounded to float
  __half* a2[2] = {nullptr, nullptr};
  float* q_col_scale = nullptr;     // 1 / s_i
  CUtensorMap qmaps[6][2];
  CUtensorMap pmaps[5][2];          // boxes of BN / 2 rows for the SM-pair tiles
  // exact refresh: fixed-point slices of A (per-row power-of-two scale)
  int w = 7, K = 5;
  __nv_bfloat16* aK = nullptr;      // K slices, m x ld_bf each
  float* col_scale = nullptr;       // s_i
  float* inv_anorm = nullptr;       // 1 / ||a_i|| (drift statistic of the refresh)
  CUtensorMap rmaps[kMaxSlices];
  int bn_fixed = 0;                 // q GEMM tile width set by the autotuner (0: cost model)
  double bound_factor = 0.0;        // |p_exact - p| <= bound_factor * s_i * t_c
};

void tc_gemm_tile_for(int n_chains, int m, int* bn, int* stages) {
  // One-SM tiles (128 chains x BN rows of A, code BN) or SM-pair tiles (256
  // chains x BN), run by the persistent kernel (code kPersistCode + BN; the
  // one-launch-per-tile pair kernel is code kPairCode + BN).  With at least
  // 256 chains the persistent pair form is taken: per product it reads ~40 %
  // fewer bytes from L2 and from shared memory, and its epilogue overlaps the
  // next tile.  Within a form, pick the width that minimises (tiles per slot)
  // x (tile width): the per-tile time grows with BN, and the last round is
  // padded to the number of tile slots (SMs, or SM pairs).
  // (ESS_Q_BN fixes the code at build time, for tuning sweeps.)
  const int sms = num_sms();
  if (stages) *stages = 0;
#ifdef ESS_Q_BN
  *bn = ESS_Q_BN;
  (void)sms;
  return;
#endif
  const bool pair = n_chains >= 2 * BM;
  const int slots = pair ? std::max(1, sms / 2) : sms;
  const long long mt = pair ? (n_chains + 2 * BM - 1) / (2 * BM) : (n_chains + BM - 1) / BM;
  int best = 256;
  long long best_cost = -1;
  for (int w : kWidths) {
    if (pair && std::find(kPairWidths, kPairWidths + 5, w) == kPairWidths + 5) continue;
    const long long tiles = mt * ((m + w - 1) / w);
    const long long waves = (tiles + slots - 1) / slots;
    const long long cost = waves * w;
    if (best_cost < 0 || cost < best_cost || (cost == best_cost && w > best)) {
      best_cost = cost;
      best = w;
    }
  }
  *bn = pair ? kPersistCode + best : best;
}

int tc_refresh_slices(int d, int* w_out, int bits) {
  // widest slice w with (2^w - 1)^2 d <= 2^24 (exact FP32 sums), at most 8 bits;
  // K = ceil(bits / w) slices per operand
  int w = 8;
  while (w > 1 && (double)((1 << w) - 1) * ((1 << w) - 1) * d > 16777216.0) --w;
  int K = (bits + w - 1) / w;
  if (K > kMaxSlices) K = kMaxSlices;
  if (w_out) *w_out = w;
  return K;
}

cudaError_t tc_gemm_create(TcGemmPlan** plan, const double* A, int m, int d, int exact_bits,
                           bool with_q) {
  *plan = nullptr;
  TcGemmPlan* p = new TcGemmPlan();
  p->m = m;
  p->d = d;
  p->ld16 = (d + 7) & ~7;
  const int ld = p->ld16;
  auto fail = [&](cudaError_t e) {
    tc_gemm_destroy(p);
    return e;
  };
  cudaError_t e = cudaSuccess;
  if (with_q) {
  // --- FP16x3 operands: A rounded to float, row i scaled by s_i = 2^(15 - e_i)
  // (max_j |a_ij| in [2^(e_i - 1), 2^e_i)) and split as a s_i = a0 + a1
  std::vector<__half> h0((size_t)m * ld, __float2half_rn(0.f)), h1 = h0;
  std::vector<float> qcs(m);
  for (int i = 0; i < m; ++i) {
    float mx = 0.f;
    for (int j = 0; j < d; ++j) mx = std::fmax(mx, std::fabs((float)A[(size_t)i * d + j]));
    int ex = 0;
    if (mx > 0.f) (void)std::frexp(mx, &ex);
    const float t = mx > 0.f ? std::ldexp(1.f, 15 - ex) : 1.f;
    qcs[i] = mx > 0.f ? std::ldexp(1.f, ex - 15) : 0.f;
    for (int j = 0; j < d; ++j) {
      const float y = (float)A[(size_t)i * d + j] * t;
      const __half a = __float2half_rn(y);
      h0[(size_t)i * ld + j] = a;
      h1[(size_t)i * ld + j] = __float2half_rn(y - __half2float(a));
    }
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaMalloc(&p->a2[k], sizeof(__half) * (size_t)m * ld);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->a2[k], (k == 0 ? h0 : h1).data(), sizeof(__half) * (size_t)m * ld,
                     cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->q_col_scale, sizeof(float) * m);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->q_col_scale, qcs.data(), sizeof(float) * m, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i)
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      e = make_map(&p->qmaps[i][k], p->a2[k], m, d, ld, kWidths[i], false);
  for (int i = 0; i < 5 && e == cudaSuccess; ++i)
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      e = make_map(&p->pmaps[i][k], p->a2[k], m, d, ld, kPairWidths[i] / 2, false);
  if (e != cudaSuccess) return fail(e);
  }  // with_q

  // --- exact products: fixed-point slices of A in FP64 on the host
  p->K = tc_refresh_slices(d, &p->w, exact_bits);
  const int w = p->w, K = p->K;
  std::vector<__nv_bfloat16> slices((size_t)K * m * ld, __float2bfloat16_rn(0.f));
  std::vector<float> cs(m);
  for (int i = 0; i < m; ++i) {
    const double* a = A + (size_t)i * d;
    double mx = 0.0;
    for (int j = 0; j < d; ++j) mx = std::fmax(mx, std::fabs(a[j]));
    int ex = 0;
    if (mx > 0.0) (void)std::frexp(mx, &ex);
    cs[i] = mx > 0.0 ? std::ldexp(1.0f, ex) : 0.0f;
    for (int j = 0; j < d; ++j) {
      double y = mx > 0.0 ? std::ldexp(a[j], -ex) : 0.0;
      for (int k = 0; k < K; ++k) {
        y = std::ldexp(y, w);
        const double c = std::trunc(y);
        y -= c;
        slices[(size_t)k * m * ld + (size_t)i * ld + j] = __float2bfloat16_rn((float)c);
      }
    }
  }
  e = cudaMalloc(&p->aK, sizeof(__nv_bfloat16) * slices.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(p->aK, slices.data(), sizeof(__nv_bfloat16) * slices.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&p->col_scale, sizeof(float) * m);
  if (e == cudaSuccess) e = cudaMemcpy(p->col_scale, cs.data(), sizeof(float) * m, cudaMemcpyHostToDevice);
  {
    std::vector<float> ia(m);
    for (int i = 0; i < m; ++i) {
      double nn = 0.0;
      for (int j = 0; j < d; ++j) nn += A[(size_t)i * d + j] * A[(size_t)i * d + j];
      ia[i] = nn > 0.0 ? (float)(1.0 / std::sqrt(nn)) : 0.f;
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->inv_anorm, sizeof(float) * m);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->inv_anorm, ia.data(), sizeof(float) * m, cudaMemcpyHostToDevice);
  }
  for (int k = 0; k < K && e == cudaSuccess; ++k)
    e = make_map(&p->rmaps[k], p->aK + (size_t)k * m * ld, m, d, ld, kRefreshBN);
  if (e != cudaSuccess) return fail(e);
  // truncation of both operands (3 terms) plus the dropped pairs k + l > K + 1,
  // each below 2^(-wK) per element, summed over d elements
  p->bound_factor = (double)d * (3.0 + K * (K - 1) / 2.0) * std::ldexp(1.0, -w * K);
  *plan = p;
  return cudaSuccess;
}

void tc_gemm_destroy(TcGemmPlan* plan) {
  if (!plan) return;
  for (int k = 0; k < 2; ++k)
    if (plan->a2[k]) cudaFree(plan->a2[k]);
  if (plan->q_col_scale) cudaFree(plan->q_col_scale);
  if (plan->aK) cudaFree(plan->aK);
  if (plan->col_scale) cudaFree(plan->col_scale);
  if (plan->inv_anorm) cudaFree(plan->inv_anorm);
  delete plan;
}

const int kTcWidths[16] = {64, 128, 160, 192, 224, 256,
                           kPairCode + 128, kPairCode + 160, kPairCode + 192, kPairCode + 224,
                           kPairCode + 256,
                           kPersistCode + 128, kPersistCode + 160, kPersistCode + 192,
                           kPersistCode + 224, kPersistCode + 256};

cudaError_t tc_gemm_set_width(TcGemmPlan* plan, int bn) {
  if (!plan) return cudaErrorInvalidValue;
  if (bn != 0 && std::find(kTcWidths, kTcWidths + 16, bn) == kTcWidths + 16)
    return cudaErrorInvalidValue;
  plan->bn_fixed = bn;
  return cudaSuccess;
}

int tc_gemm_width(const TcGemmPlan* plan, int n_chains) {
  if (plan->bn_fixed) return plan->bn_fixed;
  int bn = 0;
  tc_gemm_tile_for(n_chains, plan->m, &bn, nullptr);
  return bn;
}

int tc_refresh_num_slices(const TcGemmPlan* plan) { return plan->K; }
double tc_refresh_bound_factor(const TcGemmPlan* plan) { return plan->bound_factor; }
const float* tc_refresh_col_scale(const TcGemmPlan* plan) { return plan->col_scale; }

cudaError_t tc_split2_rows(const float* src, int ld, int rows, int cols, __half* h0, __half* h1,
                           int ld16, float* unscale, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  split2_rows_kernel<<<grid_for((long long)rows * 32, 256), 256, 0, s>>>(src, ld, rows, cols, h0,
                                                                          h1, ld16, unscale);
  return cudaGetLastError();
}

cudaError_t tc_gemm_q(TcGemmPlan* plan, __half* const nu[2], const float* nu_unscale, int ld16,
                      int n_chains, float* Q, int ldq, int* status, cudaStream_t s) {
  if (!plan) return cudaErrorInvalidValue;
  if (n_chains == 0) return cudaSuccess;
  if (ld16 != plan->ld16) return cudaErrorInvalidValue;
  const int code = tc_gemm_width(plan, n_chains);
  const bool persist = code > kPersistCode;
  const bool pair = code > kPairCode;
  const int bn = persist ? code - kPersistCode : pair ? code - kPairCode : code;
  const int* widths = pair ? kPairWidths : kWidths;
  const int nw = pair ? 5 : 6;
  int wi = 0;
  while (wi < nw && widths[wi] != bn) ++wi;
  if (wi == nw) return cudaErrorInvalidValue;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = make_map(&maps.x[k], nu[k], n_chains, plan->d, ld16, BM, false);
    if (e != cudaSuccess) return e;
    maps.b[k] = pair ? plan->pmaps[wi][k] : plan->qmaps[wi][k];
  }
  // the persistent form stores Q by TMA: rows of 16-byte multiples
  bool use_persist = persist && (ldq & 3) == 0 && (reinterpret_cast<uintptr_t>(Q) & 15) == 0;
  if (use_persist && make_map_q(&maps.q, Q, n_chains, plan->m, ldq) != cudaSuccess)
    use_persist = false;
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_rows = n_chains;
  a.n_cols = plan->m;
  a.kblocks = (plan->d + BK - 1) / BK;
  // accumulator 0: h0.a0; accumulator 1: h1.a0 + h0.a1 (weight 2^-11 each)
  a.ngroups = 2;
  a.Q = Q;
  a.ldq = ldq;
  a.row_scale = nu_unscale;
  a.row_const = 1.f / kNuSplitScale;
  a.col_scale = plan->q_col_scale;
  a.status = status;
  return use_persist ? launch_persist(bn, maps, a, s)
         : pair      ? launch_pair(bn, maps, a, s)
                     : launch_sum(bn, maps, a, s);
}

namespace {
template <typename TI>
cudaError_t exact_product(TcGemmPlan* plan, const TI* X, int ldx, int n_chains,
                          __nv_bfloat16* x_slices, size_t slice_stride, float* row_scale,
                          float* P32, double* P64, int ldp, unsigned long long* drift_bits,
                          int* status, cudaStream_t s) {
  if (!plan) return cudaErrorInvalidValue;
  if (n_chains == 0) return cudaSuccess;
  const int K = plan->K, ld = plan->ld16;
  slice_rows_kernel<TI><<<grid_for((long long)n_chains * 32, 256), 256, 0, s>>>(
      X, ldx, n_chains, plan->d, plan->w, K, x_slices, ld, slice_stride, row_scale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int k = 0; k < K; ++k) {
    e = make_map(&maps.x[k], x_slices + (size_t)k * slice_stride, n_chains, plan->d, ld, BM);
    if (e != cudaSuccess) return e;
    maps.b[k] = plan->rmaps[k];
  }
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_rows = n_chains;
  a.n_cols = plan->m;
  a.kblocks = (plan->d + BK - 1) / BK;
  // slice pairs (x slice l, A slice k), k + l <= K + 1 (1-based), grouped into
  // rounds of at most kMaxPairs pairs whose x and A tiles (each loaded once per
  // round) fit one stage; within a round the pairs of one x tile with A tiles
  // that sit next to each other in the stage share one MMA (N <= 256).  The
  // pairs are taken row by row (x slice by x slice) or in 2 x 2 blocks of
  // (x, A) slices, whichever loads fewer tile bytes per K block.
  constexpr int kMaxPairs = 8;
  constexpr uint32_t kXTile = (uint32_t)BM * BK * 2, kATile = (uint32_t)kRefreshBN * BK * 2;
  static_assert(kXTile + kATile <= kRefreshStage, "one slice pair must fit a stage");
  auto pos_of = [](const unsigned char* arr, int n, int v) {
    for (int i = 0; i < n; ++i)
      if (arr[i] == (unsigned char)v) return i;
    return -1;
  };
  // fills t.round / t.nrounds; returns the tile bytes of all rounds per K
  // block, or 0 if the pairs need more than kMaxRounds rounds
  auto build = [&](TcArgs& t, bool blocks) -> uint32_t {
    int nr = 0;
    bool overflow = false;
    auto open_round = [&]() {
      std::memset(&t.round[nr], 0, sizeof(RefreshRound));
      ++nr;
    };
    auto add = [&](int l, int k) {
      if (overflow) return;
      RefreshRound* R = &t.round[nr - 1];
      int xi = pos_of(R->x, R->nx, l - 1), ai = pos_of(R->a, R->na, k - 1);
      const uint32_t bytes = (uint32_t)(R->nx + (xi < 0 ? 1 : 0)) * kXTile +
                             (uint32_t)(R->na + (ai < 0 ? 1 : 0)) * kATile;
      if (R->npairs == kMaxPairs || bytes > kRefreshStage) {
        if (nr == kMaxRounds) {
          overflow = true;
          return;
        }
        open_round();
        R = &t.round[nr - 1];
        xi = ai = -1;
      }
      if (xi < 0) {
        xi = R->nx;
        R->x[R->nx++] = (unsigned char)(l - 1);
      }
      if (ai < 0) {
        ai = R->na;
        R->a[R->na++] = (unsigned char)(k - 1);
      }
      const int col = R->npairs++;
      R->shift[col] = (unsigned char)(plan->w * (k + l));
      RefreshGroup* G = R->ngroups ? &R->g[R->ngroups - 1] : nullptr;
      if (G && G->xs == xi && G->a0 + G->na == ai && G->na < 4 && G->col + G->na == col) {
        ++G->na;
      } else {
        G = &R->g[R->ngroups++];
        G->xs = (unsigned char)xi;
        G->a0 = (unsigned char)ai;
        G->na = 1;
        G->col = (unsigned char)col;
      }
    };
    open_round();
    if (blocks) {
      for (int lb = 1; lb <= K; lb += 2)
        for (int kb = 1; kb <= K; kb += 2)
          for (int l = lb; l <= lb + 1 && l <= K; ++l)
            for (int k = kb; k <= kb + 1 && k <= K; ++k)
              if (k + l <= K + 1) add(l, k);
    } else {
      for (int l = 1; l <= K; ++l)
        for (int k = 1; k + l <= K + 1; ++k) add(l, k);
    }
    if (overflow) return 0u;
    // every round's tiles fit a stage (the copies of a stage land inside it)
    uint32_t total = 0;
    for (int r = 0; r < nr; ++r) {
      const uint32_t b = (uint32_t)t.round[r].nx * kXTile + (uint32_t)t.round[r].na * kATile;
      if (b > kRefreshStage) return 0u;
      total += b;
    }
    t.nrounds = nr;
    return total;
  };
  {
    TcArgs alt = a;
    const uint32_t rows_bytes = build(a, false);
    const uint32_t block_bytes = build(alt, true);
    if (rows_bytes == 0u && block_bytes == 0u) return cudaErrorInvalidValue;
    if (block_bytes != 0u && (rows_bytes == 0u || block_bytes < rows_bytes)) a = alt;
  }
  a.ngroups = 0;
  a.row_scale = row_scale;
  a.col_scale = plan->col_scale;
  a.P32 = P32;
  a.P64 = P64;
  a.ldp = ldp;
  a.inv_anorm = plan->inv_anorm;
  a.drift_bits = drift_bits;
  a.status = status;
  return launch_bn<kRefreshBN, kModePairs>(maps, a, s);
}
}  // namespace

cudaError_t tc_refresh(TcGemmPlan* plan, const float* X, int ldx, int n_chains,
                       __nv_bfloat16* x_slices, size_t slice_stride, float* row_scale,
                       float* P32, double* P64, int ldp, unsigned long long* drift_bits,
                       int* status, cudaStream_t s) {
  return exact_product<float>(plan, X, ldx, n_chains, x_slices, slice_stride, row_scale, P32,
                              P64, ldp, drift_bits, status, s);
}

cudaError_t tc_exact_f64(TcGemmPlan* plan, const double* X, int ldx, int n_chains,
                         __nv_bfloat16* x_slices, size_t slice_stride, float* row_scale,
                         double* P64, int ldp, unsigned long long* drift_bits, int* status,
                         cudaStream_t s) {
  return exact_product<double>(plan, X, ldx, n_chains, x_slices, slice_stride, row_scale,
                               nullptr, P64, ldp, drift_bits, status, s);
}

cudaError_t tc_batch_map(CUtensorMap* map, const __half* base, int rows, int cols, int ld,
                         int box_rows) {
  return make_map(map, base, rows, cols, ld, box_rows, false);
}

cudaError_t tc_batch_q(const TcBatchItem* items, int n_items, const CUtensorMap* maps,
                       const float* arow_unscale, const float* chain_unscale, float* Q,
                       int* status, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const size_t smem = (size_t)kBqStages * kBqStageBytes + 1024 + 256;
  cudaError_t e = cudaFuncSetAttribute(tc_batch_q_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(n_items, num_sms());
  tc_batch_q_kernel<<<grid, kThreads, smem, s>>>(items, n_items, maps, arow_unscale,
                                                  chain_unscale, Q, status);
  return cudaGetLastError();
}

}  // namespace ess
