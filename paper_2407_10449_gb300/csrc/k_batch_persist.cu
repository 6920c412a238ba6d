// k_batch_persist.cu -- a whole refresh period of the batched mixed-form
// sampler (many polytopes of uneven d and m, each with its own chains) in ONE
// persistent cooperative launch: one CTA of 32 warps per SM, every step's
// work taken from work queues, the chain steps gated by per-problem
// dependency counters, steps separated by bounded grid barriers.
//
// Per step j of the period (Alg. 1 for every chain of every problem):
//   warps 0..5   q = A_p nu for every problem on the tensor cores (tcgen05,
//                TMA; the FP16x3 products of the one-problem form, items of
//                128 rows of A_p x up to 64 of its chains, walked b, b + G,
//                ... largest first), with the TMA ring, MMA issue and TMEM
//                accumulators kept live from step to step; each epilogue warp
//                counts its finished rows of an item on the item's problem
//                (a release: fence, then atomic add);
//   warps 6..21  draw nu of step j + 1 (Philox + Box-Muller, its fp16
//                splits) into the other nu buffers;
//   warps 22..31 from the start of the step, take chains from a device work
//                queue (problems in the order their q items finish) and run
//                the warp-per-chain step (App. B roots, domination prune,
//                Alg. 3 sort and sweep, theta, move, Sec. 3.3 check), each
//                after a bounded wait for its problem's count to reach the
//                problem's items x 4 (an acquire); their shared memory lies
//                behind the GEMM's ring;
//   warps 0..21  join the chain queue once the CTA's own q items are done
//                (a named barrier; the idle ring becomes their step areas);
//   chains with too many arcs go to a list, which whole CTAs take after a
//   grid barrier with the CTA-per-chain step (overflow phase).
// The refresh of p = A x and the draw of step 0 run before the launch (the
// caller's graph nodes).  Every wait -- the mbarriers of the GEMM, the
// dependency counters and the grid barriers -- is bounded: on expiry the
// warp sets the time-out status and an abort flag that every other wait
// sees, the CTA drains its own copies in flight, frees its tensor memory and
// returns.
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "chain_cta_step.cuh"
#include "chain_warp_step.cuh"
#include "ess_batch_persist.cuh"
#include "ess_gemm_tc.cuh"
#include "grid_sync.cuh"
#include "tc_ptx.cuh"

namespace ess {
namespace {

using namespace tcptx;

constexpr int kPW = 32;                 // warps per CTA
constexpr int kPT = kPW * 32;           // threads per CTA
constexpr int kGemmWarps = 6;           // producer, MMA issuer, 4 epilogue warps
constexpr int kPBK = 64;                // 16-bit elements per 128-byte swizzle row
constexpr uint32_t kPA = 128 * 64 * 2;  // bytes of one A split tile (128 rows x 64)
constexpr uint32_t kPStage = 2 * kPA + 2 * 64 * 64 * 2;  // two A and two nu tiles
constexpr int kPStages = 3;
constexpr uint32_t kPTmemCols = 256;    // two buffers x (two accumulators x 64 columns)
constexpr int kPHead = 128;             // mbarriers, TMEM address (before the 1 KB alignment)
// the CTA-per-chain step of the overflow phase: 1024 threads x 8 rows each
constexpr int kPItems = kChainItems;
constexpr int kDrawWarps = 16;                       // warps 6..21
constexpr int kEarlyWarp = kGemmWarps + kDrawWarps;  // warps 22.. step chains from the start
constexpr int kLateThreads = kEarlyWarp * 32;        // warps 0..21: the named barrier
// warp w's step area is the region's w-th kWarpStepSmem bytes: those of the
// early warps lie behind the ring
static_assert((size_t)kEarlyWarp * kWarpStepSmem >= (size_t)kPStages * kPStage,
              "the early warps' step areas overlap the TMA ring");

// nu of chain c at step t (the batch draw: Philox blocks (seed, j / 4, chain,
// t, problem), Box-Muller, the two-way fp16 split of nu * 2^12), one warp.
__device__ __forceinline__ void persist_draw_chain(const ChainDesc& cd, uint64_t seed, uint32_t t,
                                                   float* __restrict__ NU, __half* __restrict__ H0,
                                                   __half* __restrict__ H1, int lane) {
  float* row = NU + cd.x_off;
  const int nblk = (cd.d + 3) >> 2;
  for (int n = lane; n < nblk; n += 32) {
    uint32_t r[4];
    rng_block(seed, (uint32_t)n, cd.chain, t, cd.problem, 0u, r);
    float z[4];
    box_muller4(r, z);
    const int left = cd.d - 4 * n;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k >= left) break;
      row[4 * n + k] = z[k];
      const float y = z[k] * kNuSplitScale;
      const __half a = __float2half_rn(y);
      H0[cd.h_off + 4 * n + k] = a;
      H1[cd.h_off + 4 * n + k] = __float2half_rn(y - __half2float(a));
    }
  }
}

// State of the GEMM roles carried from step to step (the mbarrier phases run on).
struct GemmState {
  int s = 0;            // producer / MMA: ring stage
  uint32_t phase = 0;   // producer / MMA: ring phase
  long long count = 0;  // producer: K blocks issued so far
  long long items = 0;  // MMA / epilogue: items processed so far (accumulator buffer)
  bool loaded[kPStages];
  uint32_t last_phase[kPStages];
};

__device__ __forceinline__ void persist_abort(const BatchPersistArgs& a) {
  atomicOr(a.prm.status, kStatusTimeout);
  atomicExch(a.abort_flag, 1);
}

__device__ __forceinline__ bool persist_aborted(const BatchPersistArgs& a) {
  return *reinterpret_cast<volatile int*>(a.abort_flag) != 0;
}

// TMA producer (warp 0, lane 0) for one step's items.
__device__ void persist_produce(const BatchPersistArgs& a, const CUtensorMap* maps, uint32_t sbase,
                                uint64_t* bars, GemmState& g) {
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + kPStages + s); };
  asm volatile("fence.proxy.async.global;" ::: "memory");  // nu splits written this launch
  for (int it = blockIdx.x; it < a.n_titems && !persist_aborted(a); it += gridDim.x) {
    const TcBatchItem I = a.titems[it];
    const CUtensorMap* mp = maps + 4 * I.problem;
    const uint32_t bytes = 2u * kPA + 2u * (uint32_t)I.ntile * 128u;
    for (int kb = 0; kb < I.kblocks; ++kb, ++g.count) {
      if (g.count >= kPStages && !mbar_wait(empty_bar(g.s), g.phase ^ 1u)) {
        persist_abort(a);
        return;
      }
      const uint32_t sa = sbase + g.s * kPStage;
      mbar_expect_tx(full_bar(g.s), bytes);
      tma_load_2d(sa, mp + 0, kb * kPBK, I.row0, full_bar(g.s));
      tma_load_2d(sa + kPA, mp + 1, kb * kPBK, I.row0, full_bar(g.s));
      tma_load_2d(sa + 2 * kPA, mp + 2, kb * kPBK, I.chain0, full_bar(g.s));
      tma_load_2d(sa + 2 * kPA + (uint32_t)I.ntile * 128u, mp + 3, kb * kPBK, I.chain0,
                  full_bar(g.s));
      g.loaded[g.s] = true;
      g.last_phase[g.s] = g.phase;
      if (++g.s == kPStages) {
        g.s = 0;
        g.phase ^= 1u;
      }
    }
  }
}

// MMA issuer (warp 1, lane 0) for one step's items.
__device__ void persist_mma(const BatchPersistArgs& a, uint32_t sbase, uint64_t* bars, uint32_t tmem_d,
                            GemmState& g) {
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + kPStages + s); };
  auto accf_bar = [&](int b) { return smem_u32(bars + 2 * kPStages + b); };
  auto acce_bar = [&](int b) { return smem_u32(bars + 2 * kPStages + 2 + b); };
  for (int it = blockIdx.x; it < a.n_titems; it += gridDim.x, ++g.items) {
    const TcBatchItem I = a.titems[it];
    const int buf = (int)(g.items & 1);
    // the epilogue has read this buffer's previous item
    if (g.items >= 2 && !mbar_wait(acce_bar(buf), (uint32_t)(((g.items - 2) >> 1) & 1))) {
      persist_abort(a);
      return;
    }
    tc_fence_after();
    const uint32_t idesc = idesc_f16(128, I.ntile, false);
    const uint32_t acc0 = tmem_d + (uint32_t)(buf * 128), acc1 = acc0 + 64;
    for (int kb = 0; kb < I.kblocks; ++kb) {
      if (!mbar_wait(full_bar(g.s), g.phase)) {
        persist_abort(a);
        return;
      }
      tc_fence_after();
      const uint32_t sa = sbase + g.s * kPStage;
      const uint64_t a0 = smem_desc_sw128(sa);
      const uint64_t a1 = smem_desc_sw128(sa + kPA);
      const uint64_t h0 = smem_desc_sw128(sa + 2 * kPA);
      const uint64_t h1 = smem_desc_sw128(sa + 2 * kPA + (uint32_t)I.ntile * 128u);
#pragma unroll
      for (int k = 0; k < kPBK / 16; ++k)
        umma_bf16(acc0, a0 + 2 * k, h0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
      for (int k = 0; k < kPBK / 16; ++k)
        umma_bf16(acc1, a1 + 2 * k, h0 + 2 * k, idesc, (kb == 0 && k == 0) ? 0u : 1u);
#pragma unroll
      for (int k = 0; k < kPBK / 16; ++k) umma_bf16(acc1, a0 + 2 * k, h1 + 2 * k, idesc, 1u);
      umma_commit(empty_bar(g.s));
      if (++g.s == kPStages) {
        g.s = 0;
        g.phase ^= 1u;
      }
    }
    umma_commit(accf_bar(buf));
  }
}

// Epilogue warps 2..5 (TMEM lane quarter warp % 4) for one step's items: the
// two accumulators summed, unscaled and stored as each chain's q, 16 chains
// at a time.
__device__ void persist_epilogue(const BatchPersistArgs& a, uint64_t* bars, uint32_t tmem_d, int warp,
                                 int lane, GemmState& g) {
  auto accf_bar = [&](int b) { return smem_u32(bars + 2 * kPStages + b); };
  auto acce_bar = [&](int b) { return smem_u32(bars + 2 * kPStages + 2 + b); };
  const int quarter = warp & 3;
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
  for (int it = blockIdx.x; it < a.n_titems; it += gridDim.x, ++g.items) {
    const int buf = (int)(g.items & 1);
    if (persist_aborted(a) || !mbar_wait(accf_bar(buf), (uint32_t)((g.items >> 1) & 1))) {
      persist_abort(a);
      return;
    }
    tc_fence_after();
    const TcBatchItem I = a.titems[it];
    const int r = quarter * 32 + lane;  // row within the item
    const bool row_ok = r < I.rows;
    const float ru = row_ok ? a.arow_unscale[I.urow + r] : 0.f;
    const uint32_t acc0 = tmem_d + lane_off + (uint32_t)(buf * 128), acc1 = acc0 + 64;
    float* qrow = a.Q + I.q_off + I.row0 + r;  // chain c of the item at qrow[c * m]
    for (int c0 = 0; c0 < I.ntile; c0 += 16) {
      uint32_t v[16], w[16];
      tmem_ld_16cols(acc0 + (uint32_t)c0, v);
      tmem_ld_16cols(acc1 + (uint32_t)c0, w);
      tmem_ld_wait();
      if (row_ok) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int c = c0 + jj;
          const float qv = __uint_as_float(v[jj]) + __uint_as_float(w[jj]);
          if (c < I.chains) qrow[(size_t)c * I.m] = qv * ru * (1.f / kNuSplitScale);
        }
      }
    }
    // TMEM buffer free for the item after next; this warp's rows of the
    // item's q counted for its problem (each lane's stores fenced first)
    tc_fence_before();
    __threadfence();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(acce_bar(buf));
      atomicAdd(a.dep_done + I.problem, 1u);
    }
  }
}

// Bounded wait of a warp until problem p's count reaches target (every q item
// of the problem stored in this step), then an acquire fence.  False if the
// wait ran out (time-out status and abort flag set) or another CTA aborted.
__device__ __forceinline__ bool persist_dep_wait(const BatchPersistArgs& a, int p,
                                                 unsigned target, int lane) {
  int ok = 1;
  if (lane == 0) {
    const volatile unsigned* f = a.dep_done + p;
    if (*f < target) {
      const unsigned long long t0 = grid_now();
      while (*f < target) {
        if (persist_aborted(a)) {
          ok = 0;
          break;
        }
        if (grid_now() - t0 > a.wait_ns) {
          persist_abort(a);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncwarp();
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __noinline__ void persist_overflow_chain(const ChainParams<float>& p, int c,
                                                  unsigned char* region, uint32_t bytes) {
  cta_chain_step<float, kPT, kPItems, true>(p, c, region, bytes);
}

template <bool LONG>
__global__ void __launch_bounds__(kPT, 1) batch_persist_kernel(BatchPersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);  // full[S], empty[S], accf[2], acce[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kPStages + 4);
  // the phases' shared memory (TMA ring / 32 warp-step areas / CTA step), 1 KB aligned
  const uint32_t raw = smem_u32(smem_raw + kPHead);
  unsigned char* region = smem_raw + kPHead + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(region);
  uint32_t dyn_smem;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
  const uint32_t region_bytes = dyn_smem - (uint32_t)(region - smem_raw);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPStages; ++s) {
      mbar_init(smem_u32(bars + s), 1);
      mbar_init(smem_u32(bars + kPStages + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(bars + 2 * kPStages + b), 1);
      mbar_init(smem_u32(bars + 2 * kPStages + 2 + b), 4);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), kPTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;

  GemmState g;
#pragma unroll
  for (int s = 0; s < kPStages; ++s) {
    g.loaded[s] = false;
    g.last_phase[s] = 0;
  }
  long long sort_keys = 0;
  const int n = a.prm.n_chains;
  const int draw_warps = gridDim.x * kDrawWarps;
  const int draw_id = blockIdx.x * kDrawWarps + (warp - kGemmWarps);
  const uint32_t t_base = a.prm.t_dev ? *a.prm.t_dev : 0u;
  unsigned char* wsm = region + kWarpStepSmem * warp;
  bool ok = true;

  for (int j = 0; j < a.steps && ok; ++j) {
    const int cur = j & 1, nxt = cur ^ 1;
    if (warp < kEarlyWarp) {
      // ---- q of step j on the tensor cores; nu of step j + 1 beside it ------
      if (warp == 0) {
        if (lane == 0) persist_produce(a, a.maps[cur], sbase, bars, g);
      } else if (warp == 1) {
        if (lane == 0) persist_mma(a, sbase, bars, tmem_d, g);
      } else if (warp < kGemmWarps) {
        persist_epilogue(a, bars, tmem_d, warp, lane, g);
      } else if (j + 1 < a.steps) {
        const uint32_t tt = a.prm.t + (uint32_t)(j + 1) + t_base;
        for (int c = draw_id; c < n; c += draw_warps)
          persist_draw_chain(a.desc[c], a.prm.seed, tt, a.NU[nxt], a.H0[nxt], a.H1[nxt], lane);
        asm volatile("fence.proxy.async.global;" ::: "memory");  // read by TMA next step
      }
      __syncwarp();
      // this CTA's items are done: the ring is idle until the next step and
      // its shared memory becomes the step areas of warps 0..21
      tc_fence_before();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, %0;" ::"n"(kLateThreads) : "memory");
      tc_fence_after();
    }

    // ---- chain steps from the work queue, each after its problem's q --------
    ChainParams<float> p = a.prm;
    p.t = a.prm.t + (uint32_t)j;
    p.P_in = a.P[cur];
    p.P_out = a.P[nxt];
    p.NU = a.NU[cur];
    p.overflow_count = a.queue + 2 * j + 1;
    p.overflow_list = a.ovf_list;
    p.chain_list = nullptr;
    p.list_count = nullptr;
    for (;;) {
      int ticket = 0;
      if (lane == 0) ticket = atomicAdd(a.queue + 2 * j, 1);
      ticket = __shfl_sync(0xffffffffu, ticket, 0);
      if (ticket >= n) break;
      const int c = a.order[ticket];
      const int prob = a.desc[c].problem;
      const unsigned target = (unsigned)(j + 1) * (unsigned)a.dep_target[prob] + a.hold;
      if (!persist_dep_wait(a, prob, target, lane)) break;
      const int keys = warp_chain_step<float, true, LONG>(p, c, wsm, lane);
      if (keys > 0) sort_keys += keys;
    }
    tc_fence_before();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    ok = grid_barrier(a.bar, a.abort_flag, a.prm.status, a.wait_ns);
    if (!ok) break;
    tc_fence_after();

    // ---- overflow phase: chains with too many arcs, one CTA each -------------
    const int n_ovf = *reinterpret_cast<volatile int*>(a.queue + 2 * j + 1);
    if (n_ovf > 0) {
      for (int w = blockIdx.x; w < n_ovf; w += gridDim.x)
        persist_overflow_chain(p, a.ovf_list[w], region, region_bytes);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ok = grid_barrier(a.bar, a.abort_flag, a.prm.status, a.wait_ns);
    }
  }

  // ---- leave: copies in flight drained, tensor memory freed ------------------
  if (warp == 0 && lane == 0 && persist_aborted(a)) {
#pragma unroll
    for (int s = 0; s < kPStages; ++s)
      if (g.loaded[s]) (void)mbar_wait(smem_u32(bars + s), g.last_phase[s]);
  }
  if (lane == 0 && sort_keys) atomicAdd(&a.prm.stats->sort_keys, (unsigned long long)sort_keys);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem_d, kPTmemCols);
}

}  // namespace

namespace {

size_t persist_region_bytes() {
  return std::max<size_t>((size_t)kPStages * kPStage, (size_t)kPW * kWarpStepSmem);
}

size_t persist_smem_bytes() { return kPHead + 1024 + persist_region_bytes(); }

// shared memory of the overflow phase's CTA step (keys, values, x', flags,
// merge buckets) for states of up to max_d elements
size_t persist_cta_bytes(int max_d) {
  const size_t nslot = (size_t)kPT * kPItems, npad = nslot + nslot / 32;
  return 2 * npad * sizeof(float) + (size_t)((max_d + 1) & ~1) * sizeof(float) +
         nslot * sizeof(int) + 2 * std::min<size_t>(nslot, 2048) * sizeof(float);
}

template <bool LONG>
int persist_grid(size_t smem) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(batch_persist_kernel<LONG>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persist_kernel<LONG>, kPT,
                                                    smem) != cudaSuccess)
    return 0;
  return per_sm >= 1 ? sms : 0;
}

}  // namespace

bool batch_persist_supported(int max_m, int max_d) {
  if (max_m > kPT * kPItems || max_m < 1 || max_d < 1) return false;
  if (persist_cta_bytes(max_d) > persist_region_bytes()) return false;
  return persist_grid<false>(persist_smem_bytes()) > 0 && persist_grid<true>(persist_smem_bytes()) > 0;
}

cudaError_t launch_batch_persist(const BatchPersistArgs& a, cudaStream_t s) {
  if (a.steps <= 0 || a.prm.n_chains <= 0) return cudaSuccess;
  if ((a.steps & 1) || !a.queue || !a.bar || !a.abort_flag || !a.order || !a.ovf_list ||
      !a.dep_target || !a.dep_done || !a.prm.slack || a.P[0] == a.P[1])
    return cudaErrorInvalidValue;
  const size_t smem = persist_smem_bytes();
  const int grid = a.prm.long_arcs ? persist_grid<true>(smem) : persist_grid<false>(smem);
  if (grid <= 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return a.prm.long_arcs ? cudaLaunchKernelEx(&cfg, batch_persist_kernel<true>, a)
                         : cudaLaunchKernelEx(&cfg, batch_persist_kernel<false>, a);
}

}  // namespace ess
