// k_gemm_tc.cu -- q = A nu on the GB300 tensor cores (tcgen05 + TMA).
//
// The products q_i = a_i . nu of Sec. 2.2 for all chains form one GEMM
// Q (chains x m) = NU (chains x d) . A^T (A: m x d), both operands K-major.
// The mixed form evaluates it with the BF16x3 scheme: with nu = nu_hi + nu_lo
// and a = a_hi + a_lo (bf16 splits of the float values),
//     q ~= nu_hi.a_hi + nu_lo.a_hi + nu_hi.a_lo,
// three BF16 products accumulated in one FP32 accumulator in tensor memory.
//
// Kernel structure (one 128 x BN output tile per CTA, 4 warps):
//   warp 0 / lane 0   TMA producer: for every (K block, pass) loads the
//                     128 x 64 nu tile and the BN x 64 A tile of that pass
//                     into a ring of shared-memory stages (128-byte swizzle),
//                     completion signalled on the stage's "full" mbarrier;
//   warp 1 / lane 0   MMA issuer: waits "full", issues four
//                     tcgen05.mma.kind::f16 (K = 16 each) into the TMEM
//                     accumulator and commits to the stage's "empty"
//                     mbarrier so the producer can refill it;
//   all 4 warps       epilogue: tcgen05.ld of the accumulator rows (TMEM lane
//                     = chain row) and coalesced 16-byte stores to Q.
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the kernel
// sets kStatusTimeout, drains its own copies, frees TMEM and returns.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "ess_common.cuh"
#include "ess_gemm_tc.cuh"

namespace ess {
namespace {

constexpr int BM = 128;             // chains per tile (MMA M)
constexpr int BK = 64;              // bf16 elements per 128-byte swizzle row
constexpr int NTHREADS = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound per wait

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
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

// Bounded wait for the phase with the given parity to complete.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 256; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 32 TMEM lanes (one per thread of the warp) x 32 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row atoms 1024 bytes apart (tile base 1024-byte aligned).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);       // start address
  d |= (uint64_t)1u << 16;                      // leading byte offset (unused here)
  d |= (uint64_t)(1024u >> 4) << 32;            // stride byte offset: next 8-row atom
  d |= (uint64_t)1u << 46;                      // descriptor version
  d |= (uint64_t)2u << 61;                      // swizzle: 128 bytes
  return d;
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 accumulator, both
// operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                          // D format: F32
         | (1u << 7)                        // A format: BF16
         | (1u << 10)                       // B format: BF16
         | ((uint32_t)(N >> 3) << 17)       // N / 8
         | ((uint32_t)(M >> 4) << 24);      // M / 16
}

struct TcArgs {
  int n_rows;    // total chains
  int n_cols;    // total constraints
  int kblocks;   // ceil(d / 64)
  int npass;     // 3 = BF16x3, 1 = plain BF16
  float* Q;
  int ldq;
  int* status;
};

template <int BN>
constexpr uint32_t tmem_cols_for() {
  return BN <= 32 ? 32u : BN <= 64 ? 64u : BN <= 128 ? 128u : 256u;
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(NTHREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap map_x0, const __grid_constant__ CUtensorMap map_x1,
               const __grid_constant__ CUtensorMap map_b0, const __grid_constant__ CUtensorMap map_b1,
               TcArgs args) {
  constexpr uint32_t A_BYTES = BM * BK * 2;
  constexpr uint32_t B_BYTES = BN * BK * 2;
  constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr uint32_t TMEM_COLS = tmem_cols_for<BN>();
  static_assert(B_BYTES % 1024 == 0, "BN must be a multiple of 8");
  static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "BN in {32, ..., 256}, multiple of 32");

  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars[0, S): full, bars[S, 2S): empty, bars[2S]: accumulator ready
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  const uint32_t accum_bar = smem_u32(bars + 2 * STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN;
  const int m0 = blockIdx.y * BM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(accum_bar, 1);
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
  const int total = args.kblocks * args.npass;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int last_round[STAGES];
#pragma unroll
    for (int s = 0; s < STAGES; ++s) last_round[s] = -1;
    for (int it = 0; it < total; ++it) {
      const int s = it % STAGES;
      const int round = it / STAGES;
      if (round > 0 && !mbar_wait(empty_bar(s), (uint32_t)((round - 1) & 1))) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      const int kb = it / args.npass, pass = it % args.npass;
      // pass 0: hi.hi, pass 1: lo.hi, pass 2: hi.lo
      const CUtensorMap* mx = pass == 1 ? &map_x1 : &map_x0;
      const CUtensorMap* mb = pass == 2 ? &map_b1 : &map_b0;
      const uint32_t sa = sbase + s * STAGE_BYTES;
      mbar_expect_tx(full_bar(s), STAGE_BYTES);
      tma_load_2d(sa, mx, kb * BK, m0, full_bar(s));
      tma_load_2d(sa + A_BYTES, mb, kb * BK, n0, full_bar(s));
      last_round[s] = round;
    }
    if (*abort_flag) {
      // let every copy this thread issued land before the CTA exits
#pragma unroll
      for (int s = 0; s < STAGES; ++s)
        if (last_round[s] >= 0) (void)mbar_wait(full_bar(s), (uint32_t)(last_round[s] & 1));
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int it = 0; it < total; ++it) {
      const int s = it % STAGES;
      const int round = it / STAGES;
      if (!mbar_wait(full_bar(s), (uint32_t)(round & 1))) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sa = sbase + s * STAGE_BYTES;
      const uint64_t adesc = smem_desc_sw128(sa);
      const uint64_t bdesc = smem_desc_sw128(sa + A_BYTES);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        // each K = 16 step advances 32 bytes inside the swizzled row
        umma_bf16(tmem_d, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), idesc,
                  (it > 0 || k > 0) ? 1u : 0u);
      }
      umma_commit(empty_bar(s));
    }
    umma_commit(accum_bar);
  }

  // ---------------- epilogue: TMEM -> registers -> Q ----------------
  __syncwarp();
  const bool ready = mbar_wait(accum_bar, 0);
  tc_fence_after();
  if (!ready) *abort_flag = 1;
  const int row = m0 + warp * 32 + lane;
  const bool row_ok = row < args.n_rows && ready && !*abort_flag;
  float* qrow = args.Q + (size_t)(row_ok ? row : 0) * args.ldq;
  const bool vec_ok = (args.ldq & 3) == 0 && ((reinterpret_cast<uintptr_t>(args.Q) & 15) == 0);
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t v[32];
    tmem_ld_32cols(tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    tmem_ld_wait();
    if (!row_ok) continue;
    const int col = n0 + c0;
    if (vec_ok && col + 32 <= args.n_cols) {
      float4* dst = reinterpret_cast<float4*>(qrow + col);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                             __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (col + j < args.n_cols) qrow[col + j] = __uint_as_float(v[j]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(args.status, kStatusTimeout);
  if (warp == 0) tmem_dealloc(tmem_d, TMEM_COLS);
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

// 2-D bf16 tensor map over a rows x cols matrix (row stride ld elements),
// box = box_rows x 64 columns, 128-byte swizzle, zero fill out of bounds.
cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int cols, int ld,
                     int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 2) % 16 != 0)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kSmemLimit = 227 * 1024;

template <int BN>
constexpr int stages_for() {
  constexpr int stage = (BM + BN) * BK * 2;
  constexpr int s = (kSmemLimit - 1024 - 256) / stage;
  return s > 6 ? 6 : s;
}

template <int BN>
size_t smem_for() {
  return (size_t)stages_for<BN>() * (BM + BN) * BK * 2 + 1024 + 256;
}

template <int BN>
cudaError_t launch_bn(const CUtensorMap& x0, const CUtensorMap& x1, const CUtensorMap& b0,
                      const CUtensorMap& b1, const TcArgs& args, cudaStream_t s) {
  constexpr int ST = stages_for<BN>();
  auto k = tc_gemm_kernel<BN, ST>;
  const size_t smem = smem_for<BN>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((args.n_cols + BN - 1) / BN, (args.n_rows + BM - 1) / BM);
  k<<<grid, NTHREADS, smem, s>>>(x0, x1, b0, b1, args);
  return cudaGetLastError();
}

cudaError_t launch_any(int bn, const CUtensorMap& x0, const CUtensorMap& x1, const CUtensorMap& b0,
                       const CUtensorMap& b1, const TcArgs& args, cudaStream_t s) {
  switch (bn) {
    case 64: return launch_bn<64>(x0, x1, b0, b1, args, s);
    case 128: return launch_bn<128>(x0, x1, b0, b1, args, s);
    case 160: return launch_bn<160>(x0, x1, b0, b1, args, s);
    case 192: return launch_bn<192>(x0, x1, b0, b1, args, s);
    case 224: return launch_bn<224>(x0, x1, b0, b1, args, s);
    case 256: return launch_bn<256>(x0, x1, b0, b1, args, s);
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

}  // namespace

struct TcGemmPlan {
  CUtensorMap a_hi[6], a_lo[6];  // one per tile width (box rows differ)
  const __nv_bfloat16* A_hi;
  const __nv_bfloat16* A_lo;
  int ld_bf, m, d;
};

static const int kWidths[6] = {64, 128, 160, 192, 224, 256};

void tc_gemm_tile_for(int n_chains, int m, int* bn, int* stages) {
  // Pick the tile width that minimises (waves of tiles) x (tile width): the
  // per-tile time grows with BN, and the last wave is padded to the SM count.
  const int sms = num_sms();
  const long long mt = (n_chains + BM - 1) / BM;
  int best = 256;
  long long best_cost = -1;
  for (int w : kWidths) {
    const long long tiles = mt * ((m + w - 1) / w);
    const long long waves = (tiles + sms - 1) / sms;
    const long long cost = waves * w;
    if (best_cost < 0 || cost < best_cost || (cost == best_cost && w > best)) {
      best_cost = cost;
      best = w;
    }
  }
  *bn = best;
  if (stages) {
    switch (best) {
      case 64: *stages = stages_for<64>(); break;
      case 128: *stages = stages_for<128>(); break;
      case 160: *stages = stages_for<160>(); break;
      case 192: *stages = stages_for<192>(); break;
      case 224: *stages = stages_for<224>(); break;
      default: *stages = stages_for<256>(); break;
    }
  }
}

cudaError_t tc_gemm_create(TcGemmPlan** plan, const __nv_bfloat16* A_hi, const __nv_bfloat16* A_lo,
                           int ld_bf, int m, int d) {
  *plan = nullptr;
  TcGemmPlan* p = new TcGemmPlan();
  p->A_hi = A_hi;
  p->A_lo = A_lo;
  p->ld_bf = ld_bf;
  p->m = m;
  p->d = d;
  for (int i = 0; i < 6; ++i) {
    cudaError_t e = make_map(&p->a_hi[i], A_hi, m, d, ld_bf, kWidths[i]);
    if (e == cudaSuccess) e = make_map(&p->a_lo[i], A_lo, m, d, ld_bf, kWidths[i]);
    if (e != cudaSuccess) {
      delete p;
      return e;
    }
  }
  *plan = p;
  return cudaSuccess;
}

void tc_gemm_destroy(TcGemmPlan* plan) {
  delete plan;
}

cudaError_t tc_gemm_bf16x3(TcGemmPlan* plan, const __nv_bfloat16* nu_hi,
                           const __nv_bfloat16* nu_lo, int ld_bf, int n_chains, float* Q, int ldq,
                           int* status, cudaStream_t s) {
  if (!plan || n_chains <= 0) return n_chains == 0 ? cudaSuccess : cudaErrorInvalidValue;
  if (ld_bf != plan->ld_bf) return cudaErrorInvalidValue;
  int bn = 0;
  tc_gemm_tile_for(n_chains, plan->m, &bn, nullptr);
  int wi = 0;
  while (kWidths[wi] != bn) ++wi;
  CUtensorMap x0, x1;
  cudaError_t e = make_map(&x0, nu_hi, n_chains, plan->d, ld_bf, BM);
  if (e == cudaSuccess) e = make_map(&x1, nu_lo, n_chains, plan->d, ld_bf, BM);
  if (e != cudaSuccess) return e;
  TcArgs a;
  a.n_rows = n_chains;
  a.n_cols = plan->m;
  a.kblocks = (plan->d + BK - 1) / BK;
  a.npass = 3;
  a.Q = Q;
  a.ldq = ldq;
  a.status = status;
  return launch_any(bn, x0, x1, plan->a_hi[wi], plan->a_lo[wi], a, s);
}

cudaError_t tc_gemm_bf16(const __nv_bfloat16* X, const __nv_bfloat16* B, int ld_bf, int n, int m,
                         int d, float* Q, int ldq, int* status, cudaStream_t s) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  int bn = 0;
  tc_gemm_tile_for(n, m, &bn, nullptr);
  CUtensorMap x0, b0;
  cudaError_t e = make_map(&x0, X, n, d, ld_bf, BM);
  if (e == cudaSuccess) e = make_map(&b0, B, m, d, ld_bf, bn);
  if (e != cudaSuccess) return e;
  TcArgs a;
  a.n_rows = n;
  a.n_cols = m;
  a.kblocks = (d + BK - 1) / BK;
  a.npass = 1;
  a.Q = Q;
  a.ldq = ldq;
  a.status = status;
  return launch_any(bn, x0, x0, b0, b0, a, s);
}

}  // namespace ess
