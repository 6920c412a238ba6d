// ess_noalloc.cu -- one FP64 chain step that allocates no device memory.
//
// Who needs this: callers that are not allowed to call cudaMalloc at the point
// where they want a step -- a plugin running inside a host framework that owns
// the whole device-memory budget and forbids allocations after start-up, or a
// latency-critical service that must keep the allocator (and its implicit
// device synchronization) off its request path.  The call is synchronous: it
// reads a status word back to the host and waits for the caller's stream.
// ess_step_noalloc gives them the FP64 one-step map of ess_step_with_draws
// without an ess_state: the caller passes A, b and every input and output as
// device pointers, and all scratch (the row norms of A, the products p = A x
// and q = A nu, the status word and counters) lives in one fixed array
// compiled into this library.
//
// That array, g_noalloc_scratch, is ESS_NOALLOC_SCRATCH_BYTES (16 MiB) of
// device memory on every GPU that loads the library, held until the process
// exits.  Every call shares it and finds the previous call's contents there,
// so the status word and counters are cleared at the start of each call, and
// two calls that overlap on the GPU (different streams or threads at the same
// time) race on it: serialize them.
//
// Host code cannot use the array's name as a device address (on the host it
// names a host-side stand-in).  The address is looked up once per device with
// cudaGetSymbolAddress, with that device current, the first time the entry
// point runs on it.
//
// Scratch layout, every region starting on a 256-byte boundary (r(v) = v
// rounded up to a multiple of 256):
//   status word              256 bytes
//   counters (DevStats)      r(sizeof(DevStats)) = 256 bytes
//   row norms of A           r(8 m)
//   P = A x                  r(8 n m)
//   Q = A nu                 r(8 n m)
// so a call needs 512 + r(8 m) + 2 r(8 n m) <= ESS_NOALLOC_SCRATCH_BYTES.
#include <mutex>
#include <string>

#include "ess.h"
#include "ess_kernels.cuh"

void ess_internal_set_error(const std::string& msg);  // ess_abi.cu

namespace {

constexpr size_t kScratchBytes = ESS_NOALLOC_SCRATCH_BYTES;
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// ||a_i||_2 for every row of A (one warp per row), used by the residual filter.
__global__ void noalloc_row_norms(const double* __restrict__ A, int d, int m,
                                  double* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  const double* a = A + (size_t)warp * d;
  double acc = 0.0;
  for (int j = lane; j < d; j += 32) acc = fma(a[j], a[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = sqrt(acc);
}

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on `dev` (looked up once, with dev current).
cudaError_t scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return cudaSuccess;
}

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

ess_status fail(ess_status st, const std::string& msg) {
  ess_internal_set_error(msg);
  return st;
}

ess_status cuda_fail(cudaError_t e, const char* what) {
  return fail(ESS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" ess_status ess_step_noalloc(const double* A, const double* b, int d, int m,
                                       const double* X, const double* nu, const double* u,
                                       int n_chains, double* X_next, double* theta,
                                       int* rejected, void* cuda_stream) {
  ess_internal_set_error("");
  if (d < 1 || m < 1 || n_chains < 0) return fail(ESS_ERR_ARG, "need d >= 1, m >= 1, n_chains >= 0");
  if (n_chains == 0) return ESS_OK;
  if (!A || !b || !X || !nu || !u || !X_next) return fail(ESS_ERR_ARG, "NULL input");
  const int threads = ess::chain_threads_for(m);
  if (threads == 0) return fail(ESS_ERR_UNSUPPORTED, "m exceeds 8192");

  // scratch layout: status | counters | row norms (m) | P (n x m) | Q (n x m)
  const size_t off_stats = kAlign;
  const size_t off_norm = off_stats + round_up(sizeof(ess::DevStats));
  const size_t off_p = off_norm + round_up(sizeof(double) * (size_t)m);
  const size_t pq = round_up(sizeof(double) * (size_t)n_chains * (size_t)m);
  const size_t need = off_p + 2 * pq;
  if (need > kScratchBytes)
    return fail(ESS_ERR_ARG,
                "n_chains * m too large for the fixed scratch of ess_step_noalloc: "
                "512 + r(8 m) + 2 r(8 n_chains m) bytes must fit in 16 MiB, r(v) = v rounded "
                "up to a multiple of 256 (need " + std::to_string(need) + ")");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  // the CTA-per-chain kernel keeps x' (d values) beside the arcs in shared
  // memory: the same limit as ess_create
  int smem_optin = 0;
  e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if (ess::chain_smem_bytes<double>(threads, d) + 1024 > (size_t)smem_optin)
    return fail(ESS_ERR_UNSUPPORTED, "d too large for the chain-step kernel's shared memory");

  unsigned char* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  int* status = reinterpret_cast<int*>(base);
  ess::DevStats* stats = reinterpret_cast<ess::DevStats*>(base + off_stats);
  double* anorm = reinterpret_cast<double*>(base + off_norm);
  double* P = reinterpret_cast<double*>(base + off_p);
  double* Q = reinterpret_cast<double*>(base + off_p + pq);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int h = 0;

  // the array keeps the previous call's contents: clear what must start at zero
  e = cudaMemsetAsync(base, 0, off_norm, st);
  if (e == cudaSuccess)
    e = ess::launch_gemm_nt_f64<double, double>(X, d, A, d, P, m, n_chains, m, d, nullptr,
                                                nullptr, st);
  if (e == cudaSuccess) e = ess::launch_check_feasible(P, m, b, n_chains, m, status, st);
  // the start points are checked before anything is written to the outputs
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ess_step_noalloc (start-point check)");
  if (h & ess::kStatusInfeasible)
    return fail(ESS_ERR_INFEASIBLE_X0, "a chain state violates A x <= b (checked in FP64)");

  noalloc_row_norms<<<(m * 32 + 255) / 256, 256, 0, st>>>(A, d, m, anorm);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = ess::launch_gemm_nt_f64<double, double>(nu, d, A, d, Q, m, n_chains, m, d, nullptr,
                                                nullptr, st);
  if (e == cudaSuccess) {
    ess::ChainParams<double> p{};
    p.d = d;
    p.m = m;
    p.n_chains = n_chains;
    p.ldx = d;
    p.ldp = m;
    p.P_in = P;
    p.P_out = P;
    p.Q = Q;
    p.b = b;
    p.b64 = b;
    p.A64 = A;
    p.anorm = anorm;
    p.X = X;
    p.X_out = X_next;
    p.NU = nu;
    p.U = u;
    p.trim_eps = 0.0;
    p.tangent_thresh = 1e-4;
    p.margin = 1e-8;
    p.theta_out = theta;
    p.rejected_out = rejected;
    p.stats = stats;
    p.status = status;
    e = ess::launch_chain_step<double>(p, threads, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ess_step_noalloc launch");
  e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ess_step_noalloc");
  if (h & ess::kStatusInfeasible)
    return fail(ESS_ERR_INFEASIBLE_X0, "a chain state violates A x <= b (checked in FP64)");
  if (h & ess::kStatusNumeric) return fail(ESS_ERR_NUMERIC, "NaN or Inf in theta or x");
  return ESS_OK;
}
