// k_chain_warp.cu -- one elliptical-slice step per chain, one WARP per chain
// (the step itself is warp_chain_step, chain_warp_step.cuh): 8 chains per
// CTA, 4 CTAs per SM for float chains.  A chain with more than 128 surviving
// arcs is either listed for the CTA-per-chain kernel, or (LOCAL) stepped at
// the end of the same CTA by the CTA-per-chain step with the CTA's 256
// threads, which saves the list, its reset and the second launch per step.
#include "chain_cta_step.cuh"
#include "chain_warp_step.cuh"

namespace ess {
namespace {

constexpr int kWarps = 8;  // chains per CTA
// LOCAL: the CTA-per-chain step of 256 threads x kChainItems rows
constexpr int kLocalThreads = kWarps * 32;

// The CTA-per-chain step of one chain the warps left (inlined: a call would
// make the kernel keep registers across it, measured 1 % slower).
template <typename T, bool BATCH>
__device__ __forceinline__ void local_cta_step(const ChainParams<T>& prm, int c,
                                               unsigned char* smem, uint32_t bytes) {
  cta_chain_step<T, kLocalThreads, kChainItems, BATCH>(prm, c, smem, bytes);
}

template <typename T, int WARPS, bool BATCH, bool LONG, bool LOCAL>
__global__ void __launch_bounds__(WARPS * 32,
                                  sizeof(T) == 4 ? ESS_WARP_MINBLOCKS : ESS_WARP_MINBLOCKS_F64)
chain_warp_kernel(ChainParams<T> prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ unsigned long long s_sort_keys;
  __shared__ int s_left[WARPS];
  __shared__ int s_nleft;
  if (threadIdx.x == 0) {
    s_sort_keys = 0;
    s_nleft = 0;
  }
  __syncthreads();
  const int c = blockIdx.x * WARPS + warp;
  if (c < prm.n_chains) {
    const int keys =
        warp_chain_step<T, BATCH, LONG>(prm, c, smem_raw + kWarpStepSmem * warp, lane);
    if (lane == 0 && keys > 0) atomicAdd(&s_sort_keys, (unsigned long long)keys);
    if constexpr (LOCAL) {
      if (lane == 0 && keys < 0) s_left[atomicAdd(&s_nleft, 1)] = c;
    }
  }
  __syncthreads();
  if constexpr (LOCAL) {
    // the chains this CTA's warps left, by the whole CTA (uniform count)
    const int n_left = s_nleft;
    if (n_left > 0) {
      uint32_t dyn_smem;
      asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
      for (int k = 0; k < n_left; ++k)
        local_cta_step<T, BATCH>(prm, s_left[k], smem_raw, dyn_smem);
    }
  }
  if (threadIdx.x == 0 && s_sort_keys) atomicAdd(&prm.stats->sort_keys, s_sort_keys);
}

}  // namespace

template <typename T>
size_t chain_warp_smem_bytes(int m) {
  (void)m;
  return (size_t)kWarps * kWarpStepSmem;
}

template <typename T>
bool chain_warp_local_fallback(int m, int d) {
  return sizeof(T) == 4 && m <= kLocalThreads * kChainItems &&
         chain_smem_bytes<T>(kLocalThreads, d) <= chain_warp_smem_bytes<T>(m);
}

template <typename T>
cudaError_t launch_chain_step_warp(const ChainParams<T>& p, cudaStream_t s) {
  if (p.n_chains <= 0) return cudaSuccess;
  const bool local = p.overflow_list == nullptr;
  if (p.P_out == p.P_in || (!local && !p.overflow_count)) return cudaErrorInvalidValue;
  if (local && !chain_warp_local_fallback<T>(p.m, p.d)) return cudaErrorInvalidValue;
  if (sizeof(T) == 4 && p.slack == nullptr) return cudaErrorInvalidValue;
  const size_t smem = chain_warp_smem_bytes<T>(p.m);
  // the long-arc union is compiled in only when some row has b_i <= 0
  void (*k)(ChainParams<T>);
  if (local) {
    if constexpr (sizeof(T) == 4) {
      k = p.desc ? (p.long_arcs ? chain_warp_kernel<T, kWarps, true, true, true>
                                : chain_warp_kernel<T, kWarps, true, false, true>)
                 : (p.long_arcs ? chain_warp_kernel<T, kWarps, false, true, true>
                                : chain_warp_kernel<T, kWarps, false, false, true>);
    } else {
      return cudaErrorInvalidValue;
    }
  } else {
    k = p.desc ? (p.long_arcs ? chain_warp_kernel<T, kWarps, true, true, false>
                              : chain_warp_kernel<T, kWarps, true, false, false>)
               : (p.long_arcs ? chain_warp_kernel<T, kWarps, false, true, false>
                              : chain_warp_kernel<T, kWarps, false, false, false>);
  }
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((p.n_chains + kWarps - 1) / kWarps);
  k<<<grid, kWarps * 32, smem, s>>>(p);
  return cudaGetLastError();
}

template size_t chain_warp_smem_bytes<float>(int);
template size_t chain_warp_smem_bytes<double>(int);
template bool chain_warp_local_fallback<float>(int, int);
template bool chain_warp_local_fallback<double>(int, int);
template cudaError_t launch_chain_step_warp<float>(const ChainParams<float>&, cudaStream_t);
template cudaError_t launch_chain_step_warp<double>(const ChainParams<double>&, cudaStream_t);

}  // namespace ess
