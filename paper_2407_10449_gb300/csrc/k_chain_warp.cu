// k_chain_warp.cu -- one elliptical-slice step per chain, one WARP per chain
// (the step itself is warp_chain_step, chain_warp_step.cuh): 8 chains per
// CTA, 4 CTAs per SM for float chains.  Chains with more than 128 surviving
// arcs are listed for the CTA-per-chain kernel.
#include "chain_warp_step.cuh"

namespace ess {
namespace {

constexpr int kWarps = 8;  // chains per CTA

template <typename T, int WARPS, bool BATCH, bool LONG>
__global__ void __launch_bounds__(WARPS * 32,
                                  sizeof(T) == 4 ? ESS_WARP_MINBLOCKS : ESS_WARP_MINBLOCKS_F64)
chain_warp_kernel(ChainParams<T> prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ unsigned long long s_sort_keys;
  if (threadIdx.x == 0) s_sort_keys = 0;
  __syncthreads();
  const int c = blockIdx.x * WARPS + warp;
  if (c < prm.n_chains) {
    const int keys =
        warp_chain_step<T, BATCH, LONG>(prm, c, smem_raw + kWarpStepSmem * warp, lane);
    if (lane == 0 && keys) atomicAdd(&s_sort_keys, (unsigned long long)keys);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_sort_keys) atomicAdd(&prm.stats->sort_keys, s_sort_keys);
}

}  // namespace

template <typename T>
size_t chain_warp_smem_bytes(int m) {
  (void)m;
  return (size_t)kWarps * kWarpStepSmem;
}

template <typename T>
cudaError_t launch_chain_step_warp(const ChainParams<T>& p, cudaStream_t s) {
  if (p.n_chains <= 0) return cudaSuccess;
  if (p.P_out == p.P_in || !p.overflow_list || !p.overflow_count) return cudaErrorInvalidValue;
  if (sizeof(T) == 4 && p.slack == nullptr) return cudaErrorInvalidValue;
  const size_t smem = chain_warp_smem_bytes<T>(p.m);
  // the long-arc union is compiled in only when some row has b_i <= 0
  auto k = p.desc ? (p.long_arcs ? chain_warp_kernel<T, kWarps, true, true>
                                 : chain_warp_kernel<T, kWarps, true, false>)
                  : (p.long_arcs ? chain_warp_kernel<T, kWarps, false, true>
                                 : chain_warp_kernel<T, kWarps, false, false>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((p.n_chains + kWarps - 1) / kWarps);
  k<<<grid, kWarps * 32, smem, s>>>(p);
  return cudaGetLastError();
}

template size_t chain_warp_smem_bytes<float>(int);
template size_t chain_warp_smem_bytes<double>(int);
template cudaError_t launch_chain_step_warp<float>(const ChainParams<float>&, cudaStream_t);
template cudaError_t launch_chain_step_warp<double>(const ChainParams<double>&, cudaStream_t);

}  // namespace ess
