// k_chain.cu -- one elliptical-slice step per chain, one CTA per chain (the
// step itself is cta_chain_step, chain_cta_step.cuh: App. B roots, Alg. 3
// by a per-bucket interval merge or a sort, inverse-CDF theta, move and the
// Sec. 3.3 safeguard).  T = double is the plain FP64 form, T = float the
// mixed form.
#include "chain_cta_step.cuh"

namespace ess {
namespace {

template <typename T, int NT, int ITEMS, bool BATCH>
__global__ void __launch_bounds__(NT, (768 / NT > 0 ? 768 / NT : 1)) chain_step_kernel(ChainParams<T> prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t dyn_smem;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
  // one chain per CTA, or (list mode) the chains of prm.chain_list, strided
  // over the grid
  const int n_work = prm.chain_list ? *prm.list_count : prm.n_chains;
  for (int work = blockIdx.x; work < n_work; work += gridDim.x) {
    const int c = prm.chain_list ? prm.chain_list[work] : work;
    cta_chain_step<T, NT, ITEMS, BATCH>(prm, c, smem_raw, dyn_smem);
  }
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
  // keys, values, x', flags (the launch adds the merge buckets when they fit)
  return 2 * npad * sizeof(T) + (size_t)((d + 1) & ~1) * sizeof(T) + nslot * sizeof(int);
}

template <typename T>
cudaError_t launch_chain_step(const ChainParams<T>& p, int threads, cudaStream_t s) {
  // the per-bucket interval merge needs two more arrays of min(threads *
  // kChainItems, merge_buckets<T>()) values; without them the kernel sorts
  size_t smem = chain_smem_bytes<T>(threads, p.d);
  const size_t merge =
      2 * std::min((size_t)threads * kChainItems, (size_t)merge_buckets<T>()) * sizeof(T);
  if (smem + merge <= (size_t)227 * 1024) smem += merge;
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // list mode: a grid that fills the GPU once and strides over the list
  dim3 grid(p.chain_list ? (unsigned)std::min(p.n_chains, sms * std::max(1, 768 / threads))
                         : (unsigned)p.n_chains);
  if (grid.x == 0) return cudaSuccess;
#define ESS_CHAIN_CASE(NT)                                                              \
  case NT: {                                                                            \
    auto k = p.desc ? chain_step_kernel<T, NT, kChainItems, true>                       \
                    : chain_step_kernel<T, NT, kChainItems, false>;                     \
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
