// ess_batch_persist.cuh -- the persistent launch of the batched mixed-form
// sampler (k_batch_persist.cu): one cooperative kernel runs a whole refresh
// period (q GEMM on the tensor cores, draws, chain steps, overflow chains)
// with work queues, per-problem dependency counters and bounded grid barriers
// (internal to the library).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include "ess_gemm_tc.cuh"
#include "ess_kernels.cuh"

namespace ess {

struct BatchPersistArgs {
  // q GEMM
  const TcBatchItem* titems;
  int n_titems;
  const CUtensorMap* maps[2];  // 4 per problem, over the nu splits of parity 0 / 1
  const float* arow_unscale;
  float* Q;
  // draws of steps 1 .. steps - 1 (step 0's nu is in the parity 0 buffers)
  const ChainDesc* desc;
  float* NU[2];
  __half* H0[2];
  __half* H1[2];
  // chain step: seed, t, t_dev, constants, X (in place), Q, stats, status,
  // desc; P_in, P_out, NU and the lists are set per step
  ChainParams<float> prm;
  float* P[2];        // step j reads P[j % 2] and writes P[(j + 1) % 2]
  const int* order;   // chain order of the work queue (n_chains entries)
  int* queue;         // 2 ints per step: chain tickets, overflow count (zero at launch)
  int* ovf_list;      // n_chains ints: chains left to the overflow phase
  int steps;          // even
  // dependencies: chain steps of problem p in step j wait until dep_done[p]
  // (4 epilogue counts per q item, kept across steps) reaches
  // (j + 1) dep_target[p] + hold
  const int* dep_target;  // per problem: 4 x its q items
  unsigned* dep_done;     // per problem, zero at launch
  unsigned hold;          // 0; 1 in the self-test of the bounded wait (never released)
  unsigned* bar;      // 2 unsigned: grid barrier state (zero at launch)
  int* abort_flag;    // zero at launch
  unsigned long long wait_ns;  // bound of every dependency and grid-barrier wait
};

// Whether the persistent launch can run here: cooperative launches, one
// 1024-thread CTA per SM with its shared memory, and the overflow phase's CTA
// step for rows up to max_m (at most 8192) and states up to max_d.
bool batch_persist_supported(int max_m, int max_d);
// Ints of the queue array for `steps` steps.
inline int batch_persist_queue_ints(int steps) { return 2 * steps; }
// One cooperative launch of the period (grid = the SM count).
cudaError_t launch_batch_persist(const BatchPersistArgs& a, cudaStream_t s);

}  // namespace ess
