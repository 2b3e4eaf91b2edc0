// The persistent 1-D propagator, instantiated for one occupancy per
// translation unit: this file is compiled once with -DQG_MINB=1 and once with
// -DQG_MINB=2 so that the two (large) instantiations build in parallel.
#include <cuda_runtime.h>

#include "qg_dom1d.cuh"

#ifndef QG_MINB
#error "compile with -DQG_MINB=1 or -DQG_MINB=2"
#endif

namespace qg {

// Persistent propagator: CTAs take instances from the work counter.  MINB is
// the number of CTAs per SM the launch is built for (1: up to 255 registers
// per thread; 2: 128, twice the warps to hide FP64 latency).
template <int MINB>
__global__ void __launch_bounds__(QG_THREADS, MINB)
    propagate_kernel(const InstDesc* __restrict__ insts, int ninst, const StepPlan P, int* counter,
                     qg_step_stats* stats, int max_n, int max_S, int nb_cap, int stage) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  __shared__ int s_idx;
  const Smem sm = carve_smem(dyn, max_n, nb_cap, P.restart, stage, max_S);
  for (int guard = 0; guard < ninst + 1; ++guard) {
    if (threadIdx.x == 0) s_idx = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= ninst) break;
    const InstDesc I = insts[idx];
    if (P.run == QG_RUN_ADJOINT)
      run_adjoint(I, P, sm, stats + idx, red, sc);
    else
      run_instance(I, P, sm, stats + idx, red, sc);
  }
}

}  // namespace qg

template <>
cudaError_t qg_launch_propagate_minb<QG_MINB>(const InstDesc* d_insts, int ninst, const StepPlan& plan, int* d_counter,
                                              qg_step_stats* d_stats, int max_n, int max_S, int nb, int stage,
                                              size_t smem, int grid, cudaStream_t st) {
  cudaError_t e = qg_allow_max_smem((const void*)qg::propagate_kernel<QG_MINB>);
  if (e != cudaSuccess || grid == 0) return e;   // grid 0: attributes only
  qg::propagate_kernel<QG_MINB><<<grid, QG_THREADS, smem, st>>>(d_insts, ninst, plan, d_counter, d_stats, max_n,
                                                                 max_S, nb, stage);
  return cudaGetLastError();
}
