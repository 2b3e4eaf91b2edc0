// The persistent cluster form of the 1-D propagator for one cluster size G
// (this file is compiled once per G with -DQG_CLUSTER_G=1, 2, 4, 8, 16).
// Cluster c of the launch takes instances c, c + nclusters, ... in the
// table's order; all CTAs of a cluster work on the same instance.
#include <cuda_runtime.h>

#include "qg_cluster.cuh"

#ifndef QG_CLUSTER_G
#error "compile with -DQG_CLUSTER_G=1, 2, 4, 8 or 16"
#endif

namespace qg {

template <int G>
__global__ void __launch_bounds__(QG_THREADS, 1)
    propagate_cluster_kernel(const InstDesc* __restrict__ insts, int ninst, const StepPlan P, qg_step_stats* stats) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  const int cid = blockIdx.x / G, ncl = gridDim.x / G;
  for (int idx = cid; idx < ninst; idx += ncl) {
    const InstDesc I = insts[idx];
    run_cluster_instance<G>(I, P, dyn, red, sc, stats + idx);
  }
}

}  // namespace qg

template <>
cudaError_t qg_launch_cluster_g<QG_CLUSTER_G>(const InstDesc* d_insts, int ninst, const StepPlan& plan,
                                              qg_step_stats* d_stats, size_t smem, cudaStream_t st) {
  constexpr int G = QG_CLUSTER_G;
  auto fn = qg::propagate_cluster_kernel<G>;
  cudaError_t e = qg_allow_max_smem((const void*)fn, G > 8);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(QG_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(G);
  int maxc = 0;
  e = cudaOccupancyMaxActiveClusters(&maxc, fn, &cfg);
  if (e != cudaSuccess) return e;
  if (maxc < 1) return cudaErrorInvalidConfiguration;
  const int ncl = ninst < maxc ? ninst : maxc;
  if (ncl < 1) return cudaSuccess;
  cfg.gridDim = dim3(ncl * G);
  e = cudaLaunchKernelEx(&cfg, fn, d_insts, ninst, plan, d_stats);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
