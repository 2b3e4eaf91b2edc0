// The 2-D propagator for one precision form per translation unit: compiled
// with -DQG_PREC=0 (complex128 solves) and -DQG_PREC=1 (complex64 inner
// solves refined in FP64), each with -Xptxas -dlcm=cg.
#include <cuda_runtime.h>

#include "qg_dom2d.cuh"

#ifndef QG_PREC
#error "compile with -DQG_PREC=0 or -DQG_PREC=1"
#endif

namespace qg {

template <int MODE>
__global__ void __launch_bounds__(QG_THREADS, 1)
    propagate2d_kernel(const Inst2D I, const StepPlan P, int fft_bytes, int stage_bytes, int tab_off,
                       qg_step_stats* st) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  Dom2D D = make_dom2d(I, dyn, fft_bytes, red, tab_off, stage_bytes);
  const size_t len = D.len;
  Counters cnt{0, 0, 0, 0, 0, 0, 0, 0, 0.0};
  long long nsub = 0;
  const long long failed = run_steps<MODE>(D, P, I.psi, I.work + 2 * len, I.work + 3 * len, I.work + 4 * len,
                                           MODE == 1, I.ckpt, I.nckpt, I.every, cnt, nsub, sc);
  if (blockIdx.x == 0) {
    write_stats(st, cnt, nsub, failed);
    if (threadIdx.x == 0 && !D.good) st->status = QG_ERR_TIMEOUT;
  }
}

}  // namespace qg

template <>
const void* qg_propagate2d_fn<QG_PREC>() {
  return (const void*)qg::propagate2d_kernel<QG_PREC>;
}
