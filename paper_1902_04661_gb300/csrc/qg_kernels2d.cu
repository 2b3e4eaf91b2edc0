// Two-dimensional grids: the Hamiltonian action and energy, the Gaussian
// initial state, the grid-barrier self-test and the host launch wrappers (the
// propagator kernels are in their own translation units).  Compiled with
// -Xptxas -dlcm=cg like every unit that uses the 2-D domain.
#include <cuda_runtime.h>

#include "qg_dom2d.cuh"

namespace qg {

// out = H psi (c = 1) or <psi|H|psi> (energy != null).
__global__ void __launch_bounds__(QG_THREADS, 1) apply_h2d_kernel(const Inst2D I, int fft_bytes, int stage_bytes,
                                                                  int tab_off, double2* out, double* energy) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  Dom2D D = make_dom2d(I, dyn, fft_bytes, red, tab_off, stage_bytes);
  D.hpsi<double>(I.psi, out, nullptr, 0.0, 0.0, make_double2(1.0, 0.0));
  if (energy) {
    double v[2] = {0.0, 0.0};
    D.each([&](int i) {
      const double2 p = I.psi[i], h = out[i];
      v[0] = fma(p.x, h.x, fma(p.y, h.y, v[0]));
      v[1] = fma(p.x, h.y, fma(-p.y, h.x, v[1]));
    });
    D.sum<2>(v, sc);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      energy[0] = I.dv * sc[0];
      energy[1] = I.dv * sc[1];
    }
  }
}

// Product Gaussian on one surface of a 2-D grid, zero elsewhere, normalised.
__global__ void __launch_bounds__(QG_THREADS)
    gaussian2d_kernel(double2* psi, int n0, int n1, int S, int surface, double qmin0, double qmin1, double dq0,
                      double dq1, double q00, double q01, double p00, double p01, double s00, double s01) {
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  const int N = n0 * n1;
  const double w0 = 1.0 / (4.0 * s00 * s00), w1 = 1.0 / (4.0 * s01 * s01);
  double v[1] = {0.0};
  for (int p = threadIdx.x; p < N; p += kThreads) {
    const int i = p / n1, j = p - i * n1;
    const double x0 = (qmin0 + dq0 * i) - q00, x1 = (qmin1 + dq1 * j) - q01;
    const double amp = exp(-w0 * x0 * x0 - w1 * x1 * x1);
    double sn, cs;
    sincos(p00 * x0 + p01 * x1, &sn, &cs);
    psi[(size_t)surface * N + p] = make_double2(amp * cs, amp * sn);
    v[0] = fma(amp, amp, v[0]);
  }
  cta_sum<1>(v, red, sc);
  const double scale = 1.0 / sqrt(dq0 * dq1 * sc[0]);
  for (int s = 0; s < S; ++s)
    for (int p = threadIdx.x; p < N; p += kThreads) {
      const size_t i = (size_t)s * N + p;
      psi[i] = (s == surface) ? cscale(scale, psi[i]) : make_double2(0.0, 0.0);
    }
}

// Failure-path check of grid_barrier: CTA `absent` never arrives, so every
// other CTA's wait must run out, raise the flag and return false.
__global__ void barrier_timeout_kernel(unsigned* bar, int* err, int absent, int* ok_count) {
  if ((int)blockIdx.x == absent) return;
  const bool ok = grid_barrier(bar, err);
  if (threadIdx.x == 0 && ok) atomicAdd(ok_count, 1);
}

}  // namespace qg

cudaError_t qg_selftest_barrier(int* d_words, int* h_timed_out, int* h_passed) {
  // d_words: 4 ints of device scratch (count, generation, error flag, passes)
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int G = sms < 8 ? sms : 8;
  cudaError_t e = cudaMemset(d_words, 0, 4 * sizeof(int));
  if (e != cudaSuccess) return e;
  unsigned* bar = reinterpret_cast<unsigned*>(d_words);
  int* err = d_words + 2;
  int* okc = d_words + 3;
  int absent = 0;
  void* args[] = {&bar, &err, &absent, &okc};
  e = cudaLaunchCooperativeKernel((const void*)qg::barrier_timeout_kernel, dim3(G), dim3(32), args, 0, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d_words, sizeof(h), cudaMemcpyDeviceToHost);
  if (h_timed_out) *h_timed_out = h[2];
  if (h_passed) *h_passed = h[3];
  return e;
}

int qg_grid2d_ctas(const Inst2D& I);

// One FFT batch holds every owned row (or column) of every surface.
static size_t fft2d_bytes(const Inst2D& I) {
  const int G = qg_grid2d_ctas(I);
  const int rp = (I.n[0] + G - 1) / G, cp = (I.n[1] + G - 1) / G;
  const size_t rows = (size_t)rp * I.n[1], cols = (size_t)cp * I.n[0];
  const int nmax = I.n[0] > I.n[1] ? I.n[0] : I.n[1];
  size_t want = (size_t)I.S * (rows > cols ? rows : cols);
  // at most 96 KB of batch; always room for one row or column of every surface
  const size_t cap = (size_t)96 * 1024 / 18;
  if (want > cap) want = cap;
  if (want < (size_t)I.S * nmax) want = (size_t)I.S * nmax;
  return qg::padded_bytes(want, sizeof(double2));
}

int qg_grid2d_ctas(const Inst2D& I) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int lim = I.n[0] < I.n[1] ? I.n[0] : I.n[1];
  int G = 1;
  while (G * 2 <= sms && G * 2 <= lim) G *= 2;
  if (I.ctas > 0 && I.ctas < G) G = I.ctas;
  return G;
}

static cudaError_t coop_launch(const void* fn, int G, size_t smem, void** args, cudaStream_t st) {
  cudaError_t e = qg_allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!coop) return cudaErrorNotSupported;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, QG_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm * sms < G) return cudaErrorCooperativeLaunchTooLarge;
  return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(QG_THREADS), args, smem, st);
}

// The FFT tables go to shared memory after the kernel's other arrays when
// the total stays within 200 KB; otherwise they are read from global memory
// (tab_off = 0).
static size_t with_tables(const Inst2D& I, size_t smem, int* tab_off) {
  const size_t off = (smem + 15) / 16 * 16;
  const size_t tab = qg::tables2d_bytes(I.n[0], I.n[1]);
  if (off + tab > (size_t)200 * 1024) {
    *tab_off = 0;
    return smem;
  }
  *tab_off = (int)off;
  return off + tab;
}

// Shared copies of x and U for one FFT batch (two arrays of the batch's
// complex-double capacity) when they fit beside the batch within 160 KB.
static int stage2d_bytes(int fft_bytes) {
  const size_t st = 2 * 16 * qg::padded_capacity((size_t)fft_bytes, 16);
  return (size_t)fft_bytes + st <= (size_t)160 * 1024 ? (int)st : 0;
}

cudaError_t qg_launch_propagate2d(const Inst2D& I, const StepPlan& P, qg_step_stats* d_stats, cudaStream_t st) {
  const int G = qg_grid2d_ctas(I);
  int fft = (int)fft2d_bytes(I);
  int stage = stage2d_bytes(fft);
  int tab_off = 0;
  const size_t smem = with_tables(I, fft + stage + qg::gmres_smem_bytes(P.restart), &tab_off);
  cudaError_t e = cudaMemsetAsync(I.bar, 0, 2 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  Inst2D Ic = I;
  StepPlan Pc = P;
  void* args[] = {&Ic, &Pc, &fft, &stage, &tab_off, &d_stats};
  const void* fn = I.precision == QG_C64_MIXED ? qg_propagate2d_fn<1>() : qg_propagate2d_fn<0>();
  return coop_launch(fn, G, smem, args, st);
}

cudaError_t qg_launch_apply_h2d(const Inst2D& I, double2* d_out, double* d_energy, cudaStream_t st) {
  const int G = qg_grid2d_ctas(I);
  int fft = (int)fft2d_bytes(I);
  int stage = stage2d_bytes(fft);
  int tab_off = 0;
  const size_t smem = with_tables(I, fft + stage + qg::gmres_smem_bytes(1), &tab_off);
  cudaError_t e = cudaMemsetAsync(I.bar, 0, 2 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  Inst2D Ic = I;
  void* args[] = {&Ic, &fft, &stage, &tab_off, &d_out, &d_energy};
  return coop_launch((const void*)qg::apply_h2d_kernel, G, smem, args, st);
}

cudaError_t qg_launch_gaussian2d(double2* d_psi, const int* n, int S, int surface, const double* qmin,
                                 const double* dq, const double* q0, const double* p0, const double* s0,
                                 cudaStream_t st) {
  qg::gaussian2d_kernel<<<1, QG_THREADS, 0, st>>>(d_psi, n[0], n[1], S, surface, qmin[0], qmin[1], dq[0], dq[1],
                                                   q0[0], q0[1], p0[0], p0[1], s0[0], s0[1]);
  return cudaGetLastError();
}
