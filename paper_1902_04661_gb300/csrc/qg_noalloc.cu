// The no-allocation entry point's kernels and launch wrapper.
#include <cuda_runtime.h>

#include <mutex>

#include "qg_dom1d.cuh"

// ---------------------------------------------------------------------------
// No-allocation variant of the propagator.
//
// For callers that cannot allocate device memory (for example code that runs
// while another component owns the CUDA allocator, or inside a host
// application that forbids allocation after start-up).  Every scratch buffer
// of one propagation -- the FFT tables, the GMRES workspace and the
// statistics record -- lives in one fixed, file-scope device array instead of
// memory from cudaMalloc.  Capacity: S * N <= QG_NA_MAX_LEN complex values,
// N <= QG_NA_MAX_N, GMRES restart length <= QG_NA_MAX_RESTART.  The array
// (about 3 MB) stays resident on every GPU that loads the library until the
// process exits.  All calls share it: calls that overlap on the GPU would
// race on it, so the host side holds a per-device lock from the start of a
// call until its stream has finished.

namespace qg {

constexpr int kNaMaxLen = QG_NA_MAX_LEN;
constexpr int kNaMaxN = QG_NA_MAX_N;
constexpr int kNaVecs = QG_NA_MAX_RESTART + 5;
constexpr size_t kNaWorkBytes = sizeof(double2) * (size_t)kNaVecs * kNaMaxLen;
constexpr size_t kNaTwBytes = sizeof(double2) * (size_t)kNaMaxN;
constexpr size_t kNaKdBytes = sizeof(double) * (size_t)kNaMaxN;
constexpr size_t kNaStatBytes = 256;
constexpr size_t kNaBytes = kNaWorkBytes + kNaTwBytes + kNaKdBytes + kNaStatBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Twiddles of the radix plan in `plan`, pass by pass (the layout fft_pass
// reads: for forward pass i with block length L, radix R and m = L / R,
// entry (r - 1) m + j holds exp(-2 pi i j r / L)), and the wave numbers of
// the digit-reversed positions (divided by n).
__global__ void noalloc_tables_kernel(unsigned char* base, FftPlan plan, double dq) {
  const int n = plan.n;
  double2* tw = reinterpret_cast<double2*>(base + kNaWorkBytes);
  double* kd = reinterpret_cast<double*>(base + kNaWorkBytes + kNaTwBytes);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int L = n, off = 0, e = 0;
    for (int i = 0; i < plan.npass - 1; ++i) {
      const int R = plan.radix[i], m = L / R, seg = (R - 1) * m;
      if (k < off + seg) {
        const int r = (k - off) / m + 1, j = (k - off) - (r - 1) * m;
        e = j * r * (n / L);
        break;
      }
      off += seg;
      L /= R;
    }
    double s, c;
    sincospi(2.0 * (double)e / (double)n, &s, &c);
    tw[k] = make_double2(c, -s);
    // frequency held at position k after the decimation-in-frequency passes
    int f = 0, mult = 1, rem = k, len = n;
    for (int i = 0; i < plan.npass; ++i) {
      const int m = len / plan.radix[i];
      const int qd = rem / m;
      rem -= qd * m;
      f += mult * qd;
      mult *= plan.radix[i];
      len = m;
    }
    const int ff = f < n / 2 ? f : f - n;
    kd[k] = (2.0 * 3.14159265358979323846 / ((double)n * dq)) * (double)ff / (double)n;
  }
}

struct NaInstance {
  int n, S, npass;
  int radix[QG_MAX_PASSES];
  double h2m, dq;
  const double* V;
  const double* F;
  double2* psi;
};

__global__ void __launch_bounds__(QG_THREADS, 1)
    propagate_noalloc_kernel(unsigned char* base, const NaInstance in, const StepPlan P, int nb_cap) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  InstDesc I;
  I.n = in.n;
  I.S = in.S;
  I.npass = in.npass;
  for (int i = 0; i < QG_MAX_PASSES; ++i) I.radix[i] = in.radix[i];
  I.h2m = in.h2m;
  I.dq = in.dq;
  I.tw = reinterpret_cast<const double2*>(base + kNaWorkBytes);
  I.kd = reinterpret_cast<const double*>(base + kNaWorkBytes + kNaTwBytes);
  I.lf = nullptr;   // the transforms run their twiddle passes from tw
  I.lff = nullptr;
  I.V = in.V;
  I.F = in.F;
  I.psi = in.psi;
  I.work = reinterpret_cast<double2*>(base);
  I.restart_cap = QG_NA_MAX_RESTART;
  I.precision = QG_C128;
  I.tw32 = nullptr;
  I.kd32 = nullptr;
  I.V32 = nullptr;
  I.F32 = nullptr;
  I.work32 = nullptr;
  I.ckpt = nullptr;
  I.nckpt = 0;
  I.every = 1;
  I.grad = nullptr;
  I.gV = nullptr;
  I.gF = nullptr;
  I.rep = 0;
  qg_step_stats* st = reinterpret_cast<qg_step_stats*>(base + kNaWorkBytes + kNaTwBytes + kNaKdBytes);
  const Smem sm = carve_smem(dyn, in.n, nb_cap, P.restart);
  run_instance(I, P, sm, st, red, sc);
}

}  // namespace qg

// Per-device set-up state of the no-allocation entry point (host side),
// guarded by the device's lock.  The tables' key (n, dq) is recorded only
// after the call's stream has finished, so a key always names tables that
// are complete in device memory.
namespace {
constexpr int kNaMaxDevices = 64;
std::mutex g_na_lock[kNaMaxDevices];
unsigned char* g_na_ptr[kNaMaxDevices] = {nullptr};
int g_na_tab_n[kNaMaxDevices] = {0};
double g_na_tab_dq[kNaMaxDevices] = {0.0};
}  // namespace

cudaError_t qg_noalloc_launch(int n, double qmin, double qmax, int S, double mass, const double* V, const double* F,
                              double2* psi, const FftPlan& plan, const StepPlan& P, qg_step_stats* host_stats,
                              cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  // one call at a time per device: the scratch array is shared by every call
  std::lock_guard<std::mutex> hold(g_na_lock[dev]);
  if (!g_na_ptr[dev]) {
    // The symbol's name in host code is only a stand-in: take the device
    // address of this device's copy once, with the device current.
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, qg::g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = reinterpret_cast<unsigned char*>(p);
    g_na_tab_n[dev] = 0;
  }
  unsigned char* base = g_na_ptr[dev];
  const double dq = (qmax - qmin) / n;
  const bool rebuild = g_na_tab_n[dev] != n || g_na_tab_dq[dev] != dq;
  if (rebuild) {
    g_na_tab_n[dev] = 0;   // invalid until this call's stream has finished
    qg::noalloc_tables_kernel<<<(n + 255) / 256, 256, 0, st>>>(base, plan, dq);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  size_t smem;
  const int nb = nb_capacity(n, S, P.restart, &smem);
  e = qg_allow_max_smem((const void*)qg::propagate_noalloc_kernel);
  if (e != cudaSuccess) return e;
  qg::NaInstance in;
  in.n = n;
  in.S = S;
  in.npass = plan.npass;
  for (int i = 0; i < QG_MAX_PASSES; ++i) in.radix[i] = plan.radix[i];
  in.h2m = 1.0 / (2.0 * mass);
  in.dq = dq;
  in.V = V;
  in.F = F;
  in.psi = psi;
  qg::propagate_noalloc_kernel<<<1, QG_THREADS, smem, st>>>(base, in, P, nb);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(host_stats, base + qg::kNaWorkBytes + qg::kNaTwBytes + qg::kNaKdBytes, sizeof(qg_step_stats),
                      cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && rebuild) {
    g_na_tab_n[dev] = n;
    g_na_tab_dq[dev] = dq;
  }
  return e;
}

