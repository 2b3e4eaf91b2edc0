// Kernels of libqgeom: the persistent propagator (composed trapezoidal /
// implicit-midpoint steps with GMRES implicit solves), the Hamiltonian action,
// observables, the Gaussian initial state and the two-state diabatic ->
// adiabatic field builder.
#include <cuda_runtime.h>

#include "qg_device.cuh"

namespace qg {

// Shared-memory layout of one CTA (dynamic part).
struct Smem {
  double2* fft;    // nb_cap * max_n
  double2* hess;   // (m + 1) * m, column j at hess + j * (m + 1)
  double2* g;      // m + 1
  double2* gs;     // m   Givens s
  double* gc;      // m   Givens c
  double2* y;      // m
  int nb_cap;
};

__device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

__device__ Smem carve_smem(void* base, int max_n, int nb_cap, int m) {
  Smem s;
  char* p = reinterpret_cast<char*>(base);
  s.fft = reinterpret_cast<double2*>(p);
  p += align16(sizeof(double2) * (size_t)nb_cap * max_n);
  s.hess = reinterpret_cast<double2*>(p);
  p += align16(sizeof(double2) * (size_t)(m + 1) * m);
  s.g = reinterpret_cast<double2*>(p);
  p += align16(sizeof(double2) * (size_t)(m + 1));
  s.gs = reinterpret_cast<double2*>(p);
  p += align16(sizeof(double2) * (size_t)m);
  s.y = reinterpret_cast<double2*>(p);
  p += align16(sizeof(double2) * (size_t)m);
  s.gc = reinterpret_cast<double*>(p);
  s.nb_cap = nb_cap;
  return s;
}

struct Counters {
  long long hpsi;
  long long krylov;
  long long ortho;
  long long update;
  long long restart;
  int max_krylov;
  double max_res;
};

// Solve (1 + i tau H) x = b by restarted GMRES (Sec. II B) in the grid inner
// product.  X holds the initial guess on entry and the solution on exit.
// Returns true on convergence (estimated relative residual <= tol).
__device__ bool gmres_solve(const InstDesc& I, const Smem& sm, const StepPlan& P, double tau, const double2* b,
                            double2* X, Counters& cnt, double* red, double* sc) {
  const int len = I.S * I.n;
  const double dv = I.dq;
  const int m = P.restart;
  double2* basis = I.work + (size_t)4 * len;
  const double2 ic = make_double2(0.0, tau);     // A = 1 + i tau H
  const double2 mic = make_double2(0.0, -tau);
  const double bn = sqrt(dv * cta_norm2(b, len, red, sc));
  const double target = P.tol * bn;
  int total = 0;
  int this_solve = 0;
  // r0 = b - A X
  apply_h_axpby(I, sm.fft, sm.nb_cap, X, basis, b, 1.0, -1.0, mic);
  cnt.hpsi++;
  for (int guard = 0; guard < P.max_iters + 2; ++guard) {
    double2* V0 = basis;
    const double beta = sqrt(dv * cta_norm2(V0, len, red, sc));
    if (beta <= target || bn == 0.0) {
      double r = (bn > 0.0) ? beta / bn : 0.0;
      if (r > cnt.max_res) cnt.max_res = r;
      if (this_solve > cnt.max_krylov) cnt.max_krylov = this_solve;
      return true;
    }
    if (total >= P.max_iters) break;
    const double ib = 1.0 / beta;
    for (int i = threadIdx.x; i < len; i += kThreads) V0[i] = cscale(ib, V0[i]);
    if (threadIdx.x == 0) {
      sm.g[0] = make_double2(beta, 0.0);
      for (int i = 1; i <= m; ++i) sm.g[i] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    int ncol = 0;
    bool conv = false;
    double res_est = beta;
    for (int j = 0; j < m; ++j) {
      double2* Vj = basis + (size_t)j * len;
      double2* W = basis + (size_t)(j + 1) * len;
      apply_h_axpby(I, sm.fft, sm.nb_cap, Vj, W, nullptr, 0.0, 1.0, ic);
      cnt.hpsi++;
      double2* hcol = sm.hess + (size_t)j * (m + 1);
      if (threadIdx.x <= j + 1) hcol[threadIdx.x] = make_double2(0.0, 0.0);
      __syncthreads();
      // Classical Gram-Schmidt, optionally repeated once (CGS2).
      for (int pass = 0; pass < (P.reorth ? 2 : 1); ++pass) {
        for (int c0 = 0; c0 <= j; c0 += 8) {
          const int nc = min(8, j + 1 - c0);
          double v[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = 0.0;
          for (int i = threadIdx.x; i < len; i += kThreads) {
            const double2 w = W[i];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              if (k < nc) {
                const double2 q = basis[(size_t)(c0 + k) * len + i];
                v[2 * k] = fma(q.x, w.x, fma(q.y, w.y, v[2 * k]));
                v[2 * k + 1] = fma(q.x, w.y, fma(-q.y, w.x, v[2 * k + 1]));
              }
            }
          }
          cta_sum<16>(v, red, sc);
          if (threadIdx.x < nc) {
            const double2 h = make_double2(dv * sc[2 * threadIdx.x], dv * sc[2 * threadIdx.x + 1]);
            hcol[c0 + threadIdx.x] = cadd(hcol[c0 + threadIdx.x], h);
            sc[32 + 2 * threadIdx.x] = h.x;
            sc[33 + 2 * threadIdx.x] = h.y;
          }
          __syncthreads();
          double2 hk[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) hk[k] = (k < nc) ? make_double2(sc[32 + 2 * k], sc[33 + 2 * k]) : make_double2(0, 0);
          __syncthreads();
          for (int i = threadIdx.x; i < len; i += kThreads) {
            double2 w = W[i];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (k < nc) w = cnaxpy(hk[k], basis[(size_t)(c0 + k) * len + i], w);
            W[i] = w;
          }
          __syncthreads();
        }
      }
      const double hn = sqrt(dv * cta_norm2(W, len, red, sc));
      if (hn > 1e-300) {
        const double ih = 1.0 / hn;
        for (int i = threadIdx.x; i < len; i += kThreads) W[i] = cscale(ih, W[i]);
      }
      if (threadIdx.x == 0) {
        hcol[j + 1] = make_double2(hn, 0.0);
        // previous rotations
        for (int i = 0; i < j; ++i) {
          const double c = sm.gc[i];
          const double2 s = sm.gs[i];
          const double2 h0 = hcol[i], h1 = hcol[i + 1];
          const double2 t = caxpy(s, h1, cscale(c, h0));                       // c h0 + s h1
          const double2 u = cnaxpy(make_double2(s.x, -s.y), h0, cscale(c, h1));  // -conj(s) h0 + c h1
          hcol[i] = t;
          hcol[i + 1] = u;
        }
        // new rotation zeroing hcol[j+1]
        const double2 a = hcol[j];
        const double bb = hcol[j + 1].x;
        const double aa = hypot(a.x, a.y);
        double c;
        double2 s, r;
        if (bb == 0.0) {
          c = 1.0;
          s = make_double2(0.0, 0.0);
          r = a;
        } else if (aa == 0.0) {
          c = 0.0;
          s = make_double2(1.0, 0.0);
          r = make_double2(bb, 0.0);
        } else {
          const double rho = hypot(aa, bb);
          const double2 ph = make_double2(a.x / aa, a.y / aa);
          c = aa / rho;
          s = make_double2(ph.x * bb / rho, ph.y * bb / rho);
          r = make_double2(ph.x * rho, ph.y * rho);
        }
        sm.gc[j] = c;
        sm.gs[j] = s;
        hcol[j] = r;
        hcol[j + 1] = make_double2(0.0, 0.0);
        const double2 gj = sm.g[j];
        sm.g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
        sm.g[j] = cscale(c, gj);
        sc[0] = hypot(sm.g[j + 1].x, sm.g[j + 1].y);
      }
      __syncthreads();
      res_est = sc[0];
      __syncthreads();
      ncol = j + 1;
      cnt.ortho += j + 1;
      total++;
      this_solve++;
      cnt.krylov++;
      if (res_est <= target) {
        conv = true;
        break;
      }
      if (total >= P.max_iters || hn <= 1e-300) break;
    }
    // y = R^{-1} g (upper triangular ncol x ncol)
    if (threadIdx.x == 0) {
      for (int i = ncol - 1; i >= 0; --i) {
        double2 acc = sm.g[i];
        for (int k = i + 1; k < ncol; ++k) acc = cnaxpy(sm.hess[(size_t)k * (m + 1) + i], sm.y[k], acc);
        const double2 d = sm.hess[(size_t)i * (m + 1) + i];
        const double dd = 1.0 / fma(d.x, d.x, d.y * d.y);
        sm.y[i] = make_double2((acc.x * d.x + acc.y * d.y) * dd, (acc.y * d.x - acc.x * d.y) * dd);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += kThreads) {
      double2 x = X[i];
      for (int k = 0; k < ncol; ++k) x = caxpy(sm.y[k], basis[(size_t)k * len + i], x);
      X[i] = x;
    }
    cnt.update += ncol;
    __syncthreads();
    if (conv && !P.true_res) {
      const double r = (bn > 0.0) ? res_est / bn : 0.0;
      if (r > cnt.max_res) cnt.max_res = r;
      if (this_solve > cnt.max_krylov) cnt.max_krylov = this_solve;
      return true;
    }
    if (total >= P.max_iters && !conv) break;
    // restart (or true-residual check): V0 = b - A X
    apply_h_axpby(I, sm.fft, sm.nb_cap, X, basis, b, 1.0, -1.0, mic);
    cnt.hpsi++;
    cnt.restart++;
  }
  if (this_solve > cnt.max_krylov) cnt.max_krylov = this_solve;
  cnt.max_res = 1e300;
  return false;
}

__device__ __forceinline__ void vcopy(double2* dst, const double2* src, int len) {
  for (int i = threadIdx.x; i < len; i += kThreads) dst[i] = src[i];
  __syncthreads();
}

// All nsteps composed steps of one instance.
__device__ void run_instance(const InstDesc& I, const StepPlan& P, const Smem& sm, qg_step_stats* st, double* red,
                             double* sc) {
  const int len = I.S * I.n;
  double2* psi = I.psi;
  double2* B = I.work + (size_t)1 * len;
  double2* X = I.work + (size_t)2 * len;
  double2* P0 = I.work + (size_t)3 * len;
  Counters cnt{0, 0, 0, 0, 0, 0, 0.0};
  long long nsub = 0;
  long long failed = -1;
  vcopy(P0, psi, len);
  for (long long step = 0; step < P.nsteps && failed < 0; ++step) {
    for (int f = 0; f < P.nfrac; ++f) {
      const double tau = 0.5 * P.frac[f] * P.dt;   // hbar = 1
      const double2 mic = make_double2(0.0, -tau);
      bool ok;
      if (P.method == QG_TRAPEZOIDAL) {
        // b = (1 - i tau H) psi ; guess x0 = (1 - i tau H) b ; solve (1 + i tau H) x = b
        apply_h_axpby(I, sm.fft, sm.nb_cap, psi, B, nullptr, 0.0, 1.0, mic);
        apply_h_axpby(I, sm.fft, sm.nb_cap, B, X, nullptr, 0.0, 1.0, mic);
        cnt.hpsi += 2;
        ok = gmres_solve(I, sm, P, tau, B, X, cnt, red, sc);
        if (ok) vcopy(psi, X, len);
      } else {
        // guess chi0 = (1 - i tau H) psi ; solve (1 + i tau H) chi = psi ;
        // psi' = (1 - i tau H) chi  (or 2 chi - psi)
        apply_h_axpby(I, sm.fft, sm.nb_cap, psi, X, nullptr, 0.0, 1.0, mic);
        cnt.hpsi += 1;
        ok = gmres_solve(I, sm, P, tau, psi, X, cnt, red, sc);
        if (ok) {
          if (P.mid_epi) {
            apply_h_axpby(I, sm.fft, sm.nb_cap, X, psi, nullptr, 0.0, 1.0, mic);
            cnt.hpsi += 1;
          } else {
            for (int i = threadIdx.x; i < len; i += kThreads) {
              const double2 c = X[i], p = psi[i];
              psi[i] = make_double2(2.0 * c.x - p.x, 2.0 * c.y - p.y);
            }
            __syncthreads();
          }
        }
      }
      if (!ok) {
        failed = step;
        break;
      }
      nsub++;
    }
  }
  if (failed >= 0) vcopy(psi, P0, len);
  if (threadIdx.x == 0) {
    st->n_hpsi = cnt.hpsi;
    st->n_krylov = cnt.krylov;
    st->n_substeps = nsub;
    st->max_krylov = cnt.max_krylov;
    st->status = failed >= 0 ? QG_ERR_NOT_CONVERGED : QG_OK;
    st->max_residual = cnt.max_res;
    st->failed_step = failed;
    st->n_ortho = cnt.ortho;
    st->n_update = cnt.update;
    st->n_restart = cnt.restart;
  }
}

__global__ void __launch_bounds__(QG_THREADS, 1)
    propagate_kernel(const InstDesc* __restrict__ insts, int ninst, const StepPlan P, int* counter,
                     qg_step_stats* stats, int max_n, int nb_cap) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  __shared__ int s_idx;
  const Smem sm = carve_smem(dyn, max_n, nb_cap, P.restart);
  for (int guard = 0; guard < ninst + 1; ++guard) {
    if (threadIdx.x == 0) s_idx = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= ninst) break;
    const InstDesc I = insts[idx];
    run_instance(I, P, sm, stats + idx, red, sc);
  }
}

__global__ void __launch_bounds__(QG_THREADS, 1)
    apply_h_kernel(const InstDesc* __restrict__ inst, double2* out, int nb_cap) {
  extern __shared__ __align__(16) unsigned char dyn[];
  const InstDesc I = *inst;
  apply_h_axpby(I, reinterpret_cast<double2*>(dyn), nb_cap, I.psi, out, nullptr, 0.0, 0.0,
                make_double2(1.0, 0.0));
}

// <psi|H|psi> with H psi written to the scratch vector B of the workspace.
__global__ void __launch_bounds__(QG_THREADS, 1)
    energy_kernel(const InstDesc* __restrict__ inst, double* out, int nb_cap) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  const InstDesc I = *inst;
  const int len = I.S * I.n;
  double2* Hx = I.work + (size_t)1 * len;
  apply_h_axpby(I, reinterpret_cast<double2*>(dyn), nb_cap, I.psi, Hx, nullptr, 0.0, 0.0, make_double2(1.0, 0.0));
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < len; i += kThreads) {
    const double2 p = I.psi[i], h = Hx[i];
    v[0] = fma(p.x, h.x, fma(p.y, h.y, v[0]));
    v[1] = fma(p.x, h.y, fma(-p.y, h.x, v[1]));
  }
  cta_sum<2>(v, red, sc);
  if (threadIdx.x == 0) {
    out[0] = I.dq * sc[0];
    out[1] = I.dq * sc[1];
  }
}

__global__ void __launch_bounds__(QG_THREADS)
    populations_kernel(const double2* __restrict__ psi, int n, int S, double dq, double* out) {
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  for (int s = 0; s < S; ++s) {
    const double r = cta_norm2(psi + (size_t)s * n, n, red, sc);
    if (threadIdx.x == 0) out[s] = dq * r;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(QG_THREADS)
    overlap_kernel(const double2* __restrict__ a, const double2* __restrict__ b, int len, double dq, double* out) {
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < len; i += kThreads) {
    const double2 p = a[i], h = b[i];
    v[0] = fma(p.x, h.x, fma(p.y, h.y, v[0]));
    v[1] = fma(p.x, h.y, fma(-p.y, h.x, v[1]));
  }
  cta_sum<2>(v, red, sc);
  if (threadIdx.x == 0) {
    out[0] = dq * sc[0];
    out[1] = dq * sc[1];
  }
}

// Gaussian of Sec. III on one surface, zero elsewhere, normalised on the grid.
__global__ void __launch_bounds__(QG_THREADS)
    gaussian_kernel(double2* psi, int n, int S, int surface, double qmin, double dq, double q0, double p0,
                    double sigma0) {
  __shared__ double red[kWarps * 16];
  __shared__ double sc[64];
  const double w = 1.0 / (4.0 * sigma0 * sigma0);
  double v[1] = {0.0};
  for (int j = threadIdx.x; j < n; j += kThreads) {
    const double x = (qmin + dq * j) - q0;
    const double amp = exp(-w * x * x);
    double sn, cs;
    sincos(p0 * x, &sn, &cs);
    const double2 val = make_double2(amp * cs, amp * sn);
    psi[(size_t)surface * n + j] = val;
    v[0] = fma(amp, amp, v[0]);
  }
  cta_sum<1>(v, red, sc);
  const double scale = 1.0 / sqrt(dq * sc[0]);
  for (int s = 0; s < S; ++s) {
    for (int j = threadIdx.x; j < n; j += kThreads) {
      const size_t i = (size_t)s * n + j;
      psi[i] = (s == surface) ? cscale(scale, psi[i]) : make_double2(0.0, 0.0);
    }
  }
}

// Two-state adiabatic fields (Sec. II E).  V ascending; the stored coupling
// F[0] = F_{ground,excited} = -F_12 of Eq. (nonadiab_c).  The paper's
// expression (W12' Delta - W12 Delta') / (W12^2 + Delta^2) is evaluated in the
// algebraically identical form (dW W12' - W12 dW') / (dW^2 + 4 W12^2),
// dW = W22 - W11, which has no cancellation where W12 is small.
__global__ void fields2_kernel(const double* __restrict__ W, const double* __restrict__ dW, int n, double* V,
                               double* F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double w11 = W[j], w12 = W[n + j], w22 = W[2 * n + j];
  const double d11 = dW[j], d12 = dW[n + j], d22 = dW[2 * n + j];
  const double dw = w22 - w11;
  const double wbar = 0.5 * (w11 + w22);
  const double r = hypot(0.5 * dw, w12);
  V[j] = wbar - r;
  V[n + j] = wbar + r;
  const double ddw = d22 - d11;
  const double f12 = (dw * d12 - w12 * ddw) / fma(dw, dw, 4.0 * w12 * w12);
  F[j] = -f12;
}

}  // namespace qg

// ---------------------------------------------------------------------------
// Host-side launch wrappers.

static int nb_capacity(int max_n, int max_S, int restart, size_t* bytes_out) {
  // one or all surfaces' FFT buffers, whichever fits next to the GMRES arrays
  const size_t budget = 200 * 1024;
  const size_t rest = (size_t)(restart + 1) * restart * 16 + (size_t)(restart + 1) * 16 + (size_t)restart * 40 + 256;
  int nb = max_S;
  if ((size_t)max_S * max_n * 16 + rest > budget) nb = 1;
  if (bytes_out) *bytes_out = (size_t)nb * max_n * 16 + rest + 64;
  return nb;
}

size_t qg_smem_bytes(int max_n, int max_S, int restart) {
  size_t b;
  nb_capacity(max_n, max_S, restart, &b);
  return b;
}

cudaError_t qg_launch_propagate(const InstDesc* d_insts, int ninst, const StepPlan& plan, int* d_counter,
                                qg_step_stats* d_stats, int max_n, int max_S, cudaStream_t st) {
  size_t smem;
  const int nb = nb_capacity(max_n, max_S, plan.restart, &smem);
  cudaError_t e = cudaFuncSetAttribute(qg::propagate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ninst < sms ? ninst : sms;
  e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  qg::propagate_kernel<<<grid, QG_THREADS, smem, st>>>(d_insts, ninst, plan, d_counter, d_stats, max_n, nb);
  return cudaGetLastError();
}

cudaError_t qg_launch_apply_h(const InstDesc* d_inst, double2* d_out, int n, int S, cudaStream_t st) {
  size_t smem;
  const int nb = nb_capacity(n, S, 1, &smem);
  cudaError_t e = cudaFuncSetAttribute(qg::apply_h_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qg::apply_h_kernel<<<1, QG_THREADS, smem, st>>>(d_inst, d_out, nb);
  return cudaGetLastError();
}

cudaError_t qg_launch_energy(const InstDesc* d_inst, double* d_out, int n, int S, cudaStream_t st) {
  size_t smem;
  const int nb = nb_capacity(n, S, 1, &smem);
  cudaError_t e = cudaFuncSetAttribute(qg::energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qg::energy_kernel<<<1, QG_THREADS, smem, st>>>(d_inst, d_out, nb);
  return cudaGetLastError();
}

cudaError_t qg_launch_populations(const double2* d_psi, int n, int S, double dq, double* d_out, cudaStream_t st) {
  qg::populations_kernel<<<1, QG_THREADS, 0, st>>>(d_psi, n, S, dq, d_out);
  return cudaGetLastError();
}

cudaError_t qg_launch_overlap(const double2* d_a, const double2* d_b, int len, double dq, double* d_out,
                              cudaStream_t st) {
  qg::overlap_kernel<<<1, QG_THREADS, 0, st>>>(d_a, d_b, len, dq, d_out);
  return cudaGetLastError();
}

cudaError_t qg_launch_gaussian(double2* d_psi, int n, int S, int surface, double qmin, double dq, double q0,
                               double p0, double sigma0, cudaStream_t st) {
  qg::gaussian_kernel<<<1, QG_THREADS, 0, st>>>(d_psi, n, S, surface, qmin, dq, q0, p0, sigma0);
  return cudaGetLastError();
}

cudaError_t qg_launch_fields2(const double* d_W, const double* d_dW, int n, double* d_V, double* d_F,
                              cudaStream_t st) {
  qg::fields2_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_W, d_dW, n, d_V, d_F);
  return cudaGetLastError();
}

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
// process exits.  All calls share it: calls that overlap on the GPU race.

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

// Twiddles exp(-2 pi i k / n) and the wave numbers of the digit-reversed
// positions (divided by n), for the radix plan in `plan`.
__global__ void noalloc_tables_kernel(unsigned char* base, FftPlan plan, double dq) {
  const int n = plan.n;
  double2* tw = reinterpret_cast<double2*>(base + kNaWorkBytes);
  double* kd = reinterpret_cast<double*>(base + kNaWorkBytes + kNaTwBytes);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
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
  I.V = in.V;
  I.F = in.F;
  I.psi = in.psi;
  I.work = reinterpret_cast<double2*>(base);
  I.restart_cap = QG_NA_MAX_RESTART;
  qg_step_stats* st = reinterpret_cast<qg_step_stats*>(base + kNaWorkBytes + kNaTwBytes + kNaKdBytes);
  const Smem sm = carve_smem(dyn, in.n, nb_cap, P.restart);
  run_instance(I, P, sm, st, red, sc);
}

}  // namespace qg

// Per-device set-up state of the no-allocation entry point (host side).
namespace {
constexpr int kNaMaxDevices = 64;
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
  if (g_na_tab_n[dev] != n || g_na_tab_dq[dev] != dq) {
    qg::noalloc_tables_kernel<<<(n + 255) / 256, 256, 0, st>>>(base, plan, dq);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    g_na_tab_n[dev] = n;
    g_na_tab_dq[dev] = dq;
  }
  size_t smem;
  const int nb = nb_capacity(n, S, P.restart, &smem);
  e = cudaFuncSetAttribute(qg::propagate_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
  return cudaStreamSynchronize(st);
}
