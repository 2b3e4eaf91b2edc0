// Kernels of libqgeom: the persistent propagator (composed trapezoidal /
// implicit-midpoint steps with GMRES implicit solves, in FP64 or with
// complex64 inner solves refined in FP64), the Hamiltonian action,
// observables, the Gaussian initial state and the two-state diabatic ->
// adiabatic field builder.
#include <cuda_runtime.h>

#include "qg_device.cuh"

namespace qg {

__device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Small GMRES arrays of one precision in shared memory.
template <typename R>
struct GSmem {
  using C = typename Cx<R>::T;
  C* hess;   // (m + 1) * m, column j at hess + j * (m + 1)
  C* g;      // m + 1
  C* gs;     // m   Givens s
  R* gc;     // m   Givens c
  C* y;      // m
};

// Dynamic shared memory: the FFT buffer (nb_cap vectors of max_n complex
// doubles, also used by the FP32 passes), then the GMRES arrays sized for
// doubles (the FP32 arrays fit in the same space).
struct Smem {
  unsigned char* fft;
  unsigned char* gm;
  int nb_cap;
  int m;
};

__device__ Smem carve_smem(void* base, int max_n, int nb_cap, int m) {
  Smem s;
  unsigned char* p = reinterpret_cast<unsigned char*>(base);
  s.fft = p;
  s.gm = p + align16(sizeof(double2) * (size_t)nb_cap * max_n);
  s.nb_cap = nb_cap;
  s.m = m;
  return s;
}

template <typename R>
__device__ GSmem<R> gsmem(const Smem& s) {
  using C = typename Cx<R>::T;
  GSmem<R> g;
  const int m = s.m;
  unsigned char* p = s.gm;
  g.hess = reinterpret_cast<C*>(p);
  p += align16(sizeof(double2) * (size_t)(m + 1) * m);
  g.g = reinterpret_cast<C*>(p);
  p += align16(sizeof(double2) * (size_t)(m + 1));
  g.gs = reinterpret_cast<C*>(p);
  p += align16(sizeof(double2) * (size_t)m);
  g.y = reinterpret_cast<C*>(p);
  p += align16(sizeof(double2) * (size_t)m);
  g.gc = reinterpret_cast<R*>(p);
  return g;
}

struct Counters {
  long long hpsi;
  long long hpsi32;
  long long krylov;
  long long ortho;
  long long update;
  long long restart;
  long long outer;
  int max_krylov;
  double max_res;
};

// H psi operands of an instance in one precision; scratch vector U given.
__device__ __forceinline__ HOp<double> hop64(const InstDesc& I, double2* U) {
  HOp<double> H;
  H.n = I.n;
  H.S = I.S;
  H.npass = I.npass;
  for (int i = 0; i < QG_MAX_PASSES; ++i) H.radix[i] = I.radix[i];
  H.h2m = I.h2m;
  H.tw = I.tw;
  H.kd = I.kd;
  H.V = I.V;
  H.F = I.F;
  H.U = U;
  return H;
}

__device__ __forceinline__ HOp<float> hop32(const InstDesc& I, float2* U) {
  HOp<float> H;
  H.n = I.n;
  H.S = I.S;
  H.npass = I.npass;
  for (int i = 0; i < QG_MAX_PASSES; ++i) H.radix[i] = I.radix[i];
  H.h2m = (float)I.h2m;
  H.tw = I.tw32;
  H.kd = I.kd32;
  H.V = I.V32;
  H.F = I.F32;
  H.U = U;
  return H;
}

struct SolveParams {
  double tol;
  int m;
  int max_iters;
  int reorth;
  int true_res;
};

// Solve (1 + i tau H) x = b by restarted GMRES (Sec. II B) in the grid inner
// product, in precision R.  X holds the initial guess on entry and the
// solution on exit; basis holds m + 1 vectors.  Returns true on convergence
// (estimated relative residual <= tol).  *res_out receives the final
// relative residual estimate.
template <typename R>
__device__ bool gmres_solve(const HOp<R>& H, const Smem& smem, const SolveParams& P, R dv, R tau,
                            const typename Cx<R>::T* b, typename Cx<R>::T* X, typename Cx<R>::T* basis,
                            Counters& cnt, R* red, R* sc, double* res_out) {
  using C = typename Cx<R>::T;
  const GSmem<R> sm = gsmem<R>(smem);
  C* fbuf = reinterpret_cast<C*>(smem.fft);
  const int nbc = sizeof(R) == 8 ? smem.nb_cap : 2 * smem.nb_cap;
  const int len = H.S * H.n;
  const int m = P.m;
  const C ic = cmk<C>((R)0, tau);     // A = 1 + i tau H
  const C mic = cmk<C>((R)0, -tau);
  const R bn = sqrt(dv * cta_norm2(b, len, red, sc));
  const R target = (R)P.tol * bn;
  int total = 0;
  // r0 = b - A X
  apply_h_axpby<R>(H, fbuf, nbc, X, basis, b, (R)1, (R)-1, mic);
  if (sizeof(R) == 8) cnt.hpsi++; else cnt.hpsi32++;
  for (int guard = 0; guard < P.max_iters + 2; ++guard) {
    C* V0 = basis;
    const R beta = sqrt(dv * cta_norm2(V0, len, red, sc));
    if (beta <= target || bn == (R)0) {
      *res_out = (bn > (R)0) ? (double)(beta / bn) : 0.0;
      if (total > cnt.max_krylov) cnt.max_krylov = total;
      return true;
    }
    if (total >= P.max_iters) break;
    const R ib = (R)1 / beta;
    for (int i = threadIdx.x; i < len; i += kThreads) V0[i] = cscale(ib, V0[i]);
    if (threadIdx.x == 0) {
      sm.g[0] = cmk<C>(beta, (R)0);
      for (int i = 1; i <= m; ++i) sm.g[i] = cmk<C>((R)0, (R)0);
    }
    __syncthreads();
    int ncol = 0;
    bool conv = false;
    R res_est = beta;
    for (int j = 0; j < m; ++j) {
      C* Vj = basis + (size_t)j * len;
      C* W = basis + (size_t)(j + 1) * len;
      apply_h_axpby<R>(H, fbuf, nbc, Vj, W, nullptr, (R)0, (R)1, ic);
      if (sizeof(R) == 8) cnt.hpsi++; else cnt.hpsi32++;
      C* hcol = sm.hess + (size_t)j * (m + 1);
      if (threadIdx.x <= j + 1) hcol[threadIdx.x] = cmk<C>((R)0, (R)0);
      __syncthreads();
      // Classical Gram-Schmidt, optionally repeated once (CGS2).
      for (int pass = 0; pass < (P.reorth ? 2 : 1); ++pass) {
        for (int c0 = 0; c0 <= j; c0 += 8) {
          const int nc = min(8, j + 1 - c0);
          R v[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = (R)0;
          for (int i = threadIdx.x; i < len; i += kThreads) {
            const C w = W[i];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              if (k < nc) {
                const C q = basis[(size_t)(c0 + k) * len + i];
                v[2 * k] = fma(q.x, w.x, fma(q.y, w.y, v[2 * k]));
                v[2 * k + 1] = fma(q.x, w.y, fma(-q.y, w.x, v[2 * k + 1]));
              }
            }
          }
          cta_sum<16>(v, red, sc);
          if (threadIdx.x < nc) {
            const C h = cmk<C>(dv * sc[2 * threadIdx.x], dv * sc[2 * threadIdx.x + 1]);
            hcol[c0 + threadIdx.x] = cadd(hcol[c0 + threadIdx.x], h);
            sc[32 + 2 * threadIdx.x] = h.x;
            sc[33 + 2 * threadIdx.x] = h.y;
          }
          __syncthreads();
          C hk[8];
#pragma unroll
          for (int k = 0; k < 8; ++k)
            hk[k] = (k < nc) ? cmk<C>(sc[32 + 2 * k], sc[33 + 2 * k]) : cmk<C>((R)0, (R)0);
          __syncthreads();
          for (int i = threadIdx.x; i < len; i += kThreads) {
            C w = W[i];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (k < nc) w = cnaxpy(hk[k], basis[(size_t)(c0 + k) * len + i], w);
            W[i] = w;
          }
          __syncthreads();
        }
      }
      const R hn = sqrt(dv * cta_norm2(W, len, red, sc));
      const R tiny = sizeof(R) == 8 ? (R)1e-300 : (R)1e-35;
      if (hn > tiny) {
        const R ih = (R)1 / hn;
        for (int i = threadIdx.x; i < len; i += kThreads) W[i] = cscale(ih, W[i]);
      }
      if (threadIdx.x == 0) {
        hcol[j + 1] = cmk<C>(hn, (R)0);
        // previous rotations
        for (int i = 0; i < j; ++i) {
          const R c = sm.gc[i];
          const C s = sm.gs[i];
          const C h0 = hcol[i], h1 = hcol[i + 1];
          const C t = caxpy(s, h1, cscale(c, h0));                    // c h0 + s h1
          const C u = cnaxpy(cmk<C>(s.x, -s.y), h0, cscale(c, h1));   // -conj(s) h0 + c h1
          hcol[i] = t;
          hcol[i + 1] = u;
        }
        // new rotation zeroing hcol[j+1]
        const C a = hcol[j];
        const R bb = hcol[j + 1].x;
        const R aa = hypot(a.x, a.y);
        R c;
        C s, r;
        if (bb == (R)0) {
          c = (R)1;
          s = cmk<C>((R)0, (R)0);
          r = a;
        } else if (aa == (R)0) {
          c = (R)0;
          s = cmk<C>((R)1, (R)0);
          r = cmk<C>(bb, (R)0);
        } else {
          const R rho = hypot(aa, bb);
          const C ph = cmk<C>(a.x / aa, a.y / aa);
          c = aa / rho;
          s = cmk<C>(ph.x * bb / rho, ph.y * bb / rho);
          r = cmk<C>(ph.x * rho, ph.y * rho);
        }
        sm.gc[j] = c;
        sm.gs[j] = s;
        hcol[j] = r;
        hcol[j + 1] = cmk<C>((R)0, (R)0);
        const C gj = sm.g[j];
        sm.g[j + 1] = cmk<C>(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
        sm.g[j] = cscale(c, gj);
        sc[0] = hypot(sm.g[j + 1].x, sm.g[j + 1].y);
      }
      __syncthreads();
      res_est = sc[0];
      __syncthreads();
      ncol = j + 1;
      cnt.ortho += j + 1;
      total++;
      cnt.krylov++;
      if (res_est <= target) {
        conv = true;
        break;
      }
      if (total >= P.max_iters || hn <= tiny) break;
    }
    // y = R^{-1} g (upper triangular ncol x ncol)
    if (threadIdx.x == 0) {
      for (int i = ncol - 1; i >= 0; --i) {
        C acc = sm.g[i];
        for (int k = i + 1; k < ncol; ++k) acc = cnaxpy(sm.hess[(size_t)k * (m + 1) + i], sm.y[k], acc);
        const C d = sm.hess[(size_t)i * (m + 1) + i];
        const R dd = (R)1 / fma(d.x, d.x, d.y * d.y);
        sm.y[i] = cmk<C>((acc.x * d.x + acc.y * d.y) * dd, (acc.y * d.x - acc.x * d.y) * dd);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += kThreads) {
      C x = X[i];
      for (int k = 0; k < ncol; ++k) x = caxpy(sm.y[k], basis[(size_t)k * len + i], x);
      X[i] = x;
    }
    cnt.update += ncol;
    __syncthreads();
    if (conv && !P.true_res) {
      *res_out = (bn > (R)0) ? (double)(res_est / bn) : 0.0;
      if (total > cnt.max_krylov) cnt.max_krylov = total;
      return true;
    }
    if (total >= P.max_iters && !conv) break;
    // restart (or true-residual check): V0 = b - A X
    apply_h_axpby<R>(H, fbuf, nbc, X, basis, b, (R)1, (R)-1, mic);
    if (sizeof(R) == 8) cnt.hpsi++; else cnt.hpsi32++;
    cnt.restart++;
  }
  if (total > cnt.max_krylov) cnt.max_krylov = total;
  *res_out = 1e300;
  return false;
}

template <typename C>
__device__ __forceinline__ void vcopy(C* dst, const C* src, int len) {
  for (int i = threadIdx.x; i < len; i += kThreads) dst[i] = src[i];
  __syncthreads();
}

// FP64 implicit solve (1 + i tau H) X = b with GMRES in FP64.
__device__ bool solve_fp64(const InstDesc& I, const Smem& sm, const StepPlan& P, double tau, const double2* b,
                           double2* X, Counters& cnt, double* red, double* sc) {
  const int len = I.S * I.n;
  const HOp<double> H = hop64(I, I.work);
  SolveParams sp{P.tol, P.restart, P.max_iters, P.reorth, P.true_res};
  double res = 0.0;
  const bool ok = gmres_solve<double>(H, sm, sp, I.dq, tau, b, X, I.work + (size_t)4 * len, cnt, red, sc, &res);
  if (ok && res > cnt.max_res) cnt.max_res = res;
  if (!ok) cnt.max_res = 1e300;
  return ok;
}

// Mixed-precision implicit solve: FP64 residual r = b - (1 + i tau H) X,
// complex64 GMRES for (1 + i tau H) d = r / ||r|| to inner_tol, X += ||r|| d,
// until ||r|| <= tol ||b||.
__device__ bool solve_mixed(const InstDesc& I, const Smem& sm, const StepPlan& P, double tau, const double2* b,
                            double2* X, Counters& cnt, double* red, double* sc) {
  const int len = I.S * I.n;
  const HOp<double> H64 = hop64(I, I.work);
  double2* Rv = I.work + (size_t)4 * len;          // FP64 residual
  const HOp<float> H32 = hop32(I, I.work32);
  float2* r32 = I.work32 + (size_t)1 * len;
  float2* d32 = I.work32 + (size_t)2 * len;
  float2* basis32 = I.work32 + (size_t)3 * len;
  float* redf = reinterpret_cast<float*>(red);
  float* scf = reinterpret_cast<float*>(sc);
  const double2 mic = make_double2(0.0, -tau);
  const double dv = I.dq;
  const double bn = sqrt(dv * cta_norm2(b, len, red, sc));
  const double target = P.tol * bn;
  SolveParams sp{P.inner_tol, P.restart, P.max_iters, P.reorth, 0};
  for (int outer = 0; outer <= P.max_outer; ++outer) {
    apply_h_axpby<double>(H64, reinterpret_cast<double2*>(sm.fft), sm.nb_cap, X, Rv, b, 1.0, -1.0, mic);
    cnt.hpsi++;
    const double rho = sqrt(dv * cta_norm2(Rv, len, red, sc));
    if (rho <= target || bn == 0.0) {
      const double r = bn > 0.0 ? rho / bn : 0.0;
      if (r > cnt.max_res) cnt.max_res = r;
      return true;
    }
    if (outer == P.max_outer) break;
    cnt.outer++;
    const double ir = 1.0 / rho;
    for (int i = threadIdx.x; i < len; i += kThreads) {
      const double2 v = Rv[i];
      r32[i] = make_float2((float)(v.x * ir), (float)(v.y * ir));
      d32[i] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    double res = 0.0;
    gmres_solve<float>(H32, sm, sp, (float)dv, (float)tau, r32, d32, basis32, cnt, redf, scf, &res);
    for (int i = threadIdx.x; i < len; i += kThreads) {
      const float2 d = d32[i];
      const double2 x = X[i];
      X[i] = make_double2(fma(rho, (double)d.x, x.x), fma(rho, (double)d.y, x.y));
    }
    __syncthreads();
  }
  cnt.max_res = 1e300;
  return false;
}

// Explicit-Euler initial guess X = (1 - i tau H) src, in complex64 for the
// mixed-precision form (only the starting point of the refinement).
__device__ void guess_mixed(const InstDesc& I, const Smem& sm, double tau, const double2* src, double2* X,
                            Counters& cnt) {
  const int len = I.S * I.n;
  const HOp<float> H32 = hop32(I, I.work32);
  float2* s32 = I.work32 + (size_t)1 * len;
  float2* y32 = I.work32 + (size_t)2 * len;
  for (int i = threadIdx.x; i < len; i += kThreads) {
    const double2 v = src[i];
    s32[i] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  apply_h_axpby<float>(H32, reinterpret_cast<float2*>(sm.fft), 2 * sm.nb_cap, s32, y32, nullptr, 0.f, 1.f,
                       make_float2(0.f, (float)-tau));
  cnt.hpsi32++;
  for (int i = threadIdx.x; i < len; i += kThreads) {
    const float2 y = y32[i];
    X[i] = make_double2((double)y.x, (double)y.y);
  }
  __syncthreads();
}

// All nsteps composed steps of one instance.
__device__ void run_instance(const InstDesc& I, const StepPlan& P, const Smem& sm, qg_step_stats* st, double* red,
                             double* sc) {
  const int len = I.S * I.n;
  const bool mixed = I.precision == QG_C64_MIXED;
  double2* psi = I.psi;
  double2* B = I.work + (size_t)1 * len;
  double2* X = I.work + (size_t)2 * len;
  double2* P0 = I.work + (size_t)3 * len;
  const HOp<double> H64 = hop64(I, I.work);
  double2* fb = reinterpret_cast<double2*>(sm.fft);
  Counters cnt{0, 0, 0, 0, 0, 0, 0, 0, 0.0};
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
        apply_h_axpby<double>(H64, fb, sm.nb_cap, psi, B, nullptr, 0.0, 1.0, mic);
        cnt.hpsi += 1;
        if (mixed) {
          guess_mixed(I, sm, tau, B, X, cnt);
          ok = solve_mixed(I, sm, P, tau, B, X, cnt, red, sc);
        } else {
          apply_h_axpby<double>(H64, fb, sm.nb_cap, B, X, nullptr, 0.0, 1.0, mic);
          cnt.hpsi += 1;
          ok = solve_fp64(I, sm, P, tau, B, X, cnt, red, sc);
        }
        if (ok) vcopy(psi, X, len);
      } else {
        // guess chi0 = (1 - i tau H) psi ; solve (1 + i tau H) chi = psi ;
        // psi' = (1 - i tau H) chi  (or 2 chi - psi)
        if (mixed) {
          guess_mixed(I, sm, tau, psi, X, cnt);
          ok = solve_mixed(I, sm, P, tau, psi, X, cnt, red, sc);
        } else {
          apply_h_axpby<double>(H64, fb, sm.nb_cap, psi, X, nullptr, 0.0, 1.0, mic);
          cnt.hpsi += 1;
          ok = solve_fp64(I, sm, P, tau, psi, X, cnt, red, sc);
        }
        if (ok) {
          if (P.mid_epi) {
            apply_h_axpby<double>(H64, fb, sm.nb_cap, X, psi, nullptr, 0.0, 1.0, mic);
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
    st->n_hpsi32 = cnt.hpsi32;
    st->n_outer = cnt.outer;
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
  const HOp<double> H = hop64(I, I.work);
  apply_h_axpby<double>(H, reinterpret_cast<double2*>(dyn), nb_cap, I.psi, out, nullptr, 0.0, 0.0,
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
  const HOp<double> H = hop64(I, I.work);
  apply_h_axpby<double>(H, reinterpret_cast<double2*>(dyn), nb_cap, I.psi, Hx, nullptr, 0.0, 0.0,
                        make_double2(1.0, 0.0));
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

__global__ void to_f32_kernel(const double* __restrict__ in, float* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
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

cudaError_t qg_launch_to_f32(const double* d_in, float* d_out, size_t n, cudaStream_t st) {
  const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  qg::to_f32_kernel<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(d_in, d_out, n);
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
  I.precision = QG_C128;
  I.tw32 = nullptr;
  I.kd32 = nullptr;
  I.V32 = nullptr;
  I.F32 = nullptr;
  I.work32 = nullptr;
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
