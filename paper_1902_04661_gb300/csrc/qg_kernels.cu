// Kernels of libqgeom: the persistent propagator (composed trapezoidal /
// implicit-midpoint steps with GMRES implicit solves, in FP64 or with
// complex64 inner solves refined in FP64), the Hamiltonian action,
// observables, the Gaussian initial state and the two-state diabatic ->
// adiabatic field builder.
#include <cuda_runtime.h>

#include "qg_solver.cuh"

namespace qg {

// Dynamic shared memory of the 1-D kernels: the FFT buffer (nb_cap vectors of
// max_n complex doubles, also used by the FP32 passes), then the GMRES arrays
// sized for doubles (the FP32 arrays fit in the same space).
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
  s.gm = p + padded_bytes((size_t)nb_cap * max_n, sizeof(double2));
  s.nb_cap = nb_cap;
  s.m = m;
  return s;
}

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

// One CTA owns one whole 1-D instance.
struct Dom1D {
  int len;
  double dv;
  unsigned char* gm;
  double* red;
  HOp<double> H64;
  HOp<float> H32;
  unsigned char* fb;
  int nb_cap;
  double2* basis64;
  double2* res64;
  float2* r32;
  float2* d32;
  float2* basis32;

  template <class F>
  __device__ __forceinline__ void each(F&& f) {
    for (int i = threadIdx.x; i < len; i += kThreads) f(i);
  }
  template <int K, typename R>
  __device__ __forceinline__ bool sum(R (&v)[K], R* out) {
    cta_sum<K>(v, reinterpret_cast<R*>(red), out);
    return true;
  }
  template <typename R>
  __device__ __forceinline__ void hpsi(const typename Cx<R>::T* x, typename Cx<R>::T* y,
                                       const typename Cx<R>::T* z, R e, R a, typename Cx<R>::T c) {
    if constexpr (sizeof(R) == 8)
      apply_h_axpby<double>(H64, reinterpret_cast<double2*>(fb), nb_cap, x, y, z, e, a, c);
    else
      apply_h_axpby<float>(H32, reinterpret_cast<float2*>(fb), 2 * nb_cap, x, y, z, e, a, c);
  }
  __device__ __forceinline__ bool ok() const { return true; }
};

__device__ Dom1D make_dom1d(const InstDesc& I, const Smem& sm, int m, double* red) {
  const int len = I.S * I.n;
  Dom1D D;
  D.len = len;
  D.dv = I.dq;
  D.gm = sm.gm;
  D.red = red;
  D.H64 = hop64(I, I.work);
  D.fb = sm.fft;
  D.nb_cap = sm.nb_cap;
  D.basis64 = I.work + (size_t)4 * len;
  D.res64 = I.work + (size_t)4 * len;     // mixed form: the FP64 basis is unused
  if (I.work32) {
    D.H32 = hop32(I, I.work32);
    D.r32 = I.work32 + (size_t)1 * len;
    D.d32 = I.work32 + (size_t)2 * len;
    D.basis32 = I.work32 + (size_t)3 * len;
  } else {
    D.r32 = D.d32 = D.basis32 = nullptr;
  }
  return D;
}

// All nsteps composed steps of one instance.
__device__ void run_instance(const InstDesc& I, const StepPlan& P, const Smem& sm, qg_step_stats* st, double* red,
                             double* sc) {
  const int len = I.S * I.n;
  Dom1D D = make_dom1d(I, sm, P.restart, red);
  Counters cnt{0, 0, 0, 0, 0, 0, 0, 0, 0.0};
  long long nsub = 0;
  const long long failed =
      run_steps(D, P, I.psi, I.work + (size_t)1 * len, I.work + (size_t)2 * len, I.work + (size_t)3 * len,
                I.precision == QG_C64_MIXED, I.ckpt, I.nckpt, I.every, cnt, nsub, sc);
  write_stats(st, cnt, nsub, failed);
}

// Adjoint of nsteps composed steps (reverse-mode differentiation without
// storing the trajectory).  Every elementary step is the Cayley map
// U = (1 + i tau H)^{-1} (1 - i tau H), unitary and exactly reversible, so
// going backward from psi(t_f):
//   psi_prev = U(-tau) psi   (implicit midpoint with -tau: chi solves
//              (1 - i tau H) chi = psi, psi_prev = 2 chi - psi),
//   g_prev   = U^dagger g = U(-tau) g, whose implicit intermediate
//              mu = (1 - i tau H)^{-1} g is exactly (A^{-1})^dagger g,
//   dL      += Re(g^H dU psi_prev) = tau Im(mu^H dH (psi + psi_prev)),
// with dU = -i tau A^{-1} dH (U + 1).  For H = -hbar^2/2m (D + F)^2 + V:
//   dL/dV_s(q_j)  += tau Im(conj(mu_s) phi_s),  phi = psi + psi_prev,
//   dL/dF_ab(q_j) += tau Im(-hbar^2/2m [-(conj(nu_a) phi_b - conj(nu_b) phi_a)
//                                       + (conj(mu_a) u_b - conj(mu_b) u_a)]),
//   u = (D + F) phi, nu = (D + F) mu.
// psi is reset to the stored checkpoint at every checkpointed step boundary
// to bound the reconstruction drift.  g follows the torch convention
// dL = Re(sum conj(g) dpsi).
__device__ void run_adjoint(const InstDesc& I, const StepPlan& P, const Smem& sm, qg_step_stats* st, double* red,
                            double* sc) {
  const int len = I.S * I.n;
  const int n = I.n, S = I.S;
  Dom1D D = make_dom1d(I, sm, P.restart, red);
  double2* psi = I.psi;
  double2* g = I.grad;
  double2* B = I.work + (size_t)1 * len;
  double2* X = I.work + (size_t)2 * len;
  double2* P0 = I.work + (size_t)3 * len;
  double2* M = I.work + (size_t)(5 + P.restart) * len;
  double2* PHI = I.work + (size_t)(6 + P.restart) * len;
  double2* UU = I.work + (size_t)(7 + P.restart) * len;
  double2* NU = I.work + (size_t)(8 + P.restart) * len;
  double2* fb = reinterpret_cast<double2*>(sm.fft);
  Counters cnt{0, 0, 0, 0, 0, 0, 0, 0, 0.0};
  long long nsub = 0, failed = -1;
  const double h2m = I.h2m;
  dcopy(D, P0, psi);
  for (long long step = P.nsteps - 1; step >= 0 && failed < 0; --step) {
    for (int f = P.nfrac - 1; f >= 0; --f) {
      const double tau = 0.5 * P.frac[f] * P.dt;
      const double2 pic = make_double2(0.0, tau);
      // psi_prev = U(-tau) psi
      D.hpsi<double>(psi, X, nullptr, 0.0, 1.0, pic);
      cnt.hpsi++;
      bool ok = solve_fp64(D, P, -tau, psi, X, cnt, sc);
      // mu = (1 - i tau H)^{-1} g
      if (ok) {
        D.hpsi<double>(g, M, nullptr, 0.0, 1.0, pic);
        cnt.hpsi++;
        ok = solve_fp64(D, P, -tau, g, M, cnt, sc);
      }
      if (!ok) {
        failed = step;
        break;
      }
      for (int i = threadIdx.x; i < len; i += kThreads) {
        const double2 c = X[i], p = psi[i];
        const double2 pp = make_double2(2.0 * c.x - p.x, 2.0 * c.y - p.y);
        B[i] = pp;                                   // psi_prev
        PHI[i] = make_double2(p.x + pp.x, p.y + pp.y);
      }
      __syncthreads();
      apply_d_plus_f<double>(D.H64, fb, sm.nb_cap, PHI, UU);
      apply_d_plus_f<double>(D.H64, fb, sm.nb_cap, M, NU);
      for (int j = threadIdx.x; j < n; j += kThreads) {
        for (int s = 0; s < S; ++s) {
          const double2 mu = M[s * n + j], ph = PHI[s * n + j];
          I.gV[s * n + j] += tau * (mu.x * ph.y - mu.y * ph.x);          // Im(conj(mu) phi)
        }
        int pr = 0;
        for (int a = 0; a < S; ++a)
          for (int b = a + 1; b < S; ++b) {
            const double2 na = NU[a * n + j], nb_ = NU[b * n + j];
            const double2 pa = PHI[a * n + j], pb = PHI[b * n + j];
            const double2 ma = M[a * n + j], mb = M[b * n + j];
            const double2 ua = UU[a * n + j], ub = UU[b * n + j];
            // Im of conj(x) y is x.re y.im - x.im y.re
            const double t1 = (na.x * pb.y - na.y * pb.x) - (nb_.x * pa.y - nb_.y * pa.x);
            const double t2 = (ma.x * ub.y - ma.y * ub.x) - (mb.x * ua.y - mb.y * ua.x);
            I.gF[(size_t)pr * n + j] += tau * (-h2m) * (t2 - t1);
            ++pr;
          }
      }
      for (int i = threadIdx.x; i < len; i += kThreads) {
        const double2 m = M[i], gg = g[i];
        g[i] = make_double2(2.0 * m.x - gg.x, 2.0 * m.y - gg.y);
        psi[i] = B[i];
      }
      __syncthreads();
      nsub++;
    }
    if (failed < 0 && I.ckpt && step % I.every == 0 && step / I.every < I.nckpt)
      dcopy(D, psi, I.ckpt + (size_t)(step / I.every) * len);
  }
  if (failed >= 0) dcopy(D, psi, P0);
  write_stats(st, cnt, nsub, failed);
}

// Persistent propagator: CTAs take instances from the work counter.  MINB is
// the number of CTAs per SM the launch is built for (1: up to 255 registers
// per thread; 2: 128, twice the warps to hide FP64 latency).
template <int MINB>
__global__ void __launch_bounds__(QG_THREADS, MINB)
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
    if (P.run == QG_RUN_ADJOINT)
      run_adjoint(I, P, sm, stats + idx, red, sc);
    else
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
__global__ void fields2_kernel(const double* __restrict__ W, const double* __restrict__ dW, int n, int D, double* V,
                               double* F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double w11 = W[j], w12 = W[n + j], w22 = W[2 * n + j];
  const double dw = w22 - w11;
  const double wbar = 0.5 * (w11 + w22);
  const double r = hypot(0.5 * dw, w12);
  V[j] = wbar - r;
  V[n + j] = wbar + r;
  for (int d = 0; d < D; ++d) {
    const double* g = dW + (size_t)d * 3 * n;
    const double d11 = g[j], d12 = g[n + j], d22 = g[2 * n + j];
    const double ddw = d22 - d11;
    const double f12 = (dw * d12 - w12 * ddw) / fma(dw, dw, 4.0 * w12 * w12);
    F[(size_t)d * n + j] = -f12;
  }
}

// Adiabatic fields for S >= 2 surfaces (Sec. II E in general form): per grid
// point the eigen-decomposition W = O diag(V) O^T by cyclic Jacobi rotations
// (eigenvalues ascending), raw couplings by the Hellmann-Feynman identity
// F_ij = <phi_i| W' |phi_j> / (V_j - V_i) (= (O^T O')_ij), and the raw
// eigenvectors for the sign-continuity pass.  W, dW: S(S+1)/2 (x D) upper
// triangles; out: V (S x n), F (S(S-1)/2 x n), vec (n x S x S, column i =
// eigenvector i).
__global__ void fieldsS_eigen_kernel(const double* __restrict__ W, const double* __restrict__ dW, int n, int S,
                                     double* V, double* F, double* vec) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double a[QG_MAX_S][QG_MAX_S], o[QG_MAX_S][QG_MAX_S], d[QG_MAX_S][QG_MAX_S];
  int t = 0;
  for (int r = 0; r < S; ++r)
    for (int c = r; c < S; ++c) {
      a[r][c] = a[c][r] = W[(size_t)t * n + j];
      d[r][c] = d[c][r] = dW[(size_t)t * n + j];
      ++t;
    }
  for (int r = 0; r < S; ++r)
    for (int c = 0; c < S; ++c) o[r][c] = (r == c) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int r = 0; r < S; ++r) {
      diag += a[r][r] * a[r][r];
      for (int c = r + 1; c < S; ++c) off += a[r][c] * a[r][c];
    }
    if (off <= 1e-34 * diag || off == 0.0) break;
    for (int p = 0; p < S - 1; ++p)
      for (int q = p + 1; q < S; ++q) {
        if (a[p][q] == 0.0) continue;
        // rotation zeroing a[p][q] (symmetric Schur decomposition)
        const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        const double tt = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(tt * tt + 1.0), sn = tt * c;
        for (int k = 0; k < S; ++k) {
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - sn * akq;
          a[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < S; ++k) {
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - sn * aqk;
          a[q][k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < S; ++k) {
          const double okp = o[k][p], okq = o[k][q];
          o[k][p] = c * okp - sn * okq;
          o[k][q] = sn * okp + c * okq;
        }
      }
  }
  // ascending order (selection sort on the diagonal)
  int idx[QG_MAX_S];
  for (int i = 0; i < S; ++i) idx[i] = i;
  for (int i = 0; i < S; ++i)
    for (int k = i + 1; k < S; ++k)
      if (a[idx[k]][idx[k]] < a[idx[i]][idx[i]]) {
        const int tmp = idx[i];
        idx[i] = idx[k];
        idx[k] = tmp;
      }
  for (int i = 0; i < S; ++i) {
    V[(size_t)i * n + j] = a[idx[i]][idx[i]];
    for (int r = 0; r < S; ++r) vec[((size_t)j * S + r) * S + i] = o[r][idx[i]];
  }
  int pr = 0;
  for (int i = 0; i < S; ++i)
    for (int k = i + 1; k < S; ++k) {
      double num = 0.0;
      for (int r = 0; r < S; ++r)
        for (int c = 0; c < S; ++c) num += o[r][idx[i]] * d[r][c] * o[c][idx[k]];
      F[(size_t)pr * n + j] = num / (a[idx[k]][idx[k]] - a[idx[i]][idx[i]]);
      ++pr;
    }
}

// Sign gauge along the grid: at the first point each eigenvector's largest
// component is made positive; afterwards each eigenvector is flipped when its
// overlap with the (already fixed) eigenvector at the previous point is
// negative.  One thread per model walks the grid (pre-processing, once per
// model); the couplings are rescaled by the product of the two signs.
__global__ void fieldsS_gauge_kernel(int n, int S, double* F, double* vec) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = 0; j < n; ++j) {
    double sg[QG_MAX_S];
    for (int i = 0; i < S; ++i) {
      double* v = vec + (size_t)j * S * S;
      double dot = 0.0;
      if (j == 0) {
        int big = 0;
        for (int r = 1; r < S; ++r)
          if (fabs(v[r * S + i]) > fabs(v[big * S + i])) big = r;
        dot = v[big * S + i];
      } else {
        const double* u = vec + (size_t)(j - 1) * S * S;
        for (int r = 0; r < S; ++r) dot += v[r * S + i] * u[r * S + i];
      }
      sg[i] = dot < 0.0 ? -1.0 : 1.0;
      if (sg[i] < 0.0)
        for (int r = 0; r < S; ++r) v[r * S + i] = -v[r * S + i];
    }
    int pr = 0;
    for (int i = 0; i < S; ++i)
      for (int k = i + 1; k < S; ++k) {
        F[(size_t)pr * n + j] *= sg[i] * sg[k];
        ++pr;
      }
  }
}

__global__ void to_f32_kernel(const double* __restrict__ in, float* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

}  // namespace qg

// ---------------------------------------------------------------------------
// Host-side launch wrappers.

static int nb_capacity(int max_n, int max_S, int restart, size_t* bytes_out, size_t budget = 200 * 1024,
                       int force_nb = 0) {
  // one or all surfaces' FFT buffers, whichever fits next to the GMRES arrays
  const size_t rest = qg::gmres_smem_bytes(restart);
  int nb = max_S;
  if (qg::padded_bytes((size_t)max_S * max_n, 16) + rest > budget) nb = 1;
  if (force_nb > 0 && force_nb < nb) nb = force_nb;
  if (bytes_out) *bytes_out = qg::padded_bytes((size_t)nb * max_n, 16) + rest + 64;
  return nb;
}

size_t qg_smem_bytes(int max_n, int max_S, int restart) {
  size_t b;
  nb_capacity(max_n, max_S, restart, &b);
  return b;
}

cudaError_t qg_launch_propagate_tuned(const InstDesc* d_insts, int ninst, const StepPlan& plan, int* d_counter,
                                      qg_step_stats* d_stats, int max_n, int max_S, int ctas_per_sm, int nb_pref,
                                      cudaStream_t st) {
  size_t smem;
  const size_t budget = ctas_per_sm >= 2 ? 110 * 1024 : 200 * 1024;
  const int nb = nb_capacity(max_n, max_S, plan.restart, &smem, budget, nb_pref);
  if (smem > budget + 1024) return cudaErrorInvalidConfiguration;
  const void* fn = ctas_per_sm >= 2 ? (const void*)qg::propagate_kernel<2> : (const void*)qg::propagate_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (ninst == 0) return cudaSuccess;   // attributes only
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slots = sms * (ctas_per_sm >= 2 ? 2 : 1);
  const int grid = ninst < slots ? ninst : slots;
  e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (ctas_per_sm >= 2)
    qg::propagate_kernel<2><<<grid, QG_THREADS, smem, st>>>(d_insts, ninst, plan, d_counter, d_stats, max_n, nb);
  else
    qg::propagate_kernel<1><<<grid, QG_THREADS, smem, st>>>(d_insts, ninst, plan, d_counter, d_stats, max_n, nb);
  return cudaGetLastError();
}

cudaError_t qg_launch_propagate(const InstDesc* d_insts, int ninst, const StepPlan& plan, int* d_counter,
                                qg_step_stats* d_stats, int max_n, int max_S, cudaStream_t st) {
  return qg_launch_propagate_tuned(d_insts, ninst, plan, d_counter, d_stats, max_n, max_S, 1, 0, st);
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

cudaError_t qg_launch_fieldsS(const double* d_W, const double* d_dW, int n, int S, double* d_V, double* d_F,
                              double* d_vec, cudaStream_t st) {
  qg::fieldsS_eigen_kernel<<<(n + 127) / 128, 128, 0, st>>>(d_W, d_dW, n, S, d_V, d_F, d_vec);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  qg::fieldsS_gauge_kernel<<<1, 32, 0, st>>>(n, S, d_F, d_vec);
  return cudaGetLastError();
}

cudaError_t qg_launch_fields2(const double* d_W, const double* d_dW, int n, int D, double* d_V, double* d_F,
                              cudaStream_t st) {
  qg::fields2_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_W, d_dW, n, D, d_V, d_F);
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
  I.ckpt = nullptr;
  I.nckpt = 0;
  I.every = 1;
  I.grad = nullptr;
  I.gV = nullptr;
  I.gF = nullptr;
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
