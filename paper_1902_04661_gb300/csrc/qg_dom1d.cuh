// The one-CTA-per-instance domain of the 1-D propagator and the device
// routines built on it (composed steps, adjoint), shared by the translation
// units that instantiate the persistent kernels.  Also the host-side sizing of
// their dynamic shared memory.
#pragma once
#include <cuda_runtime.h>

#include "qg_solver.cuh"

namespace qg {
// Dynamic shared memory of the 1-D kernels: the FFT buffer (nb_cap vectors of
// max_n complex doubles, also used by the FP32 passes), then the GMRES arrays
// sized for doubles (the FP32 arrays fit in the same space).
// Optional staging regions follow (flags of the launch, see stage_plan):
// kStageTables -- the instance's FP64 transform tables (the Linzer-Feig
// factors, lf_table_bytes(max_n), and max_n wave numbers), so the FFT passes
// read them from shared memory;
// kStageU -- the intermediate U = (D + F) x of H psi (max_S x max_n double2),
// so H psi makes fewer passes over global memory.
enum { kStageTables = 1, kStageU = 2 };

struct Smem {
  unsigned char* fft;
  unsigned char* gm;
  unsigned char* lf;   // staged factor tables (entries, then form words) or null
  double* kd;    // staged wave numbers or null
  double2* su;   // staged U or null
  int nb_cap;
  int m;
};

__host__ __device__ inline size_t gm_region_bytes(int m) { return (gmres_smem_bytes(m) + 255) & ~size_t(255); }

// The kStageTables region: factor tables, then wave numbers.
__host__ __device__ inline size_t lf_region_bytes(int max_n) { return (lf_table_bytes(max_n) + 255) & ~size_t(255); }
__host__ __device__ inline size_t table_region_bytes(int max_n) {
  return lf_region_bytes(max_n) + (((size_t)max_n * sizeof(double) + 255) & ~size_t(255));
}

static __device__ Smem carve_smem(void* base, int max_n, int nb_cap, int m, int stage = 0, int max_S = 0) {
  Smem s;
  unsigned char* p = reinterpret_cast<unsigned char*>(base);
  s.fft = p;
  p += (padded_bytes((size_t)nb_cap * max_n, sizeof(double2)) + 255) & ~size_t(255);
  s.gm = p;
  p += gm_region_bytes(m);
  s.lf = nullptr;
  s.kd = nullptr;
  s.su = nullptr;
  if (stage & kStageTables) {
    s.lf = p;
    s.kd = reinterpret_cast<double*>(p + lf_region_bytes(max_n));
    p += table_region_bytes(max_n);
  }
  if (stage & kStageU) s.su = reinterpret_cast<double2*>(p);
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
  H.n8 = count_radix8(I.radix, I.npass);
  H.h2m = I.h2m;
  H.tw = I.tw;
  H.kd = I.kd;
  H.lf = I.lf;
  H.lff = I.lff;
  H.V = I.V;
  H.F = I.F;
  H.U = U;
  H.diab = I.rep;
  return H;
}

__device__ __forceinline__ HOp<float> hop32(const InstDesc& I, float2* U) {
  HOp<float> H;
  H.n = I.n;
  H.S = I.S;
  H.npass = I.npass;
  H.n8 = count_radix8(I.radix, I.npass);
  H.h2m = (float)I.h2m;
  H.tw = I.tw32;
  H.kd = I.kd32;
  H.V = I.V32;
  H.F = I.F32;
  H.U = U;
  H.diab = I.rep;
  return H;
}

// One CTA owns one whole 1-D instance.
struct Dom1D {
  // with U staged in shared memory, H psi forms Re<x, y> and ||y||^2 in its
  // last pass (hpsi with dots); without it the solvers reduce them separately
  static constexpr bool kFusedDots = true;
  // the FP64 Lanczos solve keeps its vectors in the workspace basis (lanczos_stored_solve)
  static constexpr bool kStoredLanczos = true;
  // the same for the complex64 inner solves of the mixed form (measured slower here: 82.3 against 79.9 ms per step of the mixed NaI-like batch)
  static constexpr bool kStoredLanczos32 = false;
  int len;
  double2* su;    // staged U (shared memory) or null
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

  // The loop bound is copied to a register: the stores f makes through
  // generic pointers could otherwise alias *this and force a reload of len
  // from local memory every iteration.
  template <class F>
  __device__ __forceinline__ void each(F&& f) {
    const int n = len;
    for (int i = threadIdx.x; i < n; i += kThreads) f(i);
  }
  // each with U elements per thread in flight: ld(i) returns element i's
  // operands, st(i, t) computes and stores.  The loads of a group of U
  // elements precede its stores, so each thread keeps U sets of loads in
  // flight instead of one (8 warps per SM cannot hide the L2 latency with
  // one).  ld(i) and st(i, t) must touch element i only.
  template <int U, class Ld, class St>
  __device__ __forceinline__ void each_u(Ld&& ld, St&& st) {
    const int n = len;
    using T = decltype(ld(0));
    int i = threadIdx.x;
    for (; i + (U - 1) * kThreads < n; i += U * kThreads) {
      T t[U];
#pragma unroll
      for (int u = 0; u < U; ++u) t[u] = ld(i + u * kThreads);
#pragma unroll
      for (int u = 0; u < U; ++u) st(i + u * kThreads, t[u]);
    }
    for (; i < n; i += kThreads) st(i, ld(i));
  }
  template <int K, typename R>
  __device__ __forceinline__ bool sum(R (&v)[K], R* out) {
    cta_sum<K>(v, reinterpret_cast<R*>(red), out);
    return true;
  }
  template <typename R>
  __device__ __forceinline__ void hpsi(const typename Cx<R>::T* x, typename Cx<R>::T* y,
                                       const typename Cx<R>::T* z, R e, R a, typename Cx<R>::T c) {
    if constexpr (sizeof(R) == 8) {
      if (su)
        apply_h_staged<double, false>(H64, reinterpret_cast<double2*>(fb), nb_cap, su, x, y, z, e, a, c, nullptr,
                                      nullptr);
      else
        apply_h_axpby<double>(H64, reinterpret_cast<double2*>(fb), nb_cap, x, y, z, e, a, c);
    } else {
      if (su)
        apply_h_staged<float, false>(H32, reinterpret_cast<float2*>(fb), 2 * nb_cap, reinterpret_cast<float2*>(su),
                                     x, y, z, e, a, c, nullptr, nullptr);
      else
        apply_h_axpby<float>(H32, reinterpret_cast<float2*>(fb), 2 * nb_cap, x, y, z, e, a, c);
    }
  }
  // the same, also returning the raw sums Re<x, y> (W bit 0) and ||y||^2
  // (W bit 1) in dots[0..1]
  template <typename R, int W = 3>
  __device__ __forceinline__ void hpsi(const typename Cx<R>::T* x, typename Cx<R>::T* y,
                                       const typename Cx<R>::T* z, R e, R a, typename Cx<R>::T c, R* dots) {
    using C = typename Cx<R>::T;
    R* rd = reinterpret_cast<R*>(red);
    if (su) {
      if constexpr (sizeof(R) == 8)
        apply_h_staged<double, W>(H64, reinterpret_cast<double2*>(fb), nb_cap, su, x, y, z, e, a, c, rd, dots);
      else
        apply_h_staged<float, W>(H32, reinterpret_cast<float2*>(fb), 2 * nb_cap, reinterpret_cast<float2*>(su), x,
                                 y, z, e, a, c, rd, dots);
      return;
    }
    hpsi<R>(x, y, z, e, a, c);
    R v[2] = {(R)0, (R)0};
    each([&](int i) {
      const C xs = x[i], out = y[i];
      v[0] = fma(xs.x, out.x, fma(xs.y, out.y, v[0]));
      v[1] = fma(out.x, out.x, fma(out.y, out.y, v[1]));
    });
    cta_sum<2>(v, rd, dots);
  }
  __device__ __forceinline__ bool ok() const { return true; }
};

// The instance's H psi operands; with kStageTables the FP64 factor tables
// and wave numbers are first copied into shared memory.
static __device__ Dom1D make_dom1d(const InstDesc& I, const Smem& sm, int m, double* red) {
  const int len = I.S * I.n;
  Dom1D D;
  D.len = len;
  D.dv = I.dq;
  D.gm = sm.gm;
  D.red = red;
  D.H64 = hop64(I, I.work);
  if (sm.kd) {
    for (int k = threadIdx.x; k < I.n; k += kThreads) sm.kd[k] = I.kd[k];
    D.H64.kd = sm.kd;
    if (I.lf) {
      // entries and form words are one block of whole 16-byte words
      const int words = (int)(lf_table_bytes(I.n) / 16);
      const int4* src = reinterpret_cast<const int4*>(I.lf);
      int4* dst = reinterpret_cast<int4*>(sm.lf);
      for (int k = threadIdx.x; k < words; k += kThreads) dst[k] = src[k];
      D.H64.lf = reinterpret_cast<const double2*>(sm.lf);
      D.H64.lff = reinterpret_cast<const unsigned*>(sm.lf + (reinterpret_cast<const unsigned char*>(I.lff) -
                                                             reinterpret_cast<const unsigned char*>(I.lf)));
    }
    __syncthreads();
  }
  D.su = sm.su;
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
static __device__ void run_instance(const InstDesc& I, const StepPlan& P, const Smem& sm, qg_step_stats* st, double* red,
                             double* sc) {
  const int len = I.S * I.n;
  Dom1D D = make_dom1d(I, sm, P.restart, red);
  Counters cnt{0, 0, 0, 0, 0, 0, 0, 0, 0.0};
  long long nsub = 0;
  const long long failed =
      run_steps<2>(D, P, I.psi, I.work + (size_t)1 * len, I.work + (size_t)2 * len, I.work + (size_t)3 * len,
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
static __device__ void run_adjoint(const InstDesc& I, const StepPlan& P, const Smem& sm, qg_step_stats* st, double* red,
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
      // psi_prev = U(-tau) psi
      bool ok = implicit_solve<0>(D, P, -tau, psi, X, false, cnt, sc);
      // mu = (1 - i tau H)^{-1} g
      if (ok) ok = implicit_solve<0>(D, P, -tau, g, M, false, cnt, sc);
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


}  // namespace qg

// One or all surfaces' FFT buffers, whichever fits next to the GMRES arrays
// within `budget` bytes of dynamic shared memory; force_nb > 0 caps the count.
static inline int nb_capacity(int max_n, int max_S, int restart, size_t* bytes_out, size_t budget = 200 * 1024,
                              int force_nb = 0) {
  const size_t rest = qg::gm_region_bytes(restart);
  int nb = max_S;
  if (((qg::padded_bytes((size_t)max_S * max_n, 16) + 255) & ~size_t(255)) + rest > budget) nb = 1;
  if (force_nb > 0 && force_nb < nb) nb = force_nb;
  if (bytes_out) *bytes_out = ((qg::padded_bytes((size_t)nb * max_n, 16) + 255) & ~size_t(255)) + rest + 64;
  return nb;
}

// Staging regions (qg::kStageTables, qg::kStageU) that fit after the FFT
// buffers and GMRES arrays (*bytes, updated) within the budget: tables
// first, then U.
static inline int stage_plan(int max_n, int max_S, size_t budget, size_t* bytes) {
  int stage = 0;
  const size_t tab = qg::table_region_bytes(max_n);
  if (*bytes + tab <= budget) {
    stage |= qg::kStageTables;
    *bytes += tab;
  }
  const size_t u = (size_t)max_S * max_n * 16;
  if (*bytes + u <= budget) {
    stage |= qg::kStageU;
    *bytes += u;
  }
  return stage;
}
