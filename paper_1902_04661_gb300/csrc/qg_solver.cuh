// Implicit solves, composed steps and the adjoint sweep, written once over a
// "domain" that says which elements a thread owns, how a sum over the whole
// state is formed and how H psi is applied:
//   Dom1D -- one CTA owns one whole 1-D instance (qg_dom1d.cuh);
//   Dom2D -- all CTAs of a cooperative launch share one 2-D instance
//            (qg_dom2d.cuh).
// A domain D provides
//   D.len                                  elements of one state vector
//   D.each(f)                              f(i) for every owned element i
//   D.template sum<K>(v, out)              out[0..K) = sum over the state of v
//                                          (deterministic order; out in smem;
//                                          returns false if the domain failed)
//   D.template hpsi<R>(x, y, z, e, a, c)   y = e z + a x + c (H x), precision R
//   D.dv                                   volume element of the inner product
//   D.ok()                                 false after a failed grid barrier
//   Dom::kFusedDots                        true if D.template hpsi<R>(x, y, z,
//                                          e, a, c, dots) also returns
//                                          Re<x, y> and ||y||^2 (raw sums) in
//                                          dots[0..1], reduced with H psi
// plus the smem GMRES arrays D.gm, and the workspace vectors.
#pragma once

#include <cfloat>

#include "qg_device.cuh"

namespace qg {

__host__ __device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

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

template <typename R>
__device__ GSmem<R> gsmem(unsigned char* p, int m) {
  using C = typename Cx<R>::T;
  GSmem<R> g;
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

// Bytes of the GMRES arrays for restart length m (sized for doubles).
__host__ __device__ inline size_t gmres_smem_bytes(int m) {
  return (size_t)(m + 1) * m * 16 + (size_t)(m + 1) * 16 + (size_t)m * 40 + 256;
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

struct SolveParams {
  double tol;
  int m;
  int max_iters;
  int reorth;
  int true_res;
  int solver;   // QG_SOLVER_GMRES or QG_SOLVER_LANCZOS
  int x0_zero;  // the initial guess is zero: the first residual is b itself
};

template <typename R, class Dom>
__device__ bool lanczos_solve(Dom& D, const SolveParams& P, R tau, const typename Cx<R>::T* b,
                              typename Cx<R>::T* X, typename Cx<R>::T* work, Counters& cnt, R* sc,
                              double* res_out);

// Elements per thread in flight in the Lanczos vector passes.
constexpr int kLanczosUnroll = 4;

template <typename R>
__device__ __forceinline__ void count_hpsi(Counters& cnt) {
  if (sizeof(R) == 8)
    cnt.hpsi++;
  else
    cnt.hpsi32++;
}

// Solve (1 + i tau H) x = b by restarted GMRES (Sec. II B) in the grid inner
// product, in precision R.  X holds the initial guess on entry and the
// solution on exit; basis holds m + 1 vectors.  Returns true on convergence
// (estimated relative residual <= tol); *res_out receives the final relative
// residual estimate.
template <typename R, class Dom>
__device__ bool gmres_solve(Dom& D, const SolveParams& P, R tau, const typename Cx<R>::T* b,
                            typename Cx<R>::T* X, typename Cx<R>::T* basis, Counters& cnt, R* sc, double* res_out) {
  using C = typename Cx<R>::T;
  const GSmem<R> sm = gsmem<R>(D.gm, P.m);
  const int len = D.len;
  const int m = P.m;
  const R dv = (R)D.dv;
  const C ic = cmk<C>((R)0, tau);     // A = 1 + i tau H
  const C mic = cmk<C>((R)0, -tau);
  R nv[1] = {0};
  D.each([&](int i) {
    const C a = b[i];
    nv[0] = fma(a.x, a.x, fma(a.y, a.y, nv[0]));
  });
  if (!D.template sum<1>(nv, sc)) return false;
  const R bn = sqrt(dv * sc[0]);
  const R target = (R)P.tol * bn;
  int total = 0;
  // r0 = b - A X  (= b when X starts at zero)
  if (P.x0_zero) {
    D.each([&](int i) { basis[i] = b[i]; });
    __syncthreads();
  } else {
    D.template hpsi<R>(X, basis, b, (R)1, (R)-1, mic);
    count_hpsi<R>(cnt);
  }
  for (int guard = 0; guard < P.max_iters + 2; ++guard) {
    C* V0 = basis;
    R bv[1] = {0};
    D.each([&](int i) {
      const C a = V0[i];
      bv[0] = fma(a.x, a.x, fma(a.y, a.y, bv[0]));
    });
    if (!D.template sum<1>(bv, sc)) return false;
    const R beta = sqrt(dv * sc[0]);
    if (beta <= target || bn == (R)0) {
      *res_out = (bn > (R)0) ? (double)(beta / bn) : 0.0;
      if (total > cnt.max_krylov) cnt.max_krylov = total;
      return true;
    }
    if (total >= P.max_iters) break;
    const R ib = (R)1 / beta;
    D.each([&](int i) { V0[i] = cscale(ib, V0[i]); });
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
      D.template hpsi<R>(Vj, W, nullptr, (R)0, (R)1, ic);
      count_hpsi<R>(cnt);
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
          D.each([&](int i) {
            const C w = W[i];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              if (k < nc) {
                const C q = basis[(size_t)(c0 + k) * len + i];
                v[2 * k] = fma(q.x, w.x, fma(q.y, w.y, v[2 * k]));
                v[2 * k + 1] = fma(q.x, w.y, fma(-q.y, w.x, v[2 * k + 1]));
              }
            }
          });
          if (!D.template sum<16>(v, sc)) return false;
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
          D.each([&](int i) {
            C w = W[i];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (k < nc) w = cnaxpy(hk[k], basis[(size_t)(c0 + k) * len + i], w);
            W[i] = w;
          });
          __syncthreads();
        }
      }
      R wv[1] = {0};
      D.each([&](int i) {
        const C a = W[i];
        wv[0] = fma(a.x, a.x, fma(a.y, a.y, wv[0]));
      });
      if (!D.template sum<1>(wv, sc)) return false;
      const R hn = sqrt(dv * sc[0]);
      const R tiny = sizeof(R) == 8 ? (R)1e-300 : (R)1e-35;
      if (hn > tiny) {
        const R ih = (R)1 / hn;
        D.each([&](int i) { W[i] = cscale(ih, W[i]); });
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
    D.each([&](int i) {
      C x = X[i];
      for (int k = 0; k < ncol; ++k) x = caxpy(sm.y[k], basis[(size_t)k * len + i], x);
      X[i] = x;
    });
    cnt.update += ncol;
    __syncthreads();
    if (conv && !P.true_res) {
      *res_out = (bn > (R)0) ? (double)(res_est / bn) : 0.0;
      if (total > cnt.max_krylov) cnt.max_krylov = total;
      return true;
    }
    if (total >= P.max_iters && !conv) break;
    // restart (or true-residual check): V0 = b - A X
    D.template hpsi<R>(X, basis, b, (R)1, (R)-1, mic);
    count_hpsi<R>(cnt);
    cnt.restart++;
  }
  if (total > cnt.max_krylov) cnt.max_krylov = total;
  *res_out = 1e300;
  return false;
}

// Short-recurrence minimal-residual solve of (1 + i tau H) x = b (the
// "GMRES or similar" of Sec. II B).  H is Hermitian in the grid inner product,
// so the Krylov space of A = 1 + i tau H is that of H and the Arnoldi relation
// of A is A V_k = V_{k+1} ([I; 0] + i tau T_k), T_k the real tridiagonal
// Lanczos matrix of H (alpha on the diagonal, beta off it).  The least-squares
// problem of GMRES then needs only the last two Givens rotations, and the
// iterate is updated through two search directions (minimal-residual form);
// in exact arithmetic the iterates equal GMRES's.  work holds 5 vectors.
// After convergence of the recurrence estimate the true residual is
// recomputed when P.true_res is set, and the solve restarts from X if needed.
template <typename R, class Dom>
__device__ bool lanczos_solve(Dom& D, const SolveParams& P, R tau, const typename Cx<R>::T* b,
                              typename Cx<R>::T* X, typename Cx<R>::T* work, Counters& cnt, R* sc,
                              double* res_out) {
  using C = typename Cx<R>::T;
  struct C2 {
    C a, b;
  };
  struct C5 {
    C v, dp, dq, x, w;
  };
  const int len = D.len;
  const R dv = (R)D.dv;
  const C mic = cmk<C>((R)0, -tau);
  C* Vp = work;
  C* Vc = work + (size_t)len;
  C* Wn = work + (size_t)2 * len;
  C* Dp = work + (size_t)3 * len;
  C* Dq = work + (size_t)4 * len;
  R nv[1] = {0};
  D.each([&](int i) {
    const C a = b[i];
    nv[0] = fma(a.x, a.x, fma(a.y, a.y, nv[0]));
  });
  if (!D.template sum<1>(nv, sc)) return false;
  const R bn = sqrt(dv * sc[0]);
  const R target = (R)P.tol * bn;
  int total = 0;
  for (int guard = 0; guard < P.max_iters + 2; ++guard) {
    // r = b - A X  (= b on the first pass when X starts at zero)
    R beta1;
    if (guard == 0 && P.x0_zero) {
      D.each([&](int i) { Vc[i] = b[i]; });
      __syncthreads();
      beta1 = bn;
    } else if constexpr (Dom::kFusedDots) {
      D.template hpsi<R, 2>(X, Vc, b, (R)1, (R)-1, mic, sc);
      count_hpsi<R>(cnt);
      if (!D.ok()) return false;
      beta1 = sqrt(dv * sc[1]);
    } else {
      D.template hpsi<R>(X, Vc, b, (R)1, (R)-1, mic);
      count_hpsi<R>(cnt);
      R rv[1] = {0};
      D.each([&](int i) {
        const C a = Vc[i];
        rv[0] = fma(a.x, a.x, fma(a.y, a.y, rv[0]));
      });
      if (!D.template sum<1>(rv, sc)) return false;
      beta1 = sqrt(dv * sc[0]);
    }
    if (guard > 0) cnt.restart++;
    if (beta1 <= target || bn == (R)0) {
      *res_out = (bn > (R)0) ? (double)(beta1 / bn) : 0.0;
      if (total > cnt.max_krylov) cnt.max_krylov = total;
      return true;
    }
    if (total >= P.max_iters) break;
    const R ib = (R)1 / beta1;
    D.each([&](int i) {
      Vc[i] = cscale(ib, Vc[i]);
      Dp[i] = cmk<C>((R)0, (R)0);
      Dq[i] = cmk<C>((R)0, (R)0);
    });
    __syncthreads();
    C g = cmk<C>(beta1, (R)0);
    R c1 = (R)1, c2 = (R)1;
    C s1 = cmk<C>((R)0, (R)0), s2 = cmk<C>((R)0, (R)0);
    R betak = (R)0;
    R res_est = beta1;
    bool conv = false;
    for (int k = 1; total < P.max_iters; ++k) {
      // Wn = H Vc - beta_k Vp ; alpha = <Vc, Wn> ; beta_{k+1} = ||Wn - alpha Vc||
      R alpha, betan;
      if constexpr (Dom::kFusedDots) {
        // alpha is reduced inside H psi (its closing grid barrier).  beta is
        // the norm of the formed vector Wn - alpha Vc, not ||Wn||^2 - alpha^2:
        // that shortcut cancels, and the normalisation error it leaves in
        // v_{k+1} grows from one iteration to the next on stiff problems.
        if (k == 1)
          D.template hpsi<R, 1>(Vc, Wn, nullptr, (R)0, (R)0, cmk<C>((R)1, (R)0), sc);
        else
          D.template hpsi<R, 1>(Vc, Wn, Vp, -betak, (R)0, cmk<C>((R)1, (R)0), sc);
        count_hpsi<R>(cnt);
        if (!D.ok()) return false;
        alpha = dv * sc[0];
        R wv[1] = {0};
        D.template each_u<kLanczosUnroll>([&](int i) { return C2{Vc[i], Wn[i]}; },
                                          [&](int i, const C2& t) {
                                            const C w = caxpy_r(-alpha, t.a, t.b);
                                            Wn[i] = w;
                                            wv[0] = fma(w.x, w.x, fma(w.y, w.y, wv[0]));
                                          });
        if (!D.template sum<1>(wv, sc)) return false;
        betan = sqrt(dv * sc[0]);
      } else {
        if (k == 1)
          D.template hpsi<R>(Vc, Wn, nullptr, (R)0, (R)0, cmk<C>((R)1, (R)0));
        else
          D.template hpsi<R>(Vc, Wn, Vp, -betak, (R)0, cmk<C>((R)1, (R)0));
        count_hpsi<R>(cnt);
        R av[1] = {0};
        D.each([&](int i) {
          const C v = Vc[i], w = Wn[i];
          av[0] = fma(v.x, w.x, fma(v.y, w.y, av[0]));
        });
        if (!D.template sum<1>(av, sc)) return false;
        alpha = dv * sc[0];
        R wv[1] = {0};
        D.each([&](int i) {
          const C w = caxpy_r(-alpha, Vc[i], Wn[i]);
          Wn[i] = w;
          wv[0] = fma(w.x, w.x, fma(w.y, w.y, wv[0]));
        });
        if (!D.template sum<1>(wv, sc)) return false;
        betan = sqrt(dv * sc[0]);
      }
      // column k of [I; 0] + i tau T: rows k-1, k, k+1
      C eps = cmk<C>((R)0, (R)0);
      C del = cmk<C>((R)0, tau * betak);
      C gam = cmk<C>((R)1, tau * alpha);
      const C nu = cmk<C>((R)0, tau * betan);
      if (k >= 3) {
        eps = cmul(s2, del);
        del = cscale(c2, del);
      }
      if (k >= 2) {
        const C t = caxpy(s1, gam, cscale(c1, del));                  // c1 del + s1 gam
        gam = cnaxpy(cmk<C>(s1.x, -s1.y), del, cscale(c1, gam));      // -conj(s1) del + c1 gam
        del = t;
      }
      // rotation zeroing nu
      const R aa = hypot(gam.x, gam.y);
      const R nn = hypot(nu.x, nu.y);
      R c;
      C s, r;
      if (nn == (R)0) {
        c = (R)1;
        s = cmk<C>((R)0, (R)0);
        r = gam;
      } else if (aa == (R)0) {
        c = (R)0;
        s = cmk<C>(nu.x / nn, -nu.y / nn);
        r = cmk<C>(nn, (R)0);
      } else {
        const R rho = hypot(aa, nn);
        const C ph = cmk<C>(gam.x / aa, gam.y / aa);
        c = aa / rho;
        s = cscale((R)1 / rho, cmul(ph, cmk<C>(nu.x, -nu.y)));       // (gam/|gam|) conj(nu) / rho
        r = cscale(rho, ph);
      }
      const C gk = cscale(c, g);
      const C gnext = cmk<C>(-(s.x * g.x + s.y * g.y), -(s.x * g.y - s.y * g.x));   // -conj(s) g
      const R rr = (R)1 / fma(r.x, r.x, r.y * r.y);
      const C ir = cmk<C>(r.x * rr, -r.y * rr);
      const R ibn = betan > (R)0 ? (R)1 / betan : (R)0;
      D.template each_u<kLanczosUnroll>(
          [&](int i) { return C5{Vc[i], Dp[i], Dq[i], X[i], Wn[i]}; },
          [&](int i, const C5& t) {
            C d = t.v;
            d = cnaxpy(del, t.dp, d);
            d = cnaxpy(eps, t.dq, d);
            d = cmul(d, ir);
            Dq[i] = d;                               // newest direction, in the oldest slot
            X[i] = caxpy(gk, d, t.x);
            Wn[i] = cscale(ibn, t.w);                // v_{k+1}
          });
      __syncthreads();
      C* t0 = Dq;
      Dq = Dp;
      Dp = t0;
      t0 = Vp;
      Vp = Vc;
      Vc = Wn;
      Wn = t0;
      c2 = c1;
      s2 = s1;
      c1 = c;
      s1 = s;
      betak = betan;
      g = gnext;
      res_est = hypot(g.x, g.y);
      total++;
      cnt.krylov++;
      cnt.ortho += 1;
      cnt.update += 1;
      if (res_est <= target) {
        conv = true;
        break;
      }
      if (betan <= (sizeof(R) == 8 ? (R)1e-300 : (R)1e-35)) break;
    }
    if (conv && !P.true_res) {
      *res_out = (bn > (R)0) ? (double)(res_est / bn) : 0.0;
      if (total > cnt.max_krylov) cnt.max_krylov = total;
      return true;
    }
    if (total >= P.max_iters && !conv) break;
    // restore the slot order for the restart (pointers only)
    Vp = work;
    Vc = work + (size_t)len;
    Wn = work + (size_t)2 * len;
    Dp = work + (size_t)3 * len;
    Dq = work + (size_t)4 * len;
  }
  if (total > cnt.max_krylov) cnt.max_krylov = total;
  *res_out = 1e300;
  return false;
}

// The same minimal-residual iteration with the Lanczos vectors kept: V_0..V_k
// in basis (m + 1 slots, the GMRES basis of the workspace), each times a
// tracked scale (see below).  Instead of updating two search directions and X
// in every iteration, X += V_k y once per cycle, y solving R y = g with R the
// banded upper-triangular factor of [I; 0] + i tau T_k that the Givens
// rotations build (diagonal r, then del and eps one and two rows above it)
// and g the rotated right-hand side -- in exact arithmetic the iterate of
// lanczos_solve, X_0 + V_k R^{-1} g.  Each iteration then makes one vector
// pass besides H psi.  Needs a domain whose H psi forms the dots (kFusedDots)
// and m >= 2.
template <typename R, class Dom>
__device__ bool lanczos_stored_solve(Dom& D, const SolveParams& P, R tau, const typename Cx<R>::T* b,
                                     typename Cx<R>::T* X, typename Cx<R>::T* basis, Counters& cnt, R* sc,
                                     double* res_out) {
  using C = typename Cx<R>::T;
  const GSmem<R> sm = gsmem<R>(D.gm, P.m);
  const int m = P.m;
  C* rr = sm.hess;            // R_jj
  C* rd = sm.hess + m;        // R_{j-1,j}
  C* re = sm.hess + 2 * m;    // R_{j-2,j}
  C* gv = sm.g;               // rotated right-hand side
  C* yv = sm.y;
  const int len = D.len;
  const R dv = (R)D.dv;
  const C mic = cmk<C>((R)0, -tau);
  R nv[1] = {(R)0};
  D.each([&](int i) {
    const C a = b[i];
    nv[0] = fma(a.x, a.x, fma(a.y, a.y, nv[0]));
  });
  if (!D.template sum<1>(nv, sc)) return false;
  const R bn = sqrt(dv * sc[0]);
  const R target = (R)P.tol * bn;
  int total = 0;
  for (int guard = 0; guard < P.max_iters + 2; ++guard) {
    // V_0 = r / ||r||, r = b - A X  (= b on the first cycle when X starts at zero)
    C* V0 = basis;
    R beta1;
    if (guard == 0 && P.x0_zero) {
      D.each([&](int i) { V0[i] = b[i]; });
      __syncthreads();
      beta1 = bn;
    } else {
      D.template hpsi<R, 2>(X, V0, b, (R)1, (R)-1, mic, sc);
      count_hpsi<R>(cnt);
      if (!D.ok()) return false;
      beta1 = sqrt(dv * sc[1]);
    }
    if (guard > 0) cnt.restart++;
    if (beta1 <= target || bn == (R)0) {
      *res_out = (bn > (R)0) ? (double)(beta1 / bn) : 0.0;
      if (total > cnt.max_krylov) cnt.max_krylov = total;
      return true;
    }
    if (total >= P.max_iters) break;
    const R ib = (R)1 / beta1;
    D.each([&](int i) { V0[i] = cscale(ib, V0[i]); });
    __syncthreads();
    C g = cmk<C>(beta1, (R)0);
    R c1 = (R)1, c2 = (R)1;
    C s1 = cmk<C>((R)0, (R)0), s2 = cmk<C>((R)0, (R)0);
    R betak = (R)0, res_est = beta1;
    bool conv = false;
    int nk = 0;   // columns of this cycle
    // The basis holds s_j = gam_j v_j, the Lanczos vectors times known
    // scales, so no iteration needs a normalisation pass: with x = s_{k-1},
    // H x - (gam_{k-1} beta_{k-1} / gam_{k-2}) s_{k-2} = gam_{k-1} (H v_{k-1}
    // - beta_{k-1} v_{k-2}), alpha = Re<x, that> / gam_{k-1}^2, and the pass
    // that removes alpha x leaves gam_{k-1} beta_k v_k = s_k.  A scale that
    // leaves [lo, hi] is reset to 1 by one scaling pass.
    const R lo = sizeof(R) == 8 ? (R)1e-100 : (R)1e-15, hi = (R)1 / lo;
    R gprev = (R)1, gcur = (R)1;   // gam_{k-2}, gam_{k-1}
    if (threadIdx.x == 0) sm.gc[0] = (R)1;
    for (int k = 1; k <= m && total < P.max_iters; ++k) {
      const C* Vc = basis + (size_t)(k - 1) * len;
      C* Wn = basis + (size_t)k * len;
      // Wn = gam_{k-1} (H v_{k-1} - beta_{k-1} v_{k-2}); alpha reduced inside H psi
      if (k == 1)
        D.template hpsi<R, 1>(Vc, Wn, nullptr, (R)0, (R)0, cmk<C>((R)1, (R)0), sc);
      else
        D.template hpsi<R, 1>(Vc, Wn, basis + (size_t)(k - 2) * len, -(gcur * betak / gprev), (R)0,
                           cmk<C>((R)1, (R)0), sc);
      count_hpsi<R>(cnt);
      if (!D.ok()) return false;
      const R alpha = dv * sc[0] / (gcur * gcur);
      R wv[1] = {(R)0};
      D.each([&](int i) {
        const C w = caxpy_r(-alpha, Vc[i], Wn[i]);
        Wn[i] = w;
        wv[0] = fma(w.x, w.x, fma(w.y, w.y, wv[0]));
      });
      if (!D.template sum<1>(wv, sc)) return false;
      const R betan = sqrt(dv * sc[0]) / gcur;
      // column k of [I; 0] + i tau T: rows k-1, k, k+1, rotated (as lanczos_solve)
      C eps = cmk<C>((R)0, (R)0);
      C del = cmk<C>((R)0, tau * betak);
      C gam = cmk<C>((R)1, tau * alpha);
      const C nu = cmk<C>((R)0, tau * betan);
      if (k >= 3) {
        eps = cmul(s2, del);
        del = cscale(c2, del);
      }
      if (k >= 2) {
        const C t = caxpy(s1, gam, cscale(c1, del));
        gam = cnaxpy(cmk<C>(s1.x, -s1.y), del, cscale(c1, gam));
        del = t;
      }
      const R aa = hypot(gam.x, gam.y);
      const R nn = hypot(nu.x, nu.y);
      R c;
      C s, r;
      if (nn == (R)0) {
        c = (R)1;
        s = cmk<C>((R)0, (R)0);
        r = gam;
      } else if (aa == (R)0) {
        c = (R)0;
        s = cmk<C>(nu.x / nn, -nu.y / nn);
        r = cmk<C>(nn, (R)0);
      } else {
        const R rho = hypot(aa, nn);
        const C ph = cmk<C>(gam.x / aa, gam.y / aa);
        c = aa / rho;
        s = cscale((R)1 / rho, cmul(ph, cmk<C>(nu.x, -nu.y)));
        r = cscale(rho, ph);
      }
      if (threadIdx.x == 0) {
        rr[k - 1] = r;
        rd[k - 1] = del;
        re[k - 1] = eps;
        gv[k - 1] = cscale(c, g);
      }
      g = cmk<C>(-(s.x * g.x + s.y * g.y), -(s.x * g.y - s.y * g.x));   // -conj(s) g
      res_est = hypot(g.x, g.y);
      nk = k;
      total++;
      cnt.krylov++;
      cnt.ortho += 1;
      cnt.update += 1;
      c2 = c1;
      s2 = s1;
      c1 = c;
      s1 = s;
      betak = betan;
      if (res_est <= target) {
        conv = true;
        break;
      }
      if (betan <= (sizeof(R) == 8 ? (R)1e-300 : (R)1e-35)) break;
      // gam_k of s_k = Wn; rescaled to 1 when it leaves [lo, hi]
      R gnew = gcur * betan;
      if (!(gnew >= lo && gnew <= hi)) {
        const R ig = (R)1 / gnew;
        D.each([&](int i) { Wn[i] = cscale(ig, Wn[i]); });
        __syncthreads();
        gnew = (R)1;
      }
      gprev = gcur;
      gcur = gnew;
      if (threadIdx.x == 0 && k < m) sm.gc[k] = gnew;
    }
    // y = R^{-1} g by back substitution, then X += V y = sum_j (y_j / gam_j) s_j
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int j = nk - 1; j >= 0; --j) {
        C t = gv[j];
        if (j + 1 < nk) t = cnaxpy(rd[j + 1], yv[j + 1], t);
        if (j + 2 < nk) t = cnaxpy(re[j + 2], yv[j + 2], t);
        const C q = rr[j];
        const R iq = (R)1 / fma(q.x, q.x, q.y * q.y);
        yv[j] = cmul(t, cmk<C>(q.x * iq, -q.y * iq));
      }
      for (int j = 0; j < nk; ++j) yv[j] = cscale((R)1 / sm.gc[j], yv[j]);
    }
    __syncthreads();
    D.each([&](int i) {
      C x = X[i];
      for (int j = 0; j < nk; ++j) x = caxpy(yv[j], basis[(size_t)j * len + i], x);
      X[i] = x;
    });
    __syncthreads();
    if (conv && !P.true_res) {
      *res_out = (bn > (R)0) ? (double)(res_est / bn) : 0.0;
      if (total > cnt.max_krylov) cnt.max_krylov = total;
      return true;
    }
    if (total >= P.max_iters && !conv) break;
  }
  if (total > cnt.max_krylov) cnt.max_krylov = total;
  *res_out = 1e300;
  return false;
}

template <class Dom, typename C>
__device__ __forceinline__ void dcopy(Dom& D, C* dst, const C* src) {
  D.each([&](int i) { dst[i] = src[i]; });
  __syncthreads();
}

// FP64 implicit solve (1 + i tau H) X = b with GMRES in FP64.
template <class Dom>
__device__ bool solve_fp64(Dom& D, const StepPlan& P, double tau, const double2* b, double2* X, Counters& cnt,
                           double* sc, int x0_zero = 0) {
  SolveParams sp{P.tol, P.restart, P.max_iters, P.reorth, P.true_res, P.solver, x0_zero};
  double res = 0.0;
  bool ok;
  if (P.solver == QG_SOLVER_LANCZOS) {
    ok = false;
    if constexpr (Dom::kStoredLanczos) {
      if (sp.m >= 2)
        ok = lanczos_stored_solve<double>(D, sp, tau, b, X, D.basis64, cnt, sc, &res);
      else
        ok = lanczos_solve<double>(D, sp, tau, b, X, D.basis64, cnt, sc, &res);
    } else {
      ok = lanczos_solve<double>(D, sp, tau, b, X, D.basis64, cnt, sc, &res);
    }
  } else {
    ok = gmres_solve<double>(D, sp, tau, b, X, D.basis64, cnt, sc, &res);
  }
  if (ok && res > cnt.max_res) cnt.max_res = res;
  if (!ok) cnt.max_res = 1e300;
  return ok;
}

// Mixed-precision implicit solve: FP64 residual r = b - (1 + i tau H) X,
// complex64 GMRES for (1 + i tau H) d = r / ||r|| to inner_tol, X += ||r|| d,
// until ||r|| <= tol ||b||.
//
// r0_ready: D.res64 already holds an estimate of b - (1 + i tau H) X (from
// carried H^2 psi, see run_steps).  It only seeds the first inner solve: the
// refinement stops on exactly computed FP64 residuals only.
template <class Dom>
__device__ bool solve_mixed(Dom& D, const StepPlan& P, double tau, const double2* b, double2* X, Counters& cnt,
                            double* sc, int x0_zero = 0, bool r0_ready = false) {
  double2* Rv = D.res64;
  float2* r32 = D.r32;
  float2* d32 = D.d32;
  float* scf = reinterpret_cast<float*>(sc);
  const double2 mic = make_double2(0.0, -tau);
  const double dv = D.dv;
  double nv[1] = {0.0};
  D.each([&](int i) {
    const double2 a = b[i];
    nv[0] = fma(a.x, a.x, fma(a.y, a.y, nv[0]));
  });
  if (!D.template sum<1>(nv, sc)) return false;
  const double bn = sqrt(dv * sc[0]);
  const double target = P.tol * bn;
  SolveParams sp{P.inner_tol, P.restart, P.max_iters, P.reorth, 0, P.solver, 1};
  double prev_rho = 0.0;
  bool have_prev = false;
  for (int outer = 0; outer <= P.max_outer; ++outer) {
    double rho;
    const bool estimate = outer == 0 && r0_ready && !x0_zero;
    if (outer == 0 && x0_zero) {
      D.each([&](int i) { Rv[i] = b[i]; });
      __syncthreads();
      rho = bn;
    } else if (estimate) {
      double rv[1] = {0.0};
      D.each([&](int i) {
        const double2 a = Rv[i];
        rv[0] = fma(a.x, a.x, fma(a.y, a.y, rv[0]));
      });
      if (!D.template sum<1>(rv, sc)) return false;
      rho = sqrt(dv * sc[0]);
    } else if constexpr (Dom::kFusedDots) {
      D.template hpsi<double, 2>(X, Rv, b, 1.0, -1.0, mic, sc);
      cnt.hpsi++;
      if (!D.ok()) return false;
      rho = sqrt(dv * sc[1]);
    } else {
      D.template hpsi<double>(X, Rv, b, 1.0, -1.0, mic);
      cnt.hpsi++;
      double rv[1] = {0.0};
      D.each([&](int i) {
        const double2 a = Rv[i];
        rv[0] = fma(a.x, a.x, fma(a.y, a.y, rv[0]));
      });
      if (!D.template sum<1>(rv, sc)) return false;
      rho = sqrt(dv * sc[0]);
    }
    // Converged when the exactly computed FP64 residual meets the target --
    // or when it has stopped falling at the rounding level of the FP64
    // residual itself (within 256 u ||b||): a tolerance near 1e-15 can sit
    // below what an FP64 H psi of a long, stiff grid resolves, and further
    // refinement then only moves the residual within its rounding noise.
    // max_residual reports what was reached.
    const bool at_floor = !estimate && have_prev && rho > 0.5 * prev_rho && rho <= 256.0 * DBL_EPSILON * bn;
    if (!estimate && (rho <= target || bn == 0.0 || at_floor)) {
      const double r = bn > 0.0 ? rho / bn : 0.0;
      if (r > cnt.max_res) cnt.max_res = r;
      return true;
    }
    if (!estimate) {
      prev_rho = rho;
      have_prev = true;
    }
    if (outer == P.max_outer) break;
    if (estimate && rho == 0.0) continue;   // nothing to refine: check exactly
    cnt.outer++;
    // the inner solve need not reduce the residual further than the outer
    // target asks (with a factor 4 in hand): the last refinement step is
    // usually looser than inner_tol
    sp.tol = fmax(P.inner_tol, 0.25 * target / rho);
    const double ir = 1.0 / rho;
    D.each([&](int i) {
      const double2 v = Rv[i];
      r32[i] = make_float2((float)(v.x * ir), (float)(v.y * ir));
      d32[i] = make_float2(0.f, 0.f);
    });
    __syncthreads();
    double res = 0.0;
    if (P.solver == QG_SOLVER_LANCZOS) {
      if constexpr (Dom::kStoredLanczos32) {
        if (sp.m >= 2)
          lanczos_stored_solve<float>(D, sp, (float)tau, r32, d32, D.basis32, cnt, scf, &res);
        else
          lanczos_solve<float>(D, sp, (float)tau, r32, d32, D.basis32, cnt, scf, &res);
      } else {
        lanczos_solve<float>(D, sp, (float)tau, r32, d32, D.basis32, cnt, scf, &res);
      }
    } else
      gmres_solve<float>(D, sp, (float)tau, r32, d32, D.basis32, cnt, scf, &res);
    if (!D.ok()) return false;
    D.each([&](int i) {
      const float2 d = d32[i];
      const double2 x = X[i];
      X[i] = make_double2(fma(rho, (double)d.x, x.x), fma(rho, (double)d.y, x.y));
    });
    __syncthreads();
  }
  cnt.max_res = 1e300;
  return false;
}

// Explicit-Euler initial guess X = (1 - i tau H) src, in complex64 for the
// mixed-precision form (only the starting point of the refinement).
template <class Dom>
__device__ void guess_mixed(Dom& D, double tau, const double2* src, double2* X, Counters& cnt) {
  float2* s32 = D.r32;
  float2* y32 = D.d32;
  D.each([&](int i) {
    const double2 v = src[i];
    s32[i] = make_float2((float)v.x, (float)v.y);
  });
  __syncthreads();
  D.template hpsi<float>(s32, y32, nullptr, 0.f, 1.f, make_float2(0.f, (float)-tau));
  cnt.hpsi32++;
  D.each([&](int i) {
    const float2 y = y32[i];
    X[i] = make_double2((double)y.x, (double)y.y);
  });
  __syncthreads();
}

__device__ __forceinline__ void write_stats(qg_step_stats* st, const Counters& cnt, long long nsub, long long failed) {
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

// All nsteps composed steps (Secs. II B-C) of one instance.  psi is the
// state, B/X/P0 workspace vectors, ckpt optional checkpoints (every `every`
// composed steps, nckpt of them).  Returns the index of the failed composed
// step or -1.
// Solves (1 + i tau H) X = b: in FP64 (MODE 0), in the mixed-precision form
// (MODE 1), or as `mixed` says at run time (MODE 2).  A kernel built for one
// form compiles only that form.  X starts from the explicit-Euler guess
// (1 - i tau H) b (Sec. II B) or, with QG_GUESS_ZERO, from zero: the
// minimal-residual iterate from zero after k + 2 iterations minimises over
// K_{k+2}(H, b), which contains every point the Euler guess reaches after k
// iterations for the same k + 2 H psi evaluations.
// guess_ready: X already holds the explicit-Euler start (formed by the caller
// without an H psi evaluation).
template <int MODE, class Dom>
__device__ __forceinline__ bool implicit_solve(Dom& D, const StepPlan& P, double tau, const double2* b, double2* X,
                                               bool mixed, Counters& cnt, double* sc, bool guess_ready = false,
                                               bool r0_ready = false) {
  const int zero = !guess_ready && P.guess == QG_GUESS_ZERO;
  if (zero) {
    D.each([&](int i) { X[i] = make_double2(0.0, 0.0); });
    __syncthreads();
  }
  if constexpr (MODE != 0) {
    if (MODE == 1 || mixed) {
      if (!zero && !guess_ready) guess_mixed(D, tau, b, X, cnt);
      return solve_mixed(D, P, tau, b, X, cnt, sc, zero, r0_ready);
    }
  }
  if constexpr (MODE != 1) {
    if (!zero && !guess_ready) {
      D.template hpsi<double>(b, X, nullptr, 0.0, 1.0, make_double2(0.0, -tau));
      cnt.hpsi += 1;
    }
    return solve_fp64(D, P, tau, b, X, cnt, sc, zero);
  }
  return false;
}

// The elementary comparison methods of Sec. II B, each step of size
// eps = dt (hbar = 1), never composed:
//   explicit Euler  psi' = (1 - i eps H) psi                  Eq. (exp_euler)
//   implicit Euler  (1 + i eps H) psi' = psi                  Eq. (imp_euler)
//   SOD             psi(t + eps) = psi(t - eps) - 2 i eps H psi(t)
//                                                             Eq. (sod_method)
// SOD starts from psi(-eps) taken by one two-stage Runge-Kutta step backward,
// psi + i eps H psi - (eps^2 / 2) H^2 psi (Sec. III), at the start of every
// call.  Three vectors rotate (psi, B, X); T is one more scratch vector.
// Returns the index of the failed step or -1.
template <int MODE, class Dom>
__device__ long long run_elementary(Dom& D, const StepPlan& P, double2* psi, double2* B, double2* X, double2* T,
                                    bool mixed, Counters& cnt, long long& nsub, double* sc) {
  const double eps = P.dt;
  double2* cur = psi;
  double2* nxt = X;
  long long failed = -1;
  if (P.method == QG_SOD) {
    double2* prv = B;
    D.template hpsi<double>(psi, X, nullptr, 0.0, 0.0, make_double2(1.0, 0.0));     // X = H psi
    D.template hpsi<double>(X, T, nullptr, 0.0, 0.0, make_double2(1.0, 0.0));       // T = H^2 psi
    cnt.hpsi += 2;
    const double h2 = 0.5 * eps * eps;
    D.each([&](int i) {
      const double2 p = psi[i], h = X[i], g = T[i];
      prv[i] = make_double2(p.x - eps * h.y - h2 * g.x, p.y + eps * h.x - h2 * g.y);
    });
    __syncthreads();
    for (long long step = 0; step < P.nsteps; ++step) {
      D.template hpsi<double>(cur, nxt, prv, 1.0, 0.0, make_double2(0.0, -2.0 * eps));
      cnt.hpsi += 1;
      if (!D.ok()) {
        failed = step;
        break;
      }
      double2* t = prv;
      prv = cur;
      cur = nxt;
      nxt = t;
      nsub++;
    }
  } else {
    for (long long step = 0; step < P.nsteps; ++step) {
      bool ok = true;
      if (P.method == QG_EXPLICIT_EULER) {
        D.template hpsi<double>(cur, nxt, nullptr, 0.0, 1.0, make_double2(0.0, -eps));
        cnt.hpsi += 1;
      } else {
        ok = implicit_solve<MODE>(D, P, eps, cur, nxt, mixed, cnt, sc);
      }
      if (!ok || !D.ok()) {
        failed = step;
        break;
      }
      double2* t = cur;
      cur = nxt;
      nxt = t;
      nsub++;
    }
  }
  if (failed < 0 && cur != psi) dcopy(D, psi, cur);
  return failed;
}

template <int MODE, class Dom>
__device__ long long run_steps(Dom& D, const StepPlan& P, double2* psi, double2* B, double2* X, double2* P0,
                               bool mixed, double2* ckpt, long long nckpt, long long every, Counters& cnt,
                               long long& nsub, double* sc) {
  const int len = D.len;
  long long failed = -1;
  if (P.method >= QG_EXPLICIT_EULER) {
    dcopy(D, P0, psi);
    failed = run_elementary<MODE>(D, P, psi, B, X, D.basis64, mixed, cnt, nsub, sc);
    if (failed >= 0) dcopy(D, psi, P0);
    return failed;
  }
  bool mixed_now = false;
  if constexpr (MODE == 1) mixed_now = true;
  if constexpr (MODE == 2) mixed_now = mixed;
  // midpoint with the explicit-Euler start and psi' = 2 chi - psi: carry
  // H psi from one sub-step to the next in B (unused by the midpoint rule).
  // The mixed form with a single fraction per step (order 2) recomputes the
  // carried vectors every step, which costs more FP64 H psi than its
  // complex64 Euler start, so it does not carry them.
  const bool recycle = P.method != QG_TRAPEZOIDAL && P.guess == QG_GUESS_EULER && !P.mid_epi &&
                       !(mixed_now && P.nfrac == 1);
  // the mixed form also carries H^2 psi (in the FP64 basis slot after its
  // residual, unused by that form): the residual of the Euler start is then
  // -tau^2 H^2 psi, and its first FP64 residual costs no H psi
  const bool carry2 = recycle && mixed_now;
  double2* H2 = D.res64 + len;
  dcopy(D, P0, psi);
  for (long long step = 0; step < P.nsteps && failed < 0; ++step) {
    if (P.run == QG_RUN_CHECKPOINT && ckpt && step % every == 0 && step / every < nckpt)
      dcopy(D, ckpt + (size_t)(step / every) * len, psi);
    for (int f = 0; f < P.nfrac; ++f) {
      const double tau = 0.5 * P.frac[f] * P.dt;   // hbar = 1
      const double2 mic = make_double2(0.0, -tau);
      bool ok;
      if (P.method == QG_TRAPEZOIDAL) {
        // b = (1 - i tau H) psi ; guess x0 = (1 - i tau H) b ; solve (1 + i tau H) x = b
        D.template hpsi<double>(psi, B, nullptr, 0.0, 1.0, mic);
        cnt.hpsi += 1;
        ok = implicit_solve<MODE>(D, P, tau, B, X, mixed, cnt, sc);
        if (ok) dcopy(D, psi, X);
      } else {
        // guess chi0 = (1 - i tau H) psi ; solve (1 + i tau H) chi = psi ;
        // psi' = (1 - i tau H) chi  (or 2 chi - psi)
        if (recycle) {
          // B carries H psi: exact at the first fraction of each composed
          // step, then by the recurrence below, so the explicit-Euler start
          // costs no H psi (the solve still forms its true residual)
          if (f == 0) {
            D.template hpsi<double>(psi, B, nullptr, 0.0, 0.0, make_double2(1.0, 0.0));
            cnt.hpsi += 1;
            if (carry2) {
              D.template hpsi<double>(B, H2, nullptr, 0.0, 0.0, make_double2(1.0, 0.0));
              cnt.hpsi += 1;
            }
          }
          const double t2 = tau * tau;
          double2* Rv = D.res64;
          D.each([&](int i) {
            const double2 p = psi[i], h = B[i];
            X[i] = make_double2(fma(tau, h.y, p.x), fma(-tau, h.x, p.y));
            if (carry2) {
              const double2 g = H2[i];
              Rv[i] = make_double2(-t2 * g.x, -t2 * g.y);   // psi - (1 + i tau H) X
            }
          });
          __syncthreads();
          ok = implicit_solve<MODE>(D, P, tau, psi, X, mixed, cnt, sc, true, carry2);
        } else {
          ok = implicit_solve<MODE>(D, P, tau, psi, X, mixed, cnt, sc);
        }
        if (ok) {
          if (P.mid_epi) {
            D.template hpsi<double>(X, psi, nullptr, 0.0, 1.0, mic);
            cnt.hpsi += 1;
          } else {
            // psi' = 2 chi - psi and, when recycling, H psi' = 2 H chi - H psi
            // with H chi = i (chi - psi) / tau from (1 + i tau H) chi = psi
            const double it = 1.0 / tau;
            D.each([&](int i) {
              const double2 c = X[i], p = psi[i];
              if (recycle) {
                const double2 h = B[i];
                const double dx = (c.x - p.x) * it, dy = (c.y - p.y) * it;
                const double2 hc = make_double2(-dy, dx);               // H chi
                B[i] = make_double2(2.0 * hc.x - h.x, 2.0 * hc.y - h.y);
                if (carry2) {
                  // H^2 chi = i (H chi - H psi) / tau ; H^2 psi' = 2 H^2 chi - H^2 psi
                  const double2 g = H2[i];
                  const double ex = (hc.x - h.x) * it, ey = (hc.y - h.y) * it;
                  H2[i] = make_double2(-2.0 * ey - g.x, 2.0 * ex - g.y);
                }
              }
              psi[i] = make_double2(2.0 * c.x - p.x, 2.0 * c.y - p.y);
            });
            __syncthreads();
          }
        }
      }
      if (!ok || !D.ok()) {
        failed = step;
        break;
      }
      nsub++;
    }
  }
  if (failed >= 0) dcopy(D, psi, P0);
  return failed;
}

}  // namespace qg
