// Two-dimensional grids: one instance is spread over every CTA of one
// cooperative launch (all CTAs co-resident).  Each CTA owns a band of rows
// (q1 index) for the pointwise work and the dimension-1 transforms, and a
// band of columns for the dimension-0 transforms; a bounded grid barrier
// separates the phases.  Sums over the state are formed per CTA, exchanged
// through global memory and added by every CTA in the same fixed order, so
// every CTA takes the same decisions.
//
// Every translation unit that includes this header is compiled with
// -Xptxas -dlcm=cg: global loads are cached in L2 only, so data written by
// other CTAs in the same launch is never read from a stale L1 line.
#pragma once
#include <cuda_runtime.h>

#include "qg_solver.cuh"

namespace qg {

static __device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

static __device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded sense-reversing grid barrier (all CTAs are co-resident under the
// cooperative launch).  Thread 0 of each CTA publishes the CTA's writes,
// arrives on a counter, and polls the generation word with acquire loads.
// A CTA that waits more than about a second gives up, raises the error flag
// and returns false; every later barrier then fails too, so every CTA leaves
// the kernel.
static __device__ bool grid_barrier(unsigned* bar, int* err) {
  __shared__ int s_fail;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ld_acquire_gpu(bar + 1);
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    int fail = 0;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      for (long long spins = 1; ld_acquire_gpu(bar + 1) == g; ++spins) {
        if ((spins & 31) == 0) {
          if (ld_acquire_gpu(reinterpret_cast<const unsigned*>(err))) {   // another CTA already gave up
            fail = 1;
            break;
          }
          if (globaltimer_ns() - t0 > 1000000000ull || spins > (1LL << 23)) {
            fail = 1;
            atomicExch(err, 1);
            break;
          }
        }
      }
    }
    __threadfence();
    if (ld_acquire_gpu(reinterpret_cast<const unsigned*>(err))) fail = 1;
    s_fail = fail;
  }
  __syncthreads();
  return s_fail == 0;
}

struct Dom2D {
  // H psi can form Re<x, y> and ||y||^2 in its last pass and reduce them
  // across the grid in its closing barrier (see hpsi); the solvers use that
  // for alpha and for residual norms
  static constexpr bool kFusedDots = true;
  // the FP64 Lanczos solve keeps its vectors in the workspace basis (lanczos_stored_solve)
  static constexpr bool kStoredLanczos = true;
  // the same for the complex64 inner solves of the mixed form (measured faster here: 15.3 against 15.8 ms per 2-D mixed step)
  static constexpr bool kStoredLanczos32 = true;
  const Inst2D* I;
  int len, N, n0, n1, S;
  int r_lo, r_hi, c_lo, c_hi;
  double dv;
  unsigned char* gm;
  double* red;
  unsigned char* fb;
  HOp<double> H64[2];
  HOp<float> H32[2];
  double2 *U64, *T64;
  float2 *U32, *T32;
  double2* basis64;
  double2* res64;
  float2 *r32, *d32, *basis32;
  int parity;
  bool good;
  int cap_elems;   // complex values one shared-memory FFT batch may hold
  unsigned char* stage;   // shared copies of x and U for one batch (2 cap_elems
                          // complex doubles), or null: read them from global

  // Every point of the owned rows, all surfaces.  Members are copied to
  // registers first (stores through generic pointers in f could alias *this).
  template <class F>
  __device__ __forceinline__ void each(F&& f) {
    const int per = (r_hi - r_lo) * n1;
    const int ns = S, stride = N, first = r_lo * n1;
    for (int s = 0; s < ns; ++s) {
      const int base = s * stride + first;
      for (int k = threadIdx.x; k < per; k += kThreads) f(base + k);
    }
  }
  // each with loads and stores split (see the 1-D domain); one at a time here
  template <int U, class Ld, class St>
  __device__ __forceinline__ void each_u(Ld&& ld, St&& st) {
    each([&](int i) { st(i, ld(i)); });
  }

  // Adds the per-CTA partial sums buf[b * 32 + k], b < gridDim.x, k < K:
  // warp w handles k = w, w + kWarps, ..., loads 32 partials at a time and
  // reduces with a fixed shuffle tree, so every CTA forms the same values in
  // the same order.
  template <int K, typename R>
  __device__ __forceinline__ void gather(const R* buf, R* out) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = w; k < K; k += kWarps) {
      R s = 0;
      for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(buf + b * 32 + k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) out[k] = s;
    }
    __syncthreads();
  }

  template <int K, typename R>
  __device__ __forceinline__ bool sum(R (&v)[K], R* out) {
    cta_sum<K>(v, reinterpret_cast<R*>(red), out);
    R* buf = reinterpret_cast<R*>(I->gred + (size_t)parity * gridDim.x * 32);
    parity ^= 1;
    if (threadIdx.x < K) buf[blockIdx.x * 32 + threadIdx.x] = out[threadIdx.x];
    good = good && grid_barrier(I->bar, I->err);
    gather<K>(buf, out);
    return good;
  }

  __device__ __forceinline__ bool ok() const { return good; }

  // y = e z + a x + c (H x), H = sum_d -hbar^2/2m_d (D_d + F_d)^2 + V.
  // With dots (shared memory, 2 values): also dots[0] = sum Re(conj(x) y)
  // and dots[1] = sum |y|^2 over the whole grid (without the grid weight),
  // reduced in the closing grid barrier; every CTA gets the same values.
  // Both sums are formed whichever of them W (bit 0, bit 1) asks for.
  template <typename R, int W = 3>
  __device__ __forceinline__ void hpsi(const typename Cx<R>::T* x, typename Cx<R>::T* y, const typename Cx<R>::T* z,
                                       R e, R a, typename Cx<R>::T c, R* dots = nullptr) {
    hpsi_all<R>(x, y, z, e, a, c, dots);
  }
  template <typename R>
  __device__ __noinline__ void hpsi_all(const typename Cx<R>::T* x, typename Cx<R>::T* y, const typename Cx<R>::T* z,
                                        R e, R a, typename Cx<R>::T c, R* dots) {
    using C = typename Cx<R>::T;
    // members in registers: the stores below go through generic pointers
    // that could alias *this, which would force reloads from local memory
    const int n0 = this->n0, n1 = this->n1, N = this->N, S = this->S;
    const int r_lo = this->r_lo, r_hi = this->r_hi, c_lo = this->c_lo, c_hi = this->c_hi;
    const int cap_elems = this->cap_elems;
    C* sb = in_dyn_smem(reinterpret_cast<C*>(fb));
    // staged batch: xs[e] = x and us[e] = U at the batch position e of the
    // FFT buffer (no padding), so the pointwise loops read no global memory
    C* xs = stage ? in_dyn_smem(reinterpret_cast<C*>(stage)) : nullptr;
    C* us = xs ? xs + cap_elems : nullptr;
    const HOp<R>* H = nullptr;
    C* U;
    C* T;
    const R* V;
    const R* F;
    if constexpr (sizeof(R) == 8) {
      H = H64;
      U = U64;
      T = T64;
      V = I->V;
      F = I->F;
    } else {
      H = H32;
      U = U32;
      T = T32;
      V = I->V32;
      F = I->F32;
    }
    const int npair = S * (S - 1) / 2;
    // ---- dimension 1 (rows, contiguous): T = -h2m_1 (D_1 + F_1)^2 x + V x.
    // All owned rows and all surfaces form one shared-memory FFT batch:
    // vector (row_local * S + s) holds x_s on that row.
    {
      const HOp<R>& H1 = H[1];
      const R mh = -(R)I->h2m[1];
      const R* F1 = F + (size_t)1 * npair * N;
      const int rb = max(1, min(r_hi - r_lo, cap_elems / (S * n1)));
      for (int r0 = r_lo; r0 < r_hi; r0 += rb) {
      const int nrow = min(rb, r_hi - r0);
      const int nv = nrow * S;
      for (int k = threadIdx.x; k < nv * n1; k += kThreads) {
        const int v = k / n1, j = k - v * n1;
        const int rl = v / S, s = v - rl * S;
        const C val = x[(size_t)s * N + (size_t)(r0 + rl) * n1 + j];
        sb[spad<C>(k)] = val;
        if (xs) xs[k] = val;
      }
      __syncthreads();
      if (nv > 0) spectral_derivative<R>(sb, nv, H1);
      for (int k = threadIdx.x; k < nrow * n1; k += kThreads) {
        const int rl = k / n1, j = k - rl * n1;
        const size_t p = (size_t)(r0 + rl) * n1 + j;
        for (int s = 0; s < S; ++s) {
          const int e = (rl * S + s) * n1 + j;
          C acc = sb[spad<C>(e)];
          for (int t = 0; t < S; ++t)
            if (t != s)
              acc = caxpy_r(coupling2(F1, N, S, s, t, p), xs ? xs[(rl * S + t) * n1 + j] : x[(size_t)t * N + p], acc);
          if (us)
            us[e] = acc;
          else
            U[(size_t)s * N + p] = acc;
          sb[spad<C>(e)] = acc;
        }
      }
      __syncthreads();
      if (nv > 0) spectral_derivative<R>(sb, nv, H1);
      for (int k = threadIdx.x; k < nrow * n1; k += kThreads) {
        const int rl = k / n1, j = k - rl * n1;
        const size_t p = (size_t)(r0 + rl) * n1 + j;
        for (int s = 0; s < S; ++s) {
          C acc = sb[spad<C>((rl * S + s) * n1 + j)];
          for (int t = 0; t < S; ++t)
            if (t != s)
              acc = caxpy_r(coupling2(F1, N, S, s, t, p), us ? us[(rl * S + t) * n1 + j] : U[(size_t)t * N + p], acc);
          const C xv = xs ? xs[(rl * S + s) * n1 + j] : x[(size_t)s * N + p];
          const R v = __ldg(V + (size_t)s * N + p);
          T[(size_t)s * N + p] = cmk<C>(fma(mh, acc.x, v * xv.x), fma(mh, acc.y, v * xv.y));
        }
      }
      __syncthreads();
      }
    }
    good = good && grid_barrier(I->bar, I->err);
    // ---- dimension 0 (columns, stride n1): y = e z + a x + c (T - h2m_0 (D_0 + F_0)^2 x).
    // All owned columns and surfaces form one batch: vector (col_local * S + s).
    R pd[2] = {(R)0, (R)0};
    {
      const HOp<R>& H0 = H[0];
      const R mh = -(R)I->h2m[0];
      const R* F0 = F;
      const int cb = max(1, min(c_hi - c_lo, cap_elems / (S * n0)));
      for (int c0 = c_lo; c0 < c_hi; c0 += cb) {
      const int ncol = min(cb, c_hi - c0);
      const int nv = ncol * S;
      for (int k = threadIdx.x; k < nv * n0; k += kThreads) {
        const int v = k / n0, i = k - v * n0;
        const int cl = v / S, s = v - cl * S;
        const C val = x[(size_t)s * N + (size_t)i * n1 + (c0 + cl)];
        sb[spad<C>(k)] = val;
        if (xs) xs[k] = val;
      }
      __syncthreads();
      if (nv > 0) spectral_derivative<R>(sb, nv, H0);
      for (int k = threadIdx.x; k < ncol * n0; k += kThreads) {
        const int cl = k / n0, i = k - cl * n0;
        const size_t p = (size_t)i * n1 + (c0 + cl);
        for (int s = 0; s < S; ++s) {
          const int e = (cl * S + s) * n0 + i;
          C acc = sb[spad<C>(e)];
          for (int t = 0; t < S; ++t)
            if (t != s)
              acc = caxpy_r(coupling2(F0, N, S, s, t, p), xs ? xs[(cl * S + t) * n0 + i] : x[(size_t)t * N + p], acc);
          if (us)
            us[e] = acc;
          else
            U[(size_t)s * N + p] = acc;
          sb[spad<C>(e)] = acc;
        }
      }
      __syncthreads();
      if (nv > 0) spectral_derivative<R>(sb, nv, H0);
      for (int k = threadIdx.x; k < ncol * n0; k += kThreads) {
        const int cl = k / n0, i = k - cl * n0;
        const size_t p = (size_t)i * n1 + (c0 + cl);
        for (int s = 0; s < S; ++s) {
          C acc = sb[spad<C>((cl * S + s) * n0 + i)];
          for (int t = 0; t < S; ++t)
            if (t != s)
              acc = caxpy_r(coupling2(F0, N, S, s, t, p), us ? us[(cl * S + t) * n0 + i] : U[(size_t)t * N + p], acc);
          const C tt = T[(size_t)s * N + p];
          const C hx = cmk<C>(fma(mh, acc.x, tt.x), fma(mh, acc.y, tt.y));
          const C xv = xs ? xs[(cl * S + s) * n0 + i] : x[(size_t)s * N + p];
          C out = caxpy(c, hx, cmk<C>(a * xv.x, a * xv.y));
          if (e != (R)0) out = caxpy_r(e, z[(size_t)s * N + p], out);
          y[(size_t)s * N + p] = out;
          if (dots) {
            pd[0] = fma(xv.x, out.x, fma(xv.y, out.y, pd[0]));
            pd[1] = fma(out.x, out.x, fma(out.y, out.y, pd[1]));
          }
        }
      }
      __syncthreads();
      }
    }
    R* buf = reinterpret_cast<R*>(I->gred + (size_t)parity * gridDim.x * 32);
    if (dots) {
      cta_sum<2>(pd, reinterpret_cast<R*>(red), dots);
      if (threadIdx.x < 2) buf[blockIdx.x * 32 + threadIdx.x] = dots[threadIdx.x];
    }
    good = good && grid_barrier(I->bar, I->err);
    if (dots) {
      gather<2>(buf, dots);
      parity ^= 1;
    }
  }

  // F_{st} at flattened point p from one dimension's upper triangle.
  template <typename R>
  __device__ static __forceinline__ R coupling2(const R* Fd, int N, int S, int s, int t, size_t p) {
    const int a = s < t ? s : t, b = s < t ? t : s;
    const int q = a * S - (a * (a + 1)) / 2 + (b - a - 1);
    return neg_if(__ldg(Fd + (size_t)q * N + p), s > t);   // F_ts = -F_st
  }
};

// Shared-memory copy of both dimensions' FFT tables: FP64 twiddles, FP64
// wave numbers, FP32 twiddles, FP32 wave numbers, each dimension 0 then 1
// (36 (n0 + n1) bytes), then the FP64 Linzer-Feig factor tables of
// dimension 0 and 1.  The 2-D units read global memory through L2 only, so
// tables kept in global memory would cost an L2 round trip every pass.
__host__ __device__ inline size_t tables2d_bytes(int n0, int n1) {
  return ((size_t)36 * (n0 + n1) + 15) / 16 * 16 + lf_table_bytes(n0) + lf_table_bytes(n1);
}

// tab_off > 0: the tables are copied to dyn + tab_off (16-byte aligned) and
// the transforms read them from there.
static __device__ Dom2D make_dom2d(const Inst2D& I, unsigned char* dyn, int fft_bytes, double* red,
                                   int tab_off = 0, int stage_bytes = 0) {
  Dom2D D;
  D.I = &I;
  D.n0 = I.n[0];
  D.n1 = I.n[1];
  D.S = I.S;
  D.N = D.n0 * D.n1;
  D.len = D.S * D.N;
  const int G = gridDim.x;
  const int rp = (D.n0 + G - 1) / G, cp = (D.n1 + G - 1) / G;
  D.r_lo = min(D.n0, (int)blockIdx.x * rp);
  D.r_hi = min(D.n0, D.r_lo + rp);
  D.c_lo = min(D.n1, (int)blockIdx.x * cp);
  D.c_hi = min(D.n1, D.c_lo + cp);
  D.dv = I.dv;
  D.fb = dyn;
  D.stage = stage_bytes > 0 ? dyn + fft_bytes : nullptr;
  D.gm = dyn + fft_bytes + stage_bytes;
  D.red = red;
  for (int d = 0; d < 2; ++d) {
    D.H64[d].diab = 0;
    D.H32[d].diab = 0;
    D.H64[d].n = I.n[d];
    D.H64[d].S = I.S;
    D.H64[d].npass = I.npass[d];
    D.H64[d].n8 = count_radix8(I.radix[d], I.npass[d]);
    D.H64[d].h2m = I.h2m[d];
    D.H64[d].tw = I.tw[d];
    D.H64[d].kd = I.kd[d];
    D.H64[d].lf = I.lf[d];
    D.H64[d].lff = I.lff[d];
    D.H32[d].n = I.n[d];
    D.H32[d].S = I.S;
    D.H32[d].npass = I.npass[d];
    D.H32[d].n8 = count_radix8(I.radix[d], I.npass[d]);
    D.H32[d].h2m = (float)I.h2m[d];
    D.H32[d].tw = I.tw32[d];
    D.H32[d].kd = I.kd32[d];
  }
  if (tab_off > 0) {
    const int nt = D.n0 + D.n1;
    unsigned char* t = dyn + tab_off;
    double2* tw64 = reinterpret_cast<double2*>(t);
    double* kd64 = reinterpret_cast<double*>(t + (size_t)16 * nt);
    float2* tw32 = reinterpret_cast<float2*>(t + (size_t)24 * nt);
    float* kd32 = reinterpret_cast<float*>(t + (size_t)32 * nt);
    int base = 0;
    for (int d = 0; d < 2; ++d) {
      const int n = I.n[d];
      for (int i = threadIdx.x; i < n; i += kThreads) {
        tw64[base + i] = I.tw[d][i];
        kd64[base + i] = I.kd[d][i];
        tw32[base + i] = I.tw32[d][i];
        kd32[base + i] = I.kd32[d][i];
      }
      D.H64[d].tw = tw64 + base;
      D.H64[d].kd = kd64 + base;
      D.H32[d].tw = tw32 + base;
      D.H32[d].kd = kd32 + base;
      base += n;
    }
    // then the factor tables of both dimensions (whole 16-byte words each)
    unsigned char* lft = t + (((size_t)36 * nt + 15) / 16 * 16);
    for (int d = 0; d < 2; ++d) {
      if (!I.lf[d]) continue;
      const int words = (int)(lf_table_bytes(I.n[d]) / 16);
      const int4* src = reinterpret_cast<const int4*>(I.lf[d]);
      int4* dst = reinterpret_cast<int4*>(lft);
      for (int k = threadIdx.x; k < words; k += kThreads) dst[k] = src[k];
      D.H64[d].lf = reinterpret_cast<const double2*>(lft);
      D.H64[d].lff = reinterpret_cast<const unsigned*>(
          lft + (reinterpret_cast<const unsigned char*>(I.lff[d]) - reinterpret_cast<const unsigned char*>(I.lf[d])));
      lft += (size_t)words * 16;
    }
    __syncthreads();
  }
  const size_t len = D.len;
  // FP64 workspace: U, T, B, X, P0, basis (m + 1); the mixed form keeps its
  // FP64 residual in basis slot 0.
  D.U64 = I.work;
  D.T64 = I.work + len;
  D.basis64 = I.work + 5 * len;
  D.res64 = D.basis64;
  if (I.work32) {
    D.U32 = I.work32;
    D.T32 = I.work32 + len;
    D.r32 = I.work32 + 2 * len;
    D.d32 = I.work32 + 3 * len;
    D.basis32 = I.work32 + 4 * len;
  } else {
    D.U32 = D.T32 = D.r32 = D.d32 = D.basis32 = nullptr;
  }
  D.parity = 0;
  D.good = true;
  // complex doubles (with padding) the FFT buffer holds; complex floats
  // need less room for the same count
  D.cap_elems = (int)padded_capacity((size_t)fft_bytes, 16);
  return D;
}

}  // namespace qg
