// Device building blocks: complex arithmetic, deterministic CTA reductions,
// the shared-memory FFT and the fused Hamiltonian action (Sec. II D-E),
// templated on the real type R (double for the FP64 path, float for the
// inner iterations of the mixed-precision form).
//
// Every CTA works on one instance.  All loops are bounded; nothing waits on
// another CTA.
#pragma once

#include "qg_internal.h"

namespace qg {

constexpr int kThreads = QG_THREADS;
constexpr int kWarps = QG_THREADS / 32;

// Base of the dynamic shared memory of every kernel here (all declarations
// of an extern __shared__ array name the same block).
extern __shared__ __align__(16) unsigned char qg_dyn_smem[];

// p, a generic pointer into the dynamic shared memory, rebased on
// qg_dyn_smem: the compiler then knows the address space and emits shared
// loads and stores instead of generic ones.  The FFT buffers always live in
// dynamic shared memory, but reach the transforms through structures whose
// address space the compiler cannot see.
template <typename T>
__device__ __forceinline__ T* in_dyn_smem(T* p) {
  return reinterpret_cast<T*>(qg_dyn_smem + (reinterpret_cast<unsigned char*>(p) - qg_dyn_smem));
}

template <typename R>
struct Cx;
template <>
struct Cx<double> {
  using T = double2;
};
template <>
struct Cx<float> {
  using T = float2;
};

template <typename C>
__device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) {
  C c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
// a * b
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {
  return cmk<C>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
template <typename C, typename R>
__device__ __forceinline__ C cscale(R s, C a) { return cmk<C>(s * a.x, s * a.y); }
// a + s * b (s real)
template <typename C, typename R>
__device__ __forceinline__ C caxpy_r(R s, C b, C a) { return cmk<C>(fma(s, b.x, a.x), fma(s, b.y, a.y)); }
// a + c * b (c complex)
template <typename C>
__device__ __forceinline__ C caxpy(C c, C b, C a) {
  return cmk<C>(fma(c.x, b.x, fma(-c.y, b.y, a.x)), fma(c.x, b.y, fma(c.y, b.x, a.y)));
}
// a - c * b (c complex)
template <typename C>
__device__ __forceinline__ C cnaxpy(C c, C b, C a) {
  return cmk<C>(fma(-c.x, b.x, fma(c.y, b.y, a.x)), fma(-c.x, b.y, fma(-c.y, b.x, a.y)));
}
template <typename C>
__device__ __forceinline__ C mul_i(C a) { return cmk<C>(-a.y, a.x); }

// -x when neg, else x, by flipping the sign bit with an integer operation: a
// data-dependent choice between x and -x would otherwise cost a floating-point
// negation (an FP64 add, on the FP64 pipe, for doubles).
__device__ __forceinline__ double neg_if(double x, bool neg) {
  return __hiloint2double(__double2hiint(x) ^ (neg ? (int)0x80000000 : 0), __double2loint(x));
}
__device__ __forceinline__ float neg_if(float x, bool neg) {
  return __int_as_float(__float_as_int(x) ^ (neg ? (int)0x80000000 : 0));
}

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

// Shared-memory FFT buffers are padded with one element after every 8
// (complex128) or 16 (complex64) elements: the strided butterfly accesses of
// the late passes then spread over the banks instead of hitting a few.
template <typename C>
__device__ __forceinline__ int spad(int e) {
  return e + (e >> (sizeof(C) == 16 ? 3 : 4));
}
// Bytes of a padded buffer of `elems` complex values of `elem_bytes` each.
__host__ __device__ inline size_t padded_bytes(size_t elems, size_t elem_bytes) {
  const size_t e = elems + (elems >> (elem_bytes == 16 ? 3 : 4)) + 1;
  return ((e * elem_bytes) + 15) & ~size_t(15);
}
// Largest element count whose padded buffer fits in `bytes` (the inverse of
// padded_bytes, exact).
__host__ __device__ inline size_t padded_capacity(size_t bytes, size_t elem_bytes) {
  size_t e = (bytes / elem_bytes) * 8 / 9;
  while (e > 0 && padded_bytes(e, elem_bytes) > bytes) --e;
  while (padded_bytes(e + 1, elem_bytes) <= bytes) ++e;
  return e;
}

// ---------------------------------------------------------------------------
// Deterministic CTA-wide sums of K values per thread.  The xor-butterfly
// leaves bitwise identical sums in every lane; warps are then added in a
// fixed order.  Result in out[0..K) (shared), visible after return.
template <int K, typename R>
__device__ __forceinline__ void cta_sum(R (&v)[K], R* red, R* out) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[w * K + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    R s = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) s += red[ww * K + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// sum_i |x_i|^2 over len elements (plain sum, no grid weight)
template <typename C, typename R>
__device__ __forceinline__ R cta_norm2(const C* x, int len, R* red, R* out) {
  R v[1] = {0};
  for (int i = threadIdx.x; i < len; i += kThreads) {
    C a = x[i];
    v[0] = fma(a.x, a.x, fma(a.y, a.y, v[0]));
  }
  cta_sum<1>(v, red, out);
  return out[0];
}

// ---------------------------------------------------------------------------
// Small DFTs in registers.  Forward uses w = exp(-2 pi i / R), inverse its
// conjugate; no scaling.
template <bool INV, typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// The radix-4 DFT after its first level: a = x0 + x2, b = x0 - x2, c = x1 +
// x3, d = x1 - x3 given; outputs in x0..x3.
template <bool INV, typename C>
__device__ __forceinline__ void dft4_rest(C a, C b, C c, C d, C& x0, C& x1, C& x2, C& x3) {
  C id = mul_i(d);
  x0 = cadd(a, c);
  x2 = csub(a, c);
  if (!INV) {
    x1 = csub(b, id);
    x3 = cadd(b, id);
  } else {
    x1 = cadd(b, id);
    x3 = csub(b, id);
  }
}

template <bool INV, typename C>
__device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  dft4_rest<INV>(cadd(x0, x2), csub(x0, x2), cadd(x1, x3), csub(x1, x3), x0, x1, x2, x3);
}

// The radix-8 DFT after its first level: p[k] = x_k + x_{k+4}, q[k] = x_k -
// x_{k+4} (k < 4) given; outputs in x.
template <bool INV, typename C>
__device__ __forceinline__ void dft8_rest(const C (&p)[4], const C (&q)[4], C (&x)[8]) {
  using R = decltype(C::x);
  const R r2 = (R)0.70710678118654752440;
  C e0, e1, e2, e3, o0, o1, o2, o3;
  dft4_rest<INV>(p[0], q[0], p[2], q[2], e0, e1, e2, e3);   // even inputs
  dft4_rest<INV>(p[1], q[1], p[3], q[3], o0, o1, o2, o3);   // odd inputs
  // o1 and o3 times (+-1 +- i) / sqrt2: the sums and differences of their
  // parts, the 1/sqrt2 folded into the fused multiply-adds below
  C t1, t2, t3;
  if (!INV) {
    t1 = cmk<C>(o1.x + o1.y, o1.y - o1.x);     // (1 - i) o1
    t2 = cmk<C>(o2.y, -o2.x);                  // -i o2
    t3 = cmk<C>(o3.y - o3.x, -(o3.x + o3.y));  // (-1 - i) o3
  } else {
    t1 = cmk<C>(o1.x - o1.y, o1.x + o1.y);     // (1 + i) o1
    t2 = cmk<C>(-o2.y, o2.x);                  // i o2
    t3 = cmk<C>(-(o3.x + o3.y), o3.x - o3.y);  // (-1 + i) o3
  }
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  x[1] = caxpy_r(r2, t1, e1);
  x[5] = caxpy_r(-r2, t1, e1);
  x[2] = cadd(e2, t2);
  x[6] = csub(e2, t2);
  x[3] = caxpy_r(r2, t3, e3);
  x[7] = caxpy_r(-r2, t3, e3);
}

template <bool INV, typename C>
__device__ __forceinline__ void dft8(C (&x)[8]) {
  C p[4], q[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    p[k] = cadd(x[k], x[k + 4]);
    q[k] = csub(x[k], x[k + 4]);
  }
  dft8_rest<INV>(p, q, x);
}

template <int RD, bool INV, typename C>
__device__ __forceinline__ void dft(C (&x)[RD]) {
  if constexpr (RD == 2) {
    dft2<INV>(x[0], x[1]);
  } else if constexpr (RD == 4) {
    dft4<INV>(x[0], x[1], x[2], x[3]);
  } else {
    dft8<INV>(x);
  }
}

// Operands of one H psi evaluation in one precision.  The transform of
// length n = 2^k runs n8 radix-8 passes and then npass - n8 radix-4 passes
// (decimation in frequency; the inverse runs them backwards).
template <typename R>
struct HOp {
  using C = typename Cx<R>::T;
  int n, S, npass, n8;
  R h2m;
  const C* tw;   // twiddles, pass by pass (see fft_pass)
  const R* kd;   // k at digit-reversed positions, divided by n
  const R* V;
  const R* F;
  C* U;          // scratch vector (S * n)
  int diab;      // 1: the diabatic representation, H = -hbar^2/2m D^2 + W, with
                 // V = diag W and F = the upper triangle of W (symmetric)
  // FP64 only: Linzer-Feig factor tables (entries, form words; see
  // lf_derivative), or null -- the transform then runs the passes of
  // fft_pass with the twiddles tw
  const double2* lf = nullptr;
  const unsigned* lff = nullptr;
};

// Number of leading radix-8 passes of a plan.
__host__ __device__ inline int count_radix8(const int* radix, int npass) {
  int k = 0;
  while (k < npass && radix[k] == 8) ++k;
  return k;
}

// One radix-RD pass over nb vectors of length n in shared memory, in place.
// Block length L, m = L / RD.  Forward (decimation in frequency): DFT over the
// RD elements j + r m of a block, then multiply by w_L^{j r}.  Inverse
// (decimation in time): multiply by conj(w_L^{j r}), then inverse DFT; it
// undoes the forward pass up to a factor RD.  twp is this pass's segment of
// the twiddle table: twp[(r - 1) m + j] = w_L^{j r}, so consecutive j (the
// lanes of a warp) read consecutive entries.  The tables are read with
// generic loads: they may sit in global or in shared memory.
// src (optional): read the pass's input from src (nb unpadded vectors of
// length n, global or shared memory) instead of buf -- the first forward pass
// then also does the copy into shared memory.
template <int RD, bool INV, typename C>
__device__ __forceinline__ void fft_pass(C* gbuf, int n, int nb, int L, const C* __restrict__ twp,
                                         const C* src = nullptr) {
  C* buf = in_dyn_smem(gbuf);
  const int lm = ilog2(L / RD);
  const int m = 1 << lm;
  const int lpv = ilog2(n / RD);
  const int total = nb << lpv;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int v = b >> lpv;
    const int bb = b & ((n / RD) - 1);
    const int blk = bb >> lm;
    const int j = bb & (m - 1);
    const int e0 = v * n + blk * L + j;
    C x[RD];
    if (src) {
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = src[e0 + r * m];
    } else {
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = buf[spad<C>(e0 + r * m)];
    }
    if (!INV) {
      dft<RD, false>(x);
      if (j) {
#pragma unroll
        for (int r = 1; r < RD; ++r) x[r] = cmul(x[r], twp[(r - 1) * m + j]);
      }
    } else {
      if (j) {
#pragma unroll
        for (int r = 1; r < RD; ++r) x[r] = cmulc(x[r], twp[(r - 1) * m + j]);
      }
      dft<RD, true>(x);
    }
#pragma unroll
    for (int r = 0; r < RD; ++r) buf[spad<C>(e0 + r * m)] = x[r];
  }
}

// Last forward pass (block length RD, no twiddles), multiplication by i k / n
// (or, second = 1, by (i k)^2 / n = -n (k/n)^2) at the digit-reversed
// positions, first inverse pass -- all in registers.
template <int RD, typename C, typename R>
__device__ __forceinline__ void fft_center(C* gbuf, int n, int nb, const R* __restrict__ kd, int second = 0) {
  C* buf = in_dyn_smem(gbuf);
  const int total = (nb * n) / RD;
  const R mn = -(R)n;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int e0 = b * RD;
    const int pos = e0 & (n - 1);
    C x[RD];
#pragma unroll
    for (int r = 0; r < RD; ++r) x[r] = buf[spad<C>(e0 + r)];
    dft<RD, false>(x);
    if (second) {
#pragma unroll
      for (int r = 0; r < RD; ++r) {
        const R k = kd[pos + r];
        x[r] = cscale(mn * k * k, x[r]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < RD; ++r) {
        const R k = kd[pos + r];
        x[r] = cmk<C>(-k * x[r].y, k * x[r].x);
      }
    }
    dft<RD, true>(x);
#pragma unroll
    for (int r = 0; r < RD; ++r) buf[spad<C>(e0 + r)] = x[r];
  }
}

// ---------------------------------------------------------------------------
// FP64 transform in Linzer and Feig's fused multiply-add form.  A twiddle
// factored as w = s (1 + i t) (form 0, |Re w| >= |Im w|) or w = s (t + i)
// (form 1), |t| <= 1, turns the radix-2 step (a, b) -> (a + w b, a - w b)
// into six fused multiply-adds: u = b (1 + i t) or b (t + i) in two, then a
// +- s u in four.  A radix-R step with input twiddles W^r (r = 0..R-1) is
// log2 R levels of such steps whose factors are W^(R/2), W^(R/4), ..., and
// their products with the R-th roots of unity; a product with -i (forward) or
// +i (inverse) changes only the form, the sign of t and the roles of the
// parts of s, so a radix-8 set stores W^4, W^2, W and zeta W, a radix-4 set
// W^2 and W.  The forward transform is the decimation-in-frequency sequence
// of fft_pass with each pass's twiddles moved to the input of the next pass:
// block blk of pass i then multiplies its inputs by W^r with W a root of
// unity of order (blocks x radix), indexed by the frequency the block has
// accumulated (the first pass has none).  The inverse is the
// decimation-in-time sequence, whose twiddles already sit at the input.
// Outputs of a step leave in bit-reversed register order.

// One factor: x and y multipliers of the a +- s u update (sx = -s for form
// 1, whose u is computed with its real part negated), t and the form.
struct LfW {
  double sx, sy, t;
  bool f;
};

__device__ __forceinline__ LfW lf_w(double2 st, bool f) { return LfW{neg_if(st.x, f), st.x, st.y, f}; }

// The factor of -i w (forward) or +i w (inverse).
template <bool INV>
__device__ __forceinline__ LfW lf_rot(const LfW& w) {
  return INV ? LfW{-w.sy, w.sx, -w.t, !w.f} : LfW{w.sy, -w.sx, -w.t, !w.f};
}

// (a, b) <- (a + w b, a - w b).
__device__ __forceinline__ void lf2(double2& a, double2& b, const LfW& w) {
  const double p = w.f ? b.y : b.x;
  const double q = w.f ? b.x : b.y;
  const double ux = fma(-w.t, q, p);   // form 0: Re b (1 + i t); form 1: -Re b (t + i)
  const double uy = fma(w.t, p, q);    // Im of the same product
  const double2 a0 = a;
  a = make_double2(fma(w.sx, ux, a0.x), fma(w.sy, uy, a0.y));
  b = make_double2(fma(-w.sx, ux, a0.x), fma(-w.sy, uy, a0.y));
}

// Radix-RD DFT of x_r W^r (forward) or its inverse counterpart, w[] the
// stored factors (W^4, W^2, W, zeta W or W^2, W); x[s] receives output
// bitrev(s).
template <int RD, bool INV>
__device__ __forceinline__ void lf_bfly(double2 (&x)[RD], const LfW (&w)[RD == 8 ? 4 : 2]) {
  if constexpr (RD == 8) {
#pragma unroll
    for (int r = 0; r < 4; ++r) lf2(x[r], x[r + 4], w[0]);
    const LfW w2r = lf_rot<INV>(w[1]);
    lf2(x[0], x[2], w[1]);
    lf2(x[1], x[3], w[1]);
    lf2(x[4], x[6], w2r);
    lf2(x[5], x[7], w2r);
    lf2(x[0], x[1], w[2]);
    lf2(x[2], x[3], lf_rot<INV>(w[2]));
    lf2(x[4], x[5], w[3]);
    lf2(x[6], x[7], lf_rot<INV>(w[3]));
  } else {
    lf2(x[0], x[2], w[0]);
    lf2(x[1], x[3], w[0]);
    lf2(x[0], x[1], w[1]);
    lf2(x[2], x[3], lf_rot<INV>(w[1]));
  }
}

template <int RD>
__device__ __forceinline__ int bitrev(int s) {
  return RD == 8 ? ((s & 1) << 2) | (s & 2) | (s >> 2) : ((s & 1) << 1) | (s >> 1);
}

// Set k of a pass with nsets sets (entries e * nsets + k, form word k).
template <int RD>
__device__ __forceinline__ void lf_load(const double2* __restrict__ ent, const unsigned* __restrict__ flg, int nsets,
                                        int k, LfW (&w)[RD == 8 ? 4 : 2]) {
  const unsigned fl = flg[k];
#pragma unroll
  for (int e = 0; e < (RD == 8 ? 4 : 2); ++e) w[e] = lf_w(ent[e * nsets + k], (fl >> e) & 1u);
}

// One radix-RD pass over nb vectors in shared memory, the element layout of
// fft_pass (block length L, m = L / RD, elements j + r m of a block).  TW =
// false: the untwiddled first forward pass (plain DFT; src as in fft_pass);
// TW = true: the factored step with set blk (forward) or j (inverse) of the
// pass's tables.
template <int RD, bool INV, bool TW>
__device__ __forceinline__ void lf_pass(double2* gbuf, int n, int nb, int L, const double2* __restrict__ ent,
                                        const unsigned* __restrict__ flg, const double2* src = nullptr) {
  double2* buf = in_dyn_smem(gbuf);
  const int lm = ilog2(L / RD);
  const int m = 1 << lm;
  const int lpv = ilog2(n / RD);
  const int total = nb << lpv;
  const int nsets = INV ? m : n / L;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int v = b >> lpv;
    const int bb = b & ((n / RD) - 1);
    const int blk = bb >> lm;
    const int j = bb & (m - 1);
    const int e0 = v * n + blk * L + j;
    double2 x[RD];
    if (src) {
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = src[e0 + r * m];
    } else {
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = buf[spad<double2>(e0 + r * m)];
    }
    if constexpr (!TW) {
      dft<RD, INV>(x);
#pragma unroll
      for (int r = 0; r < RD; ++r) buf[spad<double2>(e0 + r * m)] = x[r];
    } else {
      LfW w[RD == 8 ? 4 : 2];
      lf_load<RD>(ent, flg, nsets, INV ? j : blk, w);
      lf_bfly<RD, INV>(x, w);
#pragma unroll
      for (int s = 0; s < RD; ++s) buf[spad<double2>(e0 + bitrev<RD>(s) * m)] = x[s];
    }
  }
}

// Last forward pass (block length RD; factored with set blk when TW), times
// i k / n (second: -n (k/n)^2), first inverse pass (untwiddled) -- in
// registers, as fft_center.
template <int RD, bool TW, bool SECOND>
__device__ __forceinline__ void lf_center(double2* gbuf, int n, int nb, const double* __restrict__ kd,
                                          const double2* __restrict__ ent, const unsigned* __restrict__ flg) {
  double2* buf = in_dyn_smem(gbuf);
  const int total = (nb * n) / RD;
  const double mn = -(double)n;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int e0 = b * RD;
    const int pos = e0 & (n - 1);
    double2 x[RD], y[RD];
#pragma unroll
    for (int r = 0; r < RD; ++r) x[r] = buf[spad<double2>(e0 + r)];
    if constexpr (TW) {
      LfW w[RD == 8 ? 4 : 2];
      lf_load<RD>(ent, flg, n / RD, pos / RD, w);
      lf_bfly<RD, false>(x, w);
#pragma unroll
      for (int k = 0; k < RD; ++k) y[k] = x[bitrev<RD>(k)];
    } else {
      dft<RD, false>(x);
#pragma unroll
      for (int k = 0; k < RD; ++k) y[k] = x[k];
    }
    // the spectral multiplier w_k (i k / n, or -n (k/n)^2) fused into the
    // first level of the inverse DFT: w_k y_k +- w_{k+h} y_{k+h}, h = RD / 2,
    // as one multiply and two fused multiply-adds per part
    constexpr int h = RD / 2;
    double2 p[h], q[h];
#pragma unroll
    for (int k = 0; k < h; ++k) {
      double w0 = kd[pos + k], w1 = kd[pos + k + h];
      if (SECOND) {
        w0 *= mn * w0;
        w1 *= mn * w1;
      }
      const double2 t = make_double2(w0 * y[k].x, w0 * y[k].y);
      const double2 sp = caxpy_r(w1, y[k + h], t), sm = caxpy_r(-w1, y[k + h], t);
      p[k] = SECOND ? sp : mul_i(sp);   // i k: times i
      q[k] = SECOND ? sm : mul_i(sm);
    }
    if constexpr (RD == 8) {
      dft8_rest<true>(p, q, y);
    } else {
      dft4_rest<true>(p[0], q[0], p[1], q[1], y[0], y[1], y[2], y[3]);
    }
#pragma unroll
    for (int r = 0; r < RD; ++r) buf[spad<double2>(e0 + r)] = y[r];
  }
}

// spectral_derivative's FP64 transform with the factored passes; the tables
// run forward passes 1..np-1, then inverse passes np-2..0 (lf_tables).
__device__ __forceinline__ void lf_derivative(double2* buf, int nb, const HOp<double>& H, const double2* src,
                                              int second) {
  const int n = H.n, np = H.npass, n8 = H.n8;
  const double* kd = H.kd;
  const double2* ent = H.lf;
  const unsigned* flg = H.lff;
  int L = n;
  for (int i = 0; i < np - 1; ++i) {
    const int RD = i < n8 ? 8 : 4;
    if (i == 0) {
      if (RD == 8)
        lf_pass<8, false, false>(buf, n, nb, L, nullptr, nullptr, src);
      else
        lf_pass<4, false, false>(buf, n, nb, L, nullptr, nullptr, src);
    } else {
      if (RD == 8)
        lf_pass<8, false, true>(buf, n, nb, L, ent, flg);
      else
        lf_pass<4, false, true>(buf, n, nb, L, ent, flg);
      ent += (RD == 8 ? 4 : 2) * (n / L);
      flg += n / L;
    }
    L /= RD;
    __syncthreads();
  }
  if (np - 1 < n8) {
    if (second)
      lf_center<8, true, true>(buf, n, nb, kd, ent, flg);
    else
      lf_center<8, true, false>(buf, n, nb, kd, ent, flg);
  } else {
    if (second)
      lf_center<4, true, true>(buf, n, nb, kd, ent, flg);
    else
      lf_center<4, true, false>(buf, n, nb, kd, ent, flg);
  }
  ent += (L == 8 ? 4 : 2) * (n / L);
  flg += n / L;
  __syncthreads();
  for (int i = np - 2; i >= 0; --i) {
    const int RD = i < n8 ? 8 : 4;
    L *= RD;
    if (RD == 8)
      lf_pass<8, true, true>(buf, n, nb, L, ent, flg);
    else
      lf_pass<4, true, true>(buf, n, nb, L, ent, flg);
    ent += (RD == 8 ? 4 : 2) * (L / RD);
    flg += L / RD;
    __syncthreads();
  }
}

// buf <- D buf for nb vectors (spectral first derivative, Sec. II D):
// forward FFT, multiply by i k, inverse FFT (1/n folded into kd).
// One out-of-line copy per precision: its call sites share the code (fewer
// instruction-cache misses than an inlined copy at every site).
// src (optional): take the input from src (nb unpadded vectors) instead of
// buf; the first forward pass reads it.
// second = 1: the second derivative D^2 instead (same transforms).
template <typename R>
__device__ __noinline__ void spectral_derivative(typename Cx<R>::T* buf, int nb, const HOp<R>& H,
                                                 const typename Cx<R>::T* src = nullptr, int second = 0) {
  using C = typename Cx<R>::T;
  const int n = H.n, np = H.npass, n8 = H.n8;
  const C* tw = H.tw;
  const R* kd = H.kd;
  if constexpr (sizeof(R) == 8) {
    if (H.lf && np >= 2) {
      lf_derivative(buf, nb, H, src, second);
      return;
    }
  }
  if (src && np == 1) {   // no twiddled pass to fuse the copy into
    C* sb = in_dyn_smem(buf);
    for (int i = threadIdx.x; i < nb * n; i += kThreads) sb[spad<C>(i)] = src[i];
    __syncthreads();
    src = nullptr;
  }
  int L = n, off = 0;
  for (int i = 0; i < np - 1; ++i) {
    const int RD = i < n8 ? 8 : 4;
    const C* in = i == 0 ? src : nullptr;
    if (RD == 8)
      fft_pass<8, false>(buf, n, nb, L, tw + off, in);
    else
      fft_pass<4, false>(buf, n, nb, L, tw + off, in);
    off += (RD - 1) * (L / RD);
    L /= RD;
    __syncthreads();
  }
  if (np - 1 < n8)
    fft_center<8>(buf, n, nb, kd, second);
  else
    fft_center<4>(buf, n, nb, kd, second);
  __syncthreads();
  for (int i = np - 2; i >= 0; --i) {
    const int RD = i < n8 ? 8 : 4;
    L *= RD;
    off -= (RD - 1) * (L / RD);
    if (RD == 8)
      fft_pass<8, true>(buf, n, nb, L, tw + off);
    else
      fft_pass<4, true>(buf, n, nb, L, tw + off);
    __syncthreads();
  }
}

// Elements per thread in flight in the pointwise passes of H psi.
constexpr int kHpsiUnroll = 1;

// Coupling F_{st}(q_j) from the stored upper triangle (S(S-1)/2 rows of n).
template <typename R>
__device__ __forceinline__ R coupling(const R* __restrict__ F, int n, int S, int s, int t, int j) {
  const int a = s < t ? s : t, b = s < t ? t : s;
  const int p = a * S - (a * (a + 1)) / 2 + (b - a - 1);
  return neg_if(__ldg(F + (size_t)p * n + j), s > t);   // F_ts = -F_st
}

// Diabatic coupling W_st (s != t) from the stored upper triangle (symmetric).
template <typename R>
__device__ __forceinline__ R wcoupling(const R* __restrict__ F, int n, int S, int s, int t, int j) {
  const int a = s < t ? s : t, b = s < t ? t : s;
  const int p = a * S - (a * (a + 1)) / 2 + (b - a - 1);
  return __ldg(F + (size_t)p * n + j);
}

// y = e z + a x + c (H x) in the diabatic representation (Sec. II E):
// H = -hbar^2/(2m) D^2 1 + W(q), two transforms per surface and the
// pointwise symmetric W.  DOTS (bit 0, bit 1): also Re<x, y>, ||y||^2 (raw sums) in
// dots[0..1].  y may alias x or z.
template <typename R, int DOTS>
__device__ __noinline__ void apply_h_diabatic(const HOp<R>& H, typename Cx<R>::T* sbuf, int nb_cap,
                                                 const typename Cx<R>::T* x, typename Cx<R>::T* y,
                                                 const typename Cx<R>::T* z, R e, R a, typename Cx<R>::T c, R* red,
                                                 R* dots) {
  using C = typename Cx<R>::T;
  const int n = H.n, S = H.S;
  const int ln = ilog2(n);
  const R* F = H.F;
  const R* V = H.V;
  const R mh = -H.h2m;
  const int nb = (S <= nb_cap) ? S : 1;
  C* sb = in_dyn_smem(sbuf);
  R d[2] = {(R)0, (R)0};
  // the coupling reads x at other surfaces' points, so results go straight
  // to y only when all surfaces form one batch and y does not alias x; else
  // H x is formed in U first and combined in a last pass
  const bool whole = nb == S && (const void*)y != (const void*)x;
  for (int s0 = 0; s0 < S; s0 += nb) {
    spectral_derivative<R>(sbuf, nb, H, x + (size_t)s0 * n, 1);
    for (int i = threadIdx.x; i < nb * n; i += kThreads) {
      const int s = s0 + (i >> ln), j = i & (n - 1);
      const C xs = x[s * n + j];
      const R v = __ldg(V + s * n + j);
      C acc = cmk<C>(fma(mh, sb[spad<C>(i)].x, v * xs.x), fma(mh, sb[spad<C>(i)].y, v * xs.y));
      for (int t = 0; t < S; ++t)
        if (t != s) acc = caxpy_r(wcoupling(F, n, S, s, t, j), x[t * n + j], acc);
      if (whole) {
        C out = caxpy(c, acc, cmk<C>(a * xs.x, a * xs.y));
        if (e != (R)0) out = caxpy_r(e, z[s * n + j], out);
        y[s * n + j] = out;
        if (DOTS & 1) d[0] = fma(xs.x, out.x, fma(xs.y, out.y, d[0]));
        if (DOTS & 2) d[1] = fma(out.x, out.x, fma(out.y, out.y, d[1]));
      } else {
        H.U[s * n + j] = acc;
      }
    }
    __syncthreads();
  }
  if (!whole) {
    for (int i = threadIdx.x; i < S * n; i += kThreads) {
      const C xs = x[i];
      C out = caxpy(c, H.U[i], cmk<C>(a * xs.x, a * xs.y));
      if (e != (R)0) out = caxpy_r(e, z[i], out);
      y[i] = out;
      if (DOTS & 1) d[0] = fma(xs.x, out.x, fma(xs.y, out.y, d[0]));
      if (DOTS & 2) d[1] = fma(out.x, out.x, fma(out.y, out.y, d[1]));
    }
    __syncthreads();
  }
  if (DOTS) cta_sum<2>(d, red, dots);
}

// y = e z + a x + c (H x), H of Eq. (adiab_mol_ham) by the dynamic Fourier
// method.  With A = p - i hbar F = -i hbar (D + F), the Hamiltonian equals
// -hbar^2/(2m) (D + F)^2 + V exactly (F real antisymmetric, D the spectral
// derivative), so H x is two applications of (D + F): each a forward FFT,
// a multiplication by i k and an inverse FFT per surface, plus the pointwise
// coupling -- 4 transforms per surface, as counted in Table I.
// sbuf holds nb_cap vectors of length n; H.U is scratch.  y may alias x or z.
// z may be null when e == 0.
template <typename R>
__device__ __noinline__ void apply_h_axpby(const HOp<R>& H, typename Cx<R>::T* sbuf, int nb_cap,
                                              const typename Cx<R>::T* x, typename Cx<R>::T* y,
                                              const typename Cx<R>::T* z, R e, R a, typename Cx<R>::T c) {
  using C = typename Cx<R>::T;
  if (H.diab) {
    apply_h_diabatic<R, false>(H, sbuf, nb_cap, x, y, z, e, a, c, nullptr, nullptr);
    return;
  }
  const int n = H.n, S = H.S;
  const int ln = ilog2(n);
  C* U = H.U;
  const R* F = H.F;
  const R* V = H.V;
  const int nb = (S <= nb_cap) ? S : 1;
  sbuf = in_dyn_smem(sbuf);
  // U = (D + F) x
  for (int s0 = 0; s0 < S; s0 += nb) {
    for (int i = threadIdx.x; i < nb * n; i += kThreads) sbuf[spad<C>(i)] = x[s0 * n + i];
    __syncthreads();
    spectral_derivative<R>(sbuf, nb, H);
    for (int i = threadIdx.x; i < nb * n; i += kThreads) {
      const int s = s0 + (i >> ln), j = i & (n - 1);
      C acc = sbuf[spad<C>(i)];
      for (int t = 0; t < S; ++t)
        if (t != s) acc = caxpy_r(coupling(F, n, S, s, t, j), x[t * n + j], acc);
      U[s * n + j] = acc;
    }
    __syncthreads();
  }
  // y = e z + a x + c (-hbar^2/2m (D + F) U + V x)
  const R mh = -H.h2m;
  for (int s0 = 0; s0 < S; s0 += nb) {
    for (int i = threadIdx.x; i < nb * n; i += kThreads) sbuf[spad<C>(i)] = U[s0 * n + i];
    __syncthreads();
    spectral_derivative<R>(sbuf, nb, H);
    for (int i = threadIdx.x; i < nb * n; i += kThreads) {
      const int s = s0 + (i >> ln), j = i & (n - 1);
      C acc = sbuf[spad<C>(i)];
      for (int t = 0; t < S; ++t)
        if (t != s) acc = caxpy_r(coupling(F, n, S, s, t, j), U[t * n + j], acc);
      const C xs = x[s * n + j];
      const R v = __ldg(V + s * n + j);
      const C hx = cmk<C>(fma(mh, acc.x, v * xs.x), fma(mh, acc.y, v * xs.y));
      C out = caxpy(c, hx, cmk<C>(a * xs.x, a * xs.y));
      if (e != (R)0) out = caxpy_r(e, z[s * n + j], out);
      y[s * n + j] = out;
    }
    __syncthreads();
  }
}

// The same H psi with U = (D + F) x kept in shared memory (sU, S n values)
// and fewer passes: the first forward pass of each derivative reads its
// input directly (x from global memory, U from sU), and when all surfaces fit
// in one FFT batch the coupling pass leaves U in the FFT buffer for the second
// derivative.  DOTS (bit 0, bit 1): also the raw sums Re<x, y>, ||y||^2 in
// dots[0..1] (one CTA reduction).  y may alias x or z.
template <typename R, int DOTS>
__device__ __noinline__ void apply_h_staged(const HOp<R>& H, typename Cx<R>::T* sbuf, int nb_cap,
                                               typename Cx<R>::T* sU, const typename Cx<R>::T* x,
                                               typename Cx<R>::T* y, const typename Cx<R>::T* z, R e, R a,
                                               typename Cx<R>::T c, R* red, R* dots) {
  using C = typename Cx<R>::T;
  if (H.diab) {
    apply_h_diabatic<R, DOTS>(H, sbuf, nb_cap, x, y, z, e, a, c, red, dots);
    return;
  }
  const int n = H.n, S = H.S;
  const int ln = ilog2(n);
  const R* F = H.F;
  const R* V = H.V;
  const int nb = (S <= nb_cap) ? S : 1;
  const bool whole = nb == S;
  C* sb = in_dyn_smem(sbuf);
  C* su = in_dyn_smem(sU);
  const int tot = nb * n;
  constexpr int U = kHpsiUnroll;
  // (D + F) of the batch's points: the FFT result plus the coupling to the
  // other surfaces' w (S = 2: +-F_01 w_other)
  auto plus_fw = [&](int s, int j, C acc, const C* w) {
    if (S == 2) return caxpy_r(neg_if(__ldg(F + j), s != 0), w[(1 - s) * n + j], acc);
    for (int t = 0; t < S; ++t)
      if (t != s) acc = caxpy_r(coupling(F, n, S, s, t, j), w[t * n + j], acc);
    return acc;
  };
  // U = (D + F) x; U elements per thread formed before any is stored
  for (int s0 = 0; s0 < S; s0 += nb) {
    spectral_derivative<R>(sbuf, nb, H, x + (size_t)s0 * n);
    for (int i0 = threadIdx.x; i0 < tot; i0 += U * kThreads) {
      C acc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * kThreads;
        if (i < tot) acc[u] = plus_fw(s0 + (i >> ln), i & (n - 1), sb[spad<C>(i)], x);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * kThreads;
        if (i < tot) {
          su[s0 * n + i] = acc[u];
          if (whole) sb[spad<C>(i)] = acc[u];
        }
      }
    }
    __syncthreads();
  }
  // y = e z + a x + c (-hbar^2/2m (D + F) U + V x); the Lanczos iteration
  // (a = 0, c = 1) skips the scalings.  The operands of U elements per
  // thread are loaded before any result is stored (y may alias x or z, but
  // element by element only).
  const R mh = -H.h2m;
  const bool plain = a == (R)0 && c.x == (R)1 && c.y == (R)0;
  R d[2] = {(R)0, (R)0};
  for (int s0 = 0; s0 < S; s0 += nb) {
    spectral_derivative<R>(sbuf, nb, H, whole ? nullptr : su + (size_t)s0 * n);
    const C* xb = x + (size_t)s0 * n;
    const C* zb = z + (size_t)s0 * n;
    const R* Vb = V + (size_t)s0 * n;
    for (int i0 = threadIdx.x; i0 < tot; i0 += U * kThreads) {
      C acc[U], xs[U], zz[U];
      R v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * kThreads;
        if (i < tot) {
          acc[u] = plus_fw(s0 + (i >> ln), i & (n - 1), sb[spad<C>(i)], su);
          xs[u] = xb[i];
          v[u] = __ldg(Vb + i);
          zz[u] = e != (R)0 ? zb[i] : cmk<C>((R)0, (R)0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * kThreads;
        if (i < tot) {
          const C hx = cmk<C>(fma(mh, acc[u].x, v[u] * xs[u].x), fma(mh, acc[u].y, v[u] * xs[u].y));
          C out = plain ? hx : caxpy(c, hx, cmk<C>(a * xs[u].x, a * xs[u].y));
          if (e != (R)0) out = caxpy_r(e, zz[u], out);
          y[s0 * n + i] = out;
          if (DOTS & 1) d[0] = fma(xs[u].x, out.x, fma(xs[u].y, out.y, d[0]));
          if (DOTS & 2) d[1] = fma(out.x, out.x, fma(out.y, out.y, d[1]));
        }
      }
    }
    __syncthreads();
  }
  if (DOTS) cta_sum<2>(d, red, dots);
}

// y = (D + F) x (one half of H psi; used by the adjoint to form the field
// gradients).  y must not alias x.
template <typename R>
__device__ __forceinline__ void apply_d_plus_f(const HOp<R>& H, typename Cx<R>::T* sbuf, int nb_cap,
                                               const typename Cx<R>::T* x, typename Cx<R>::T* y) {
  using C = typename Cx<R>::T;
  const int n = H.n, S = H.S;
  const int ln = ilog2(n);
  const R* F = H.F;
  const int nb = (S <= nb_cap) ? S : 1;
  sbuf = in_dyn_smem(sbuf);
  for (int s0 = 0; s0 < S; s0 += nb) {
    for (int i = threadIdx.x; i < nb * n; i += kThreads) sbuf[spad<C>(i)] = x[s0 * n + i];
    __syncthreads();
    spectral_derivative<R>(sbuf, nb, H);
    for (int i = threadIdx.x; i < nb * n; i += kThreads) {
      const int s = s0 + (i >> ln), j = i & (n - 1);
      C acc = sbuf[spad<C>(i)];
      for (int t = 0; t < S; ++t)
        if (t != s) acc = caxpy_r(coupling(F, n, S, s, t, j), x[t * n + j], acc);
      y[s * n + j] = acc;
    }
    __syncthreads();
  }
}

}  // namespace qg
