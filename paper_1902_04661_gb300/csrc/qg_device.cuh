// Device building blocks: complex arithmetic, deterministic CTA reductions,
// the shared-memory FFT and the fused Hamiltonian action (Sec. II D-E).
//
// Every CTA works on one instance.  All loops are bounded; nothing waits on
// another CTA.
#pragma once

#include "qg_internal.h"

namespace qg {

constexpr int kThreads = QG_THREADS;
constexpr int kWarps = QG_THREADS / 32;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// a * b
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
// a + s * b (s real)
__device__ __forceinline__ double2 caxpy_r(double s, double2 b, double2 a) {
  return make_double2(fma(s, b.x, a.x), fma(s, b.y, a.y));
}
// a + c * b (c complex)
__device__ __forceinline__ double2 caxpy(double2 c, double2 b, double2 a) {
  return make_double2(fma(c.x, b.x, fma(-c.y, b.y, a.x)), fma(c.x, b.y, fma(c.y, b.x, a.y)));
}
// a - c * b (c complex)
__device__ __forceinline__ double2 cnaxpy(double2 c, double2 b, double2 a) {
  return make_double2(fma(-c.x, b.x, fma(c.y, b.y, a.x)), fma(-c.x, b.y, fma(-c.y, b.x, a.y)));
}
__device__ __forceinline__ double2 mul_i(double2 a) { return make_double2(-a.y, a.x); }

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

// ---------------------------------------------------------------------------
// Deterministic CTA-wide sums of K doubles per thread.  The xor-butterfly
// leaves bitwise identical sums in every lane; warps are then added in a
// fixed order.  Result in out[0..K) (shared), visible after return.
template <int K>
__device__ __forceinline__ void cta_sum(double (&v)[K], double* red, double* out) {
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
    double s = 0.0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) s += red[ww * K + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// sum_i |x_i|^2 over len elements (plain sum, no grid weight)
__device__ __forceinline__ double cta_norm2(const double2* x, int len, double* red, double* out) {
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < len; i += kThreads) {
    double2 a = x[i];
    v[0] = fma(a.x, a.x, fma(a.y, a.y, v[0]));
  }
  cta_sum<1>(v, red, out);
  return out[0];
}

// ---------------------------------------------------------------------------
// Small DFTs in registers.  Forward uses w = exp(-2 pi i / R), inverse its
// conjugate; no scaling.
template <bool INV>
__device__ __forceinline__ void dft2(double2& a, double2& b) {
  double2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(double2& x0, double2& x1, double2& x2, double2& x3) {
  double2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = csub(x1, x3);
  double2 id = mul_i(d);
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

template <bool INV>
__device__ __forceinline__ void dft8(double2 (&x)[8]) {
  const double r2 = 0.70710678118654752440;
  double2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  double2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  double2 t1, t2, t3;
  if (!INV) {
    t1 = make_double2((o1.x + o1.y) * r2, (o1.y - o1.x) * r2);     // (1 - i)/sqrt2
    t2 = make_double2(o2.y, -o2.x);                                 // -i
    t3 = make_double2((o3.y - o3.x) * r2, -(o3.x + o3.y) * r2);    // (-1 - i)/sqrt2
  } else {
    t1 = make_double2((o1.x - o1.y) * r2, (o1.x + o1.y) * r2);     // (1 + i)/sqrt2
    t2 = make_double2(-o2.y, o2.x);                                 // i
    t3 = make_double2(-(o3.x + o3.y) * r2, (o3.x - o3.y) * r2);    // (-1 + i)/sqrt2
  }
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  x[1] = cadd(e1, t1);
  x[5] = csub(e1, t1);
  x[2] = cadd(e2, t2);
  x[6] = csub(e2, t2);
  x[3] = cadd(e3, t3);
  x[7] = csub(e3, t3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(double2 (&x)[R]) {
  if constexpr (R == 2) {
    dft2<INV>(x[0], x[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(x[0], x[1], x[2], x[3]);
  } else {
    dft8<INV>(x);
  }
}

// One radix-R pass over nb vectors of length n in shared memory, in place.
// Block length L, m = L / R.  Forward (decimation in frequency): DFT over the
// R elements j + r m of a block, then multiply by w_L^{j r}.  Inverse
// (decimation in time): multiply by conj(w_L^{j r}), then inverse DFT; it
// undoes the forward pass up to a factor R.  w_L^{j r} = tw[j r n / L],
// an index below n.
template <int R, bool INV>
__device__ __forceinline__ void fft_pass(double2* buf, int n, int nb, int L, const double2* __restrict__ tw) {
  const int lm = ilog2(L / R);
  const int m = 1 << lm;
  const int lpv = ilog2(n / R);
  const int total = nb << lpv;
  const int tshift = ilog2(n / L);
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int v = b >> lpv;
    const int bb = b & ((n / R) - 1);
    const int blk = bb >> lm;
    const int j = bb & (m - 1);
    double2* p = buf + v * n + blk * L + j;
    double2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = p[r * m];
    if (!INV) {
      dft<R, false>(x);
      if (j) {
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmul(x[r], __ldg(tw + ((j * r) << tshift)));
      }
    } else {
      if (j) {
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmulc(x[r], __ldg(tw + ((j * r) << tshift)));
      }
      dft<R, true>(x);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) p[r * m] = x[r];
  }
}

// Last forward pass (block length R, no twiddles), multiplication by i k / n
// at the digit-reversed positions, first inverse pass -- all in registers.
template <int R>
__device__ __forceinline__ void fft_center(double2* buf, int n, int nb, const double* __restrict__ kd) {
  const int total = (nb * n) / R;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    double2* p = buf + b * R;
    const int pos = (b * R) & (n - 1);
    double2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = p[r];
    dft<R, false>(x);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double k = __ldg(kd + pos + r);
      x[r] = make_double2(-k * x[r].y, k * x[r].x);
    }
    dft<R, true>(x);
#pragma unroll
    for (int r = 0; r < R; ++r) p[r] = x[r];
  }
}

template <bool INV>
__device__ __forceinline__ void fft_pass_dispatch(int R, double2* buf, int n, int nb, int L, const double2* tw) {
  if (R == 8)
    fft_pass<8, INV>(buf, n, nb, L, tw);
  else if (R == 4)
    fft_pass<4, INV>(buf, n, nb, L, tw);
  else
    fft_pass<2, INV>(buf, n, nb, L, tw);
}

// buf <- D buf for nb vectors (spectral first derivative, Sec. II D):
// forward FFT, multiply by i k, inverse FFT (1/n folded into kd).
__device__ __forceinline__ void spectral_derivative(double2* buf, int nb, const InstDesc& I) {
  const int n = I.n;
  int L = n;
  for (int i = 0; i < I.npass - 1; ++i) {
    fft_pass_dispatch<false>(I.radix[i], buf, n, nb, L, I.tw);
    L /= I.radix[i];
    __syncthreads();
  }
  const int Rc = I.radix[I.npass - 1];
  if (Rc == 8)
    fft_center<8>(buf, n, nb, I.kd);
  else if (Rc == 4)
    fft_center<4>(buf, n, nb, I.kd);
  else
    fft_center<2>(buf, n, nb, I.kd);
  __syncthreads();
  for (int i = I.npass - 2; i >= 0; --i) {
    L *= I.radix[i];
    fft_pass_dispatch<true>(I.radix[i], buf, n, nb, L, I.tw);
    __syncthreads();
  }
}

// Coupling F_{st}(q_j) from the stored upper triangle.
__device__ __forceinline__ double coupling(const InstDesc& I, int s, int t, int j) {
  const int S = I.S;
  if (s < t) {
    const int p = s * S - (s * (s + 1)) / 2 + (t - s - 1);
    return __ldg(I.F + (size_t)p * I.n + j);
  } else {
    const int p = t * S - (t * (t + 1)) / 2 + (s - t - 1);
    return -__ldg(I.F + (size_t)p * I.n + j);
  }
}

// y = e z + a x + c (H x), H of Eq. (adiab_mol_ham) by the dynamic Fourier
// method.  With A = p - i hbar F = -i hbar (D + F), the Hamiltonian equals
// -hbar^2/(2m) (D + F)^2 + V exactly (F real antisymmetric, D the spectral
// derivative), so H x is two applications of (D + F): each a forward FFT,
// a multiplication by i k and an inverse FFT per surface, plus the pointwise
// coupling -- 4 transforms per surface, as counted in Table I.
// sbuf holds nb_cap vectors of length n; U = I.work (scratch).  y may alias
// x or z.  z may be null when e == 0.
__device__ __forceinline__ void apply_h_axpby(const InstDesc& I, double2* sbuf, int nb_cap, const double2* x,
                                              double2* y, const double2* z, double e, double a, double2 c) {
  const int n = I.n, S = I.S;
  const int ln = ilog2(n);
  double2* U = I.work;
  const int nb = (S <= nb_cap) ? S : 1;
  // U = (D + F) x
  for (int s0 = 0; s0 < S; s0 += nb) {
    for (int i = threadIdx.x; i < nb * n; i += kThreads) sbuf[i] = x[s0 * n + i];
    __syncthreads();
    spectral_derivative(sbuf, nb, I);
    for (int i = threadIdx.x; i < nb * n; i += kThreads) {
      const int s = s0 + (i >> ln), j = i & (n - 1);
      double2 acc = sbuf[i];
      for (int t = 0; t < S; ++t)
        if (t != s) acc = caxpy_r(coupling(I, s, t, j), x[t * n + j], acc);
      U[s * n + j] = acc;
    }
    __syncthreads();
  }
  // y = e z + a x + c (-hbar^2/2m (D + F) U + V x)
  const double mh = -I.h2m;
  for (int s0 = 0; s0 < S; s0 += nb) {
    for (int i = threadIdx.x; i < nb * n; i += kThreads) sbuf[i] = U[s0 * n + i];
    __syncthreads();
    spectral_derivative(sbuf, nb, I);
    for (int i = threadIdx.x; i < nb * n; i += kThreads) {
      const int s = s0 + (i >> ln), j = i & (n - 1);
      double2 acc = sbuf[i];
      for (int t = 0; t < S; ++t)
        if (t != s) acc = caxpy_r(coupling(I, s, t, j), U[t * n + j], acc);
      const double2 xs = x[s * n + j];
      const double v = __ldg(I.V + s * n + j);
      const double2 hx = make_double2(fma(mh, acc.x, v * xs.x), fma(mh, acc.y, v * xs.y));
      double2 out = caxpy(c, hx, make_double2(a * xs.x, a * xs.y));
      if (e != 0.0) out = caxpy_r(e, z[s * n + j], out);
      y[s * n + j] = out;
    }
    __syncthreads();
  }
}

}  // namespace qg
