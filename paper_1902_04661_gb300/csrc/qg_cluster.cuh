// The shared-memory-resident, thread-block-cluster form of the 1-D
// propagator: one instance is spread over a cluster of G CTAs (G = 1, 2, 4,
// 8, 16) and every vector the solver touches lives in shared memory.
//
// Layout.  N = G M grid points; CTA r of the cluster owns the points
// j = r + G n2 (n2 = 0..M-1) of every surface, stored locally at
// i = s M + n2.  The pointwise parts of H psi (coupling F, potential V) and
// every Krylov vector operation are then local.
//
// Spectral derivative (Sec. II D) of a vector in this layout.  With
// j = r + G n2 and k = k2 + M k1 the DFT factors as
//   X(k2 + M k1) = sum_r w_G^{r k1} [ w_N^{r k2} sum_n2 x_r(n2) w_M^{n2 k2} ],
// so each CTA first runs a local length-M DFT of its points (decimation in
// frequency, spectrum left in digit-reversed order), multiplies by the cross
// twiddle w_N^{r k2}, and the length-G DFTs over r -- one per k2 -- run in a
// "centre" phase in which CTA c handles a 1/G share of the positions: it reads
// the G values of a position from the G CTAs' shared memory (distributed
// shared memory), takes the G-point DFT, multiplies by i k / N, takes the
// inverse G-point DFT and writes the G results back where it read them.  The
// inverse local DFT (decimation in time) after the conjugate cross twiddle
// completes D x.  Two cluster barriers per derivative.
//
// Sums over the state: each CTA reduces its part, publishes it in a
// double-buffered slot of its shared memory, and after one cluster barrier
// every CTA adds the G slots in rank order, so all CTAs hold bitwise equal
// sums and take the same decisions.
#pragma once

#include <cooperative_groups.h>

#include "qg_solver.cuh"

namespace qg {

namespace cgx = cooperative_groups;

// Per-CTA capacity of the cluster form: complex values of one local vector.
constexpr int kClusterLocal = 1024;

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
template <typename T>
__device__ __forceinline__ T* dsmem(T* p, int rank) {
  return cgx::this_cluster().map_shared_rank(p, (unsigned)rank);
}

// 16-point DFT in registers as 4 x 4 (n = 4 n1 + n2, k = k1 + 4 k2):
// 4-point DFTs over n1, twiddles w16^{n2 k1}, 4-point DFTs over n2.
template <bool INV, typename C>
__device__ __forceinline__ void dft16(C (&x)[16]) {
  using R = decltype(C::x);
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, h = (R)0.70710678118654752440;
  C a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C t0 = x[n2], t1 = x[4 + n2], t2 = x[8 + n2], t3 = x[12 + n2];
    dft4<INV>(t0, t1, t2, t3);
    a[n2][0] = t0;
    a[n2][1] = t1;
    a[n2][2] = t2;
    a[n2][3] = t3;
  }
  // w16^e for e = n2 k1 (0..9): cos(pi e / 8), -+ sin(pi e / 8)
  const R cs[10] = {(R)1, c1, h, s1, (R)0, -s1, -h, -c1, (R)-1, -c1};
  const R sn[10] = {(R)0, s1, h, c1, (R)1, c1, h, s1, (R)0, -s1};
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2) {
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) {
      const int e = n2 * k1;
      const C w = cmk<C>(cs[e], INV ? sn[e] : -sn[e]);
      a[n2][k1] = cmul(a[n2][k1], w);
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C t0 = a[0][k1], t1 = a[1][k1], t2 = a[2][k1], t3 = a[3][k1];
    dft4<INV>(t0, t1, t2, t3);
    x[k1] = t0;
    x[k1 + 4] = t1;
    x[k1 + 8] = t2;
    x[k1 + 12] = t3;
  }
}

template <int G, bool INV, typename C>
__device__ __forceinline__ void dftg(C (&x)[G]) {
  if constexpr (G == 16)
    dft16<INV>(x);
  else if constexpr (G > 1)
    dft<G, INV>(x);
}

// Last forward pass (block length RD, no twiddles inside) followed by the
// cross twiddle w_N^{r k2(p)} at each position p (cw, length M).
template <int RD>
__device__ __forceinline__ void fft_last_cross(double2* gbuf, int M, int nb, const double2* __restrict__ cw) {
  double2* buf = in_dyn_smem(gbuf);
  const int total = (nb * M) / RD;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int e0 = b * RD;
    const int pos = e0 & (M - 1);
    double2 x[RD];
#pragma unroll
    for (int r = 0; r < RD; ++r) x[r] = buf[spad<double2>(e0 + r)];
    dft<RD, false>(x);
#pragma unroll
    for (int r = 0; r < RD; ++r) buf[spad<double2>(e0 + r)] = cmul(x[r], cw[pos + r]);
  }
}

// The same last forward pass in the factored form of the one-CTA transform
// (set blk of the pass's factor tables), then the cross twiddle.
template <int RD>
__device__ __forceinline__ void lf_last_cross(double2* gbuf, int M, int nb, const double2* __restrict__ ent,
                                              const unsigned* __restrict__ flg, const double2* __restrict__ cw) {
  double2* buf = in_dyn_smem(gbuf);
  const int total = (nb * M) / RD;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int e0 = b * RD;
    const int pos = e0 & (M - 1);
    double2 x[RD];
#pragma unroll
    for (int r = 0; r < RD; ++r) x[r] = buf[spad<double2>(e0 + r)];
    LfW w[RD == 8 ? 4 : 2];
    lf_load<RD>(ent, flg, M / RD, pos / RD, w);
    lf_bfly<RD, false>(x, w);
#pragma unroll
    for (int k = 0; k < RD; ++k) buf[spad<double2>(e0 + k)] = cmul(x[bitrev<RD>(k)], cw[pos + k]);
  }
}

// Conjugate cross twiddle, then the first inverse pass (block length RD).
template <int RD>
__device__ __forceinline__ void fft_first_cross_inv(double2* gbuf, int M, int nb, const double2* __restrict__ cw) {
  double2* buf = in_dyn_smem(gbuf);
  const int total = (nb * M) / RD;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int e0 = b * RD;
    const int pos = e0 & (M - 1);
    double2 x[RD];
#pragma unroll
    for (int r = 0; r < RD; ++r) x[r] = cmulc(buf[spad<double2>(e0 + r)], cw[pos + r]);
    dft<RD, true>(x);
#pragma unroll
    for (int r = 0; r < RD; ++r) buf[spad<double2>(e0 + r)] = x[r];
  }
}

// Radix plan of the local length M.  As for the full grids (radix-8 passes,
// then one or two radix-4 passes) while a radix-8 pass still gives four warps
// a butterfly each (S M / 8 >= 128); below that, radix-4 passes (one radix-8
// pass first when log2 M is odd), which occupy twice as many threads per pass
// for the same FP64 work per point -- the FP64 units of an SM sit in its four
// schedulers, and a pass of 64 radix-8 butterflies keeps only two of them
// busy.
struct LocalPlan {
  int M, npass, n8;
  int radix[QG_MAX_PASSES];
};

__host__ __device__ inline LocalPlan local_plan(int M, int S) {
  LocalPlan p;
  p.M = M;
  int k = 0;
  while ((1 << k) < M) ++k;
  p.npass = 0;
  if ((S * M) / 8 >= 4 * 32) {
    const FftPlan f = make_plan(M);
    for (int i = 0; i < f.npass; ++i) p.radix[p.npass++] = f.radix[i];
  } else {
    if (k % 2 == 1) {
      p.radix[p.npass++] = 8;
      k -= 3;
    }
    for (; k > 0; k -= 2) p.radix[p.npass++] = 4;
  }
  for (int i = p.npass; i < QG_MAX_PASSES; ++i) p.radix[i] = 1;
  p.n8 = count_radix8(p.radix, p.npass);
  return p;
}

// Bytes of the local plan's factor tables (entries, then form words).
__host__ __device__ inline size_t local_lf_bytes(int M, int S) {
  const LocalPlan p = local_plan(M, S);
  int e = 0, st = 0;
  lf_counts(p.radix, p.npass, M, &e, &st);
  return ((size_t)e * 16 + (size_t)st * 4 + 15) & ~(size_t)15;
}

// The instance's share of one cluster: shared-memory vectors and tables.
template <int G>
struct DomC {
  static constexpr bool kFusedDots = false;
  // the FP64 Lanczos solve keeps its vectors in the workspace basis (lanczos_stored_solve)
  static constexpr bool kStoredLanczos = false;
  // the same for the complex64 inner solves of the mixed form (the cluster form has no complex64 inner solve)
  static constexpr bool kStoredLanczos32 = false;
  int len;        // S M local values per vector
  double dv;
  unsigned char* gm;
  double* red;
  double* part;   // 2 x 16 partial-sum slots (same offset in every CTA)
  int parity;
  int M, S, lm, rank, q0, Q;
  LocalPlan lp;
  double h2m;
  const double* V;      // S x M
  const double* F;      // S(S-1)/2 x M
  double2* U;
  double2* fb;          // padded FFT buffer, S x M
  const double2* lf;    // factor tables of the local transform (see lf_tables)
  const unsigned* lff;
  const double2* cw;    // cross twiddles w_N^{r k2(p)}
  const double* kc;     // centre wave numbers / N: Q x G
  double2* basis64;
  double2* res64;
  float2 *r32, *d32, *basis32;

  template <class Fn>
  __device__ __forceinline__ void each(Fn&& f) {
    const int n = len;
    for (int i = threadIdx.x; i < n; i += kThreads) f(i);
  }
  template <int U, class Ld, class St>
  __device__ __forceinline__ void each_u(Ld&& ld, St&& st) {
    each([&](int i) { st(i, ld(i)); });
  }

  template <int K, typename R>
  __device__ __forceinline__ bool sum(R (&v)[K], R* out) {
    static_assert(sizeof(R) == 8, "the cluster form sums in FP64");
    cta_sum<K>(v, reinterpret_cast<R*>(red), out);
    if constexpr (G > 1) {
      double* slot = part + parity * 16;
      if (threadIdx.x < K) slot[threadIdx.x] = out[threadIdx.x];
      cluster_barrier();
      if (threadIdx.x < K) {
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < G; ++r) s += dsmem(slot, r)[threadIdx.x];
        out[threadIdx.x] = s;
      }
      __syncthreads();
      parity ^= 1;
    }
    return true;
  }

  __device__ __forceinline__ bool ok() const { return true; }

  // buf <- D buf (all S local vectors), see the file comment.  The local
  // passes are those of the one-CTA FP64 transform (lf_pass): the first
  // forward pass untwiddled, the others factored.
  __device__ __noinline__ void derivative(double2* buf) {
    const int np = lp.npass, n8 = lp.n8;
    const double2* ent = lf;
    const unsigned* flg = lff;
    int L = M;
    for (int i = 0; i < np - 1; ++i) {
      const int RD = i < n8 ? 8 : 4;
      if (i == 0) {
        if (RD == 8)
          lf_pass<8, false, false>(buf, M, S, L, nullptr, nullptr);
        else
          lf_pass<4, false, false>(buf, M, S, L, nullptr, nullptr);
      } else {
        if (RD == 8)
          lf_pass<8, false, true>(buf, M, S, L, ent, flg);
        else
          lf_pass<4, false, true>(buf, M, S, L, ent, flg);
        ent += (RD == 8 ? 4 : 2) * (M / L);
        flg += M / L;
      }
      L /= RD;
      __syncthreads();
    }
    const bool last8 = np - 1 < n8;
    if (np == 1) {
      if (last8)
        fft_last_cross<8>(buf, M, S, cw);
      else
        fft_last_cross<4>(buf, M, S, cw);
    } else {
      if (last8)
        lf_last_cross<8>(buf, M, S, ent, flg, cw);
      else
        lf_last_cross<4>(buf, M, S, ent, flg, cw);
      ent += (L == 8 ? 4 : 2) * (M / L);
      flg += M / L;
    }
    if constexpr (G > 1)
      cluster_barrier();
    else
      __syncthreads();
    double2* sb = in_dyn_smem(buf);
    for (int q = q0 + threadIdx.x; q < q0 + Q; q += kThreads) {
      const int e = spad<double2>(q);
      double2 y[G];
#pragma unroll
      for (int r = 0; r < G; ++r) y[r] = (G > 1) ? dsmem(sb, r)[e] : sb[e];
      dftg<G, false>(y);
      const double* kk = kc + (size_t)(q - q0) * G;
#pragma unroll
      for (int k1 = 0; k1 < G; ++k1) {
        const double k = kk[k1];
        y[k1] = make_double2(-k * y[k1].y, k * y[k1].x);
      }
      dftg<G, true>(y);
#pragma unroll
      for (int r = 0; r < G; ++r) {
        if constexpr (G > 1)
          dsmem(sb, r)[e] = y[r];
        else
          sb[e] = y[r];
      }
    }
    if constexpr (G > 1)
      cluster_barrier();
    else
      __syncthreads();
    if (last8)
      fft_first_cross_inv<8>(buf, M, S, cw);
    else
      fft_first_cross_inv<4>(buf, M, S, cw);
    __syncthreads();
    for (int i = np - 2; i >= 0; --i) {
      const int RD = i < n8 ? 8 : 4;
      L *= RD;
      if (RD == 8)
        lf_pass<8, true, true>(buf, M, S, L, ent, flg);
      else
        lf_pass<4, true, true>(buf, M, S, L, ent, flg);
      ent += (RD == 8 ? 4 : 2) * (L / RD);
      flg += L / RD;
      __syncthreads();
    }
  }

  __device__ __forceinline__ double coup(int s, int t, int j) const {
    const int a = s < t ? s : t, b = s < t ? t : s;
    const int p = a * S - (a * (a + 1)) / 2 + (b - a - 1);
    return neg_if(F[p * M + j], s > t);   // F_ts = -F_st
  }

  // y = e z + a x + c (H x), H = -hbar^2/2m (D + F)^2 + V (Eq. adiab_mol_ham
  // written as two applications of D + F).  y may alias x or z.
  template <typename R>
  __device__ void hpsi(const double2* x, double2* y, const double2* z, double e, double a, double2 c) {
    static_assert(sizeof(R) == 8, "the cluster form runs H psi in FP64");
    const int n = len, Mm = M, Ss = S, l2 = lm;
    double2* sb = in_dyn_smem(fb);
    for (int i = threadIdx.x; i < n; i += kThreads) sb[spad<double2>(i)] = x[i];
    __syncthreads();
    derivative(fb);
    // U = (D + F) x ; U also seeds the second derivative
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const int s = i >> l2, j = i & (Mm - 1);
      double2 acc = sb[spad<double2>(i)];
      for (int t = 0; t < Ss; ++t)
        if (t != s) acc = caxpy_r(coup(s, t, j), x[t * Mm + j], acc);
      U[i] = acc;
      sb[spad<double2>(i)] = acc;
    }
    __syncthreads();
    derivative(fb);
    const double mh = -h2m;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const int s = i >> l2, j = i & (Mm - 1);
      double2 acc = sb[spad<double2>(i)];
      for (int t = 0; t < Ss; ++t)
        if (t != s) acc = caxpy_r(coup(s, t, j), U[t * Mm + j], acc);
      const double2 xs = x[i];
      const double v = V[i];
      const double2 hx = make_double2(fma(mh, acc.x, v * xs.x), fma(mh, acc.y, v * xs.y));
      double2 out = caxpy(c, hx, make_double2(a * xs.x, a * xs.y));
      if (e != 0.0) out = caxpy_r(e, z[i], out);
      y[i] = out;
    }
    __syncthreads();
  }
};

// Dynamic shared memory of the cluster form for one instance shape.
struct ClusterSmem {
  size_t fb, vec, lanczos, V, F, lf, cw, kc, k2, part, total;
};

__host__ __device__ inline ClusterSmem cluster_smem_layout(int M, int S, int G, int restart) {
  ClusterSmem L;
  const size_t len = (size_t)S * M;
  const size_t vecb = len * 16;
  size_t gmb = (size_t)(restart + 1) * restart * 16 + (size_t)(restart + 1) * 16 + (size_t)restart * 40 + 256;
  size_t lz = 5 * vecb > gmb ? 5 * vecb : gmb;
  size_t off = 0;
  L.fb = off;
  off += (padded_bytes(len, 16) + 255) & ~size_t(255);
  L.vec = off;            // U, psi, B, X
  off += 4 * vecb;
  L.lanczos = off;        // 5 Lanczos vectors or the GMRES arrays
  off += (lz + 255) & ~size_t(255);
  L.V = off;
  off += ((size_t)S * M * 8 + 255) & ~size_t(255);
  L.F = off;
  off += ((size_t)(S * (S - 1) / 2) * M * 8 + 255) & ~size_t(255);
  L.lf = off;
  off += (local_lf_bytes(M, S) + 255) & ~size_t(255);
  L.cw = off;
  off += (size_t)M * 16;
  L.kc = off;
  off += ((len / G) * G * 8 + 255) & ~size_t(255);
  L.k2 = off;
  off += ((size_t)M * 4 + 255) & ~size_t(255);
  L.part = off;
  off += 2 * 16 * 8;
  L.total = off;
  (void)G;
  return L;
}

// w = exp(sgn 2 pi i num / den) in the factored form s (1 + i t) (form 0,
// |Re w| >= |Im w|) or s (t + i) (form 1); 2 num / den is a dyadic fraction,
// exact in a double, for sincospi.
__device__ __forceinline__ void lf_factor_dev(long long num, long long den, int sgn, double2* st, unsigned* form) {
  num %= den;
  if (num < 0) num += den;
  double s, c;
  sincospi(2.0 * (double)num / (double)den, &s, &c);
  if (sgn < 0) s = -s;
  if (fabs(c) >= fabs(s)) {
    *st = make_double2(c, s / c);
    *form = 0u;
  } else {
    *st = make_double2(s, c / s);
    *form = 1u;
  }
}

// Factor tables of the local transform, in the layout of the one-CTA
// transform's tables (forward passes 1..np-1 one set per block, then inverse
// passes np-2..0 one set per position; entry e of set k at e * nsets + k;
// one word of form bits per set).  ent must hold local_lf_bytes(M, S).
static __device__ void build_local_lf(const LocalPlan& lp, double2* ent, unsigned* flg) {
  const int M = lp.M, np = lp.npass;
  int Ls[QG_MAX_PASSES];
  for (int i = 0, L = M; i < np; ++i) {
    Ls[i] = L;
    L /= lp.radix[i];
  }
  for (int i = 1; i < np; ++i) {
    const int R = lp.radix[i], E = R == 8 ? 4 : 2, o = R == 8 ? 0 : 1, nbk = M / Ls[i];   // radix 4: W^2, W
    const long long B = (long long)nbk * R;
    for (int k = threadIdx.x; k < nbk; k += kThreads) {
      const long long K = block_frequency(k, lp.radix, nbk);
      const long long a[4] = {4 * K, 2 * K, K, 8 * K + B}, b[4] = {B, B, B, 8 * B};
      unsigned fl = 0u;
      for (int e = 0; e < E; ++e) {
        unsigned f = 0u;
        lf_factor_dev(a[e + o], b[e + o], -1, &ent[(size_t)e * nbk + k], &f);
        fl |= f << e;
      }
      flg[k] = fl;
    }
    ent += (size_t)E * nbk;
    flg += nbk;
  }
  for (int i = np - 2; i >= 0; --i) {
    const int R = lp.radix[i], E = R == 8 ? 4 : 2, o = R == 8 ? 0 : 1, m = Ls[i] / R;
    const long long Lb = Ls[i];
    for (int j = threadIdx.x; j < m; j += kThreads) {
      const long long a[4] = {4LL * j, 2LL * j, (long long)j, 8LL * j + Lb}, b[4] = {Lb, Lb, Lb, 8 * Lb};
      unsigned fl = 0u;
      for (int e = 0; e < E; ++e) {
        unsigned f = 0u;
        lf_factor_dev(a[e + o], b[e + o], +1, &ent[(size_t)e * m + j], &f);
        fl |= f << e;
      }
      flg[j] = fl;
    }
    ent += (size_t)E * m;
    flg += m;
  }
}

// Tables of the local plan: the factor tables (build_local_lf), the
// frequency k2(p) held at each position p after the forward passes, the
// cross twiddles w_N^{rank k2(p)} and the centre wave numbers k(k2 + M k1) / N
// of this CTA's centre positions.
template <int G>
__device__ void build_cluster_tables(const LocalPlan& lp, int n, double dq, int rank, int q0, int Q, double2* lfe,
                                     unsigned* lff, double2* cw, double* kc, int* k2tab) {
  const int M = lp.M;
  build_local_lf(lp, lfe, lff);
  for (int k = threadIdx.x; k < M; k += kThreads) {
    double s, c;
    int f = 0, mult = 1, rem = k, len = M;
    for (int i = 0; i < lp.npass; ++i) {
      const int m = len / lp.radix[i];
      const int qd = rem / m;
      rem -= qd * m;
      f += mult * qd;
      mult *= lp.radix[i];
      len = m;
    }
    k2tab[k] = f;
    const long long ex = ((long long)rank * f) % n;
    sincospi(2.0 * (double)ex / (double)n, &s, &c);
    cw[k] = make_double2(c, -s);
  }
  __syncthreads();
  const double k0 = 2.0 * 3.14159265358979323846 / ((double)n * dq);
  for (int t = threadIdx.x; t < Q * G; t += kThreads) {
    const int q = q0 + t / G, k1 = t % G;
    const int p = q & (M - 1);
    const int f = k2tab[p] + M * k1;
    const int ff = f < n / 2 ? f : f - n;
    kc[t] = k0 * (double)ff / (double)n;
  }
}

// All nsteps composed steps of one instance on one cluster.
template <int G>
__device__ void run_cluster_instance(const InstDesc& I, const StepPlan& P, unsigned char* dyn, double* red, double* sc,
                                     qg_step_stats* st) {
  const int rank = (G > 1) ? (int)cgx::this_cluster().block_rank() : 0;
  const int n = I.n, S = I.S, M = n / G, len = S * M, npair = S * (S - 1) / 2;
  const ClusterSmem L = cluster_smem_layout(M, S, G, P.restart);
  DomC<G> D;
  D.len = len;
  D.dv = I.dq;
  D.red = red;
  D.part = reinterpret_cast<double*>(dyn + L.part);
  D.parity = 0;
  D.M = M;
  D.S = S;
  D.lm = ilog2(M);
  D.rank = rank;
  D.Q = len / G;
  D.q0 = rank * D.Q;
  D.lp = local_plan(M, S);
  D.h2m = I.h2m;
  double* Vl = reinterpret_cast<double*>(dyn + L.V);
  double* Fl = reinterpret_cast<double*>(dyn + L.F);
  D.V = Vl;
  D.F = Fl;
  D.fb = reinterpret_cast<double2*>(dyn + L.fb);
  double2* vec = reinterpret_cast<double2*>(dyn + L.vec);
  D.U = vec;
  double2* psi = vec + len;
  double2* B = vec + 2 * len;
  double2* X = vec + 3 * len;
  int lf_entries = 0, lf_sets = 0;
  lf_counts(D.lp.radix, D.lp.npass, M, &lf_entries, &lf_sets);
  double2* lfe = reinterpret_cast<double2*>(dyn + L.lf);
  unsigned* lff = reinterpret_cast<unsigned*>(lfe + lf_entries);
  D.lf = lfe;
  D.lff = lff;
  D.cw = reinterpret_cast<const double2*>(dyn + L.cw);
  D.kc = reinterpret_cast<const double*>(dyn + L.kc);
  const size_t SN = (size_t)S * n;
  if (P.solver == QG_SOLVER_LANCZOS) {
    D.basis64 = reinterpret_cast<double2*>(dyn + L.lanczos);
    D.gm = nullptr;
  } else {
    D.basis64 = I.work + 4 * SN + (size_t)rank * (P.restart + 1) * len;
    D.gm = dyn + L.lanczos;
  }
  D.res64 = nullptr;
  D.r32 = D.d32 = D.basis32 = nullptr;
  double2* P0 = I.work + 3 * SN + (size_t)rank * len;
  build_cluster_tables<G>(D.lp, n, I.dq, rank, D.q0, D.Q, lfe, lff, reinterpret_cast<double2*>(dyn + L.cw),
                          reinterpret_cast<double*>(dyn + L.kc), reinterpret_cast<int*>(dyn + L.k2));
  // this CTA's points j = rank + G n2 of the fields and of psi
  for (int i = threadIdx.x; i < len; i += kThreads) {
    const int s = i / M, n2 = i - s * M;
    const int j = rank + G * n2;
    Vl[i] = I.V[(size_t)s * n + j];
    psi[i] = I.psi[(size_t)s * n + j];
  }
  for (int i = threadIdx.x; i < npair * M; i += kThreads) {
    const int p = i / M, n2 = i - p * M;
    Fl[i] = I.F[(size_t)p * n + rank + G * n2];
  }
  __syncthreads();
  if constexpr (G > 1) cluster_barrier();
  Counters cnt{0, 0, 0, 0, 0, 0, 0, 0, 0.0};
  long long nsub = 0;
  const long long failed = run_steps<0>(D, P, psi, B, X, P0, false, nullptr, 0, 1, cnt, nsub, sc);
  for (int i = threadIdx.x; i < len; i += kThreads) {
    const int s = i / M, n2 = i - s * M;
    I.psi[(size_t)s * n + rank + G * n2] = psi[i];
  }
  if (rank == 0) write_stats(st, cnt, nsub, failed);
  __syncthreads();
  // no CTA may leave (or reuse its shared memory for the next instance)
  // while another still reads it
  if constexpr (G > 1) cluster_barrier();
}

}  // namespace qg
