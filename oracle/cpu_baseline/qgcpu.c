/*
 * CPU timing baseline of the composed implicit midpoint propagation: the same
 * algorithm as the GPU library, written independently in plain C with FP64
 * arithmetic and OpenMP over wavepackets.
 *
 * TEST INFRASTRUCTURE ONLY: bench.py times it beside the GPU path; the tests
 * check it against the dense oracle.  It shares no code with the CUDA library.
 *
 *  - H psi (Eq. adiab_mol_ham): H = -hbar^2/(2m) (D + F)^2 + V, D the spectral
 *    first derivative (Sec. II D) by an iterative radix-2 FFT, F the real
 *    antisymmetric coupling; 4 transforms per surface.
 *  - Implicit midpoint (Eq. imp_midpoint): (1 + i tau H) chi = psi,
 *    psi' = 2 chi - psi, tau = f dt / 2; the explicit-Euler start
 *    psi - i tau H psi (Sec. II B) from H psi carried between elementary
 *    steps (H psi' = 2 H chi - H psi, H chi = i (chi - psi) / tau), exact at
 *    the first fraction of every composed step.
 *  - Each solve: minimal residual by the Lanczos three-term recurrence of the
 *    Hermitian H (A V_k = V_{k+1}([I; 0] + i tau T_k)), Givens rotations on
 *    the tridiagonal least-squares problem, stop when the recurrence residual
 *    is <= tol ||b||.
 *  - Composition: Suzuki's fractal (Eq. suzukis_fractal), recursively.
 *
 * Layout: psi is npk packets x S surfaces x N points of interleaved complex
 * doubles (re, im); V is S x N, F the upper triangle S(S-1)/2 x N.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
  int n, S, npair;
  double h2m, dq;
  const double* V;
  const double* F;
  cplx* w;       /* exp(-2 pi i k / n), k < n/2 */
  int* rev;      /* bit reversal */
  double* ikn;   /* k_j / n in natural order */
} Model;

static int log2i(int n) {
  int k = 0;
  while ((1 << k) < n) ++k;
  return k;
}

/* in-place radix-2 decimation-in-time FFT; sign -1 forward, +1 inverse
 * (unnormalised) */
static void fft(const Model* M, cplx* x, int sign) {
  const int n = M->n;
  for (int i = 0; i < n; ++i) {
    const int j = M->rev[i];
    if (j > i) {
      cplx t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1, step = n / len;
    for (int b = 0; b < n; b += len) {
      for (int j = 0; j < half; ++j) {
        cplx w = M->w[j * step];
        if (sign > 0) w = conj(w);
        const cplx u = x[b + j];
        const cplx v = w * x[b + j + half];
        x[b + j] = u + v;
        x[b + j + half] = u - v;
      }
    }
  }
}

/* x <- D x (one surface) */
static void deriv(const Model* M, cplx* x) {
  fft(M, x, -1);
  for (int j = 0; j < M->n; ++j) x[j] *= I * M->ikn[j];
  fft(M, x, +1);
}

static double coup(const Model* M, int s, int t, int j) {
  if (s == t) return 0.0;
  const int S = M->S;
  if (s < t) return M->F[(size_t)(s * S - s * (s + 1) / 2 + (t - s - 1)) * M->n + j];
  return -M->F[(size_t)(t * S - t * (t + 1) / 2 + (s - t - 1)) * M->n + j];
}

/* y = H x; U, T scratch of S n */
static void hpsi(const Model* M, const cplx* x, cplx* y, cplx* U, cplx* T) {
  const int n = M->n, S = M->S;
  for (int s = 0; s < S; ++s) {
    memcpy(T + (size_t)s * n, x + (size_t)s * n, sizeof(cplx) * n);
    deriv(M, T + (size_t)s * n);
  }
  for (int s = 0; s < S; ++s)
    for (int j = 0; j < n; ++j) {
      cplx a = T[(size_t)s * n + j];
      for (int t = 0; t < S; ++t)
        if (t != s) a += coup(M, s, t, j) * x[(size_t)t * n + j];
      U[(size_t)s * n + j] = a;
    }
  for (int s = 0; s < S; ++s) {
    memcpy(T + (size_t)s * n, U + (size_t)s * n, sizeof(cplx) * n);
    deriv(M, T + (size_t)s * n);
  }
  for (int s = 0; s < S; ++s)
    for (int j = 0; j < n; ++j) {
      cplx a = T[(size_t)s * n + j];
      for (int t = 0; t < S; ++t)
        if (t != s) a += coup(M, s, t, j) * U[(size_t)t * n + j];
      y[(size_t)s * n + j] = -M->h2m * a + M->V[(size_t)s * n + j] * x[(size_t)s * n + j];
    }
}

static double nrm2(const cplx* a, int len, double dq) {
  double s = 0.0;
  for (int i = 0; i < len; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
  return sqrt(dq * s);
}

typedef struct {
  cplx *U, *T, *Vp, *Vc, *Wn, *Dp, *Dq, *B, *X;
  long hpsi, iters;
} Work;

/* Solve (1 + i tau H) X = b from the start in X (minimal residual by the
 * Lanczos recurrence).  Returns 0 on convergence. */
static int solve(const Model* M, Work* w, double tau, const cplx* b, cplx* X, double tol, int max_iters) {
  const int len = M->S * M->n;
  const double dq = M->dq;
  const double bn = nrm2(b, len, dq);
  const double target = tol * bn;
  int total = 0;
  for (int restart = 0; restart < 4; ++restart) {
    /* r = b - A X */
    hpsi(M, X, w->Vc, w->U, w->T);
    w->hpsi++;
    for (int i = 0; i < len; ++i) w->Vc[i] = b[i] - (X[i] + I * tau * w->Vc[i]);
    const double beta1 = nrm2(w->Vc, len, dq);
    if (beta1 <= target || bn == 0.0) return 0;
    for (int i = 0; i < len; ++i) {
      w->Vc[i] /= beta1;
      w->Dp[i] = 0.0;
      w->Dq[i] = 0.0;
    }
    cplx g = beta1;
    double c1 = 1.0, c2 = 1.0, betak = 0.0;
    cplx s1 = 0.0, s2 = 0.0;
    int conv = 0;
    for (int k = 1; total < max_iters; ++k) {
      hpsi(M, w->Vc, w->Wn, w->U, w->T);
      w->hpsi++;
      double alpha = 0.0;
      for (int i = 0; i < len; ++i) {
        if (k > 1) w->Wn[i] -= betak * w->Vp[i];
        alpha += creal(conj(w->Vc[i]) * w->Wn[i]);
      }
      alpha *= dq;
      double bs = 0.0;
      for (int i = 0; i < len; ++i) {
        w->Wn[i] -= alpha * w->Vc[i];
        bs += creal(w->Wn[i]) * creal(w->Wn[i]) + cimag(w->Wn[i]) * cimag(w->Wn[i]);
      }
      const double betan = sqrt(dq * bs);
      /* column k of [I; 0] + i tau T_k: rows k-1, k, k+1 */
      cplx eps = 0.0, del = I * tau * betak, gam = 1.0 + I * tau * alpha;
      const cplx nu = I * tau * betan;
      if (k >= 3) {
        eps = s2 * del;
        del = c2 * del;
      }
      if (k >= 2) {
        const cplx t = c1 * del + s1 * gam;
        gam = -conj(s1) * del + c1 * gam;
        del = t;
      }
      const double aa = cabs(gam), nn = cabs(nu);
      double c;
      cplx s, r;
      if (nn == 0.0) {
        c = 1.0;
        s = 0.0;
        r = gam;
      } else if (aa == 0.0) {
        c = 0.0;
        s = conj(nu) / nn;
        r = nn;
      } else {
        const double rho = hypot(aa, nn);
        const cplx ph = gam / aa;
        c = aa / rho;
        s = ph * conj(nu) / rho;
        r = ph * rho;
      }
      const cplx gk = c * g;
      const cplx gnext = -conj(s) * g;
      const double ibn = betan > 0.0 ? 1.0 / betan : 0.0;
      for (int i = 0; i < len; ++i) {
        const cplx d = (w->Vc[i] - del * w->Dp[i] - eps * w->Dq[i]) / r;
        w->Dq[i] = d;
        X[i] += gk * d;
        w->Wn[i] *= ibn;
      }
      cplx* t0 = w->Dq;
      w->Dq = w->Dp;
      w->Dp = t0;
      t0 = w->Vp;
      w->Vp = w->Vc;
      w->Vc = w->Wn;
      w->Wn = t0;
      c2 = c1;
      s2 = s1;
      c1 = c;
      s1 = s;
      betak = betan;
      g = gnext;
      total++;
      w->iters++;
      if (cabs(g) <= target) {
        conv = 1;
        break;
      }
      if (betan == 0.0) break;
    }
    if (conv) return 0;
    if (total >= max_iters) break;
  }
  return 1;
}

/* Suzuki fractal fractions of order `order` (Sec. II C); returns the count */
static int suzuki(int order, double* fr) {
  int cnt = 1;
  fr[0] = 1.0;
  for (int p = 2; p < order; p += 2) {
    const double r = pow(4.0, 1.0 / (p + 1));
    const double a = 1.0 / (4.0 - r), m = -r / (4.0 - r);
    const double g[5] = {a, a, m, a, a};
    double* nx = (double*)malloc(sizeof(double) * cnt * 5);
    int k = 0;
    for (int q = 0; q < 5; ++q)
      for (int b = 0; b < cnt; ++b) nx[k++] = g[q] * fr[b];
    memcpy(fr, nx, sizeof(double) * k);
    free(nx);
    cnt = k;
  }
  return cnt;
}

/* Propagates npk packets by nsteps composed steps of the implicit midpoint
 * method, Suzuki order `order`, step dt.  Returns 0 if every solve
 * converged; *threads receives the OpenMP thread count, *hpsi and *iters the
 * totals over all packets. */
int qgcpu_propagate(int n, double qmin, double qmax, int S, double mass, const double* V, const double* F,
                    double* psi_io, int npk, int order, double dt, long nsteps, double tol, int max_iters,
                    int* threads, long* hpsi_out, long* iters_out) {
  if (n < 2 || (n & (n - 1)) || S < 2 || order < 2 || order > 8 || (order & 1)) return -1;
  Model M;
  M.n = n;
  M.S = S;
  M.npair = S * (S - 1) / 2;
  M.h2m = 1.0 / (2.0 * mass);
  M.dq = (qmax - qmin) / n;
  M.V = V;
  M.F = F;
  M.w = (cplx*)malloc(sizeof(cplx) * (n / 2));
  M.rev = (int*)malloc(sizeof(int) * n);
  M.ikn = (double*)malloc(sizeof(double) * n);
  const int lg = log2i(n);
  for (int k = 0; k < n / 2; ++k) M.w[k] = cexp(-2.0 * M_PI * I * (double)k / n);
  for (int i = 0; i < n; ++i) {
    int r = 0;
    for (int b = 0; b < lg; ++b)
      if (i & (1 << b)) r |= 1 << (lg - 1 - b);
    M.rev[i] = r;
    const int f = i < n / 2 ? i : i - n;
    M.ikn[i] = 2.0 * M_PI / (n * M.dq) * f / n;
  }
  double fr[128];
  const int nfrac = suzuki(order, fr);
  const int len = S * n;
  int fails = 0;
  long th = 1, hp = 0, it = 0;
#pragma omp parallel reduction(+ : fails, hp, it)
  {
#ifdef _OPENMP
#pragma omp single
    th = omp_get_num_threads();
#endif
    Work w;
    cplx* mem = (cplx*)malloc(sizeof(cplx) * (size_t)len * 9);
    w.U = mem;
    w.T = mem + len;
    w.Vp = mem + 2 * len;
    w.Vc = mem + 3 * len;
    w.Wn = mem + 4 * len;
    w.Dp = mem + 5 * len;
    w.Dq = mem + 6 * len;
    w.B = mem + 7 * len;
    w.X = mem + 8 * len;
    w.hpsi = 0;
    w.iters = 0;
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < npk; ++p) {
      cplx* psi = (cplx*)psi_io + (size_t)p * len;
      for (long step = 0; step < nsteps; ++step) {
        for (int f = 0; f < nfrac; ++f) {
          const double tau = 0.5 * fr[f] * dt;
          if (f == 0) {
            hpsi(&M, psi, w.B, w.U, w.T);
            w.hpsi++;
          }
          for (int i = 0; i < len; ++i) w.X[i] = psi[i] - I * tau * w.B[i];
          if (solve(&M, &w, tau, psi, w.X, tol, max_iters)) fails++;
          for (int i = 0; i < len; ++i) {
            const cplx hc = I * (w.X[i] - psi[i]) / tau;
            w.B[i] = 2.0 * hc - w.B[i];
            psi[i] = 2.0 * w.X[i] - psi[i];
          }
        }
      }
    }
    hp += w.hpsi;
    it += w.iters;
    free(mem);
  }
  free(M.w);
  free(M.rev);
  free(M.ikn);
  if (threads) *threads = (int)th;
  if (hpsi_out) *hpsi_out = hp;
  if (iters_out) *iters_out = it;
  return fails ? 1 : 0;
}
