// Host side of libqgeom: handles, FFT plans and tables, the C-ABI.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "qg_internal.h"

namespace {

thread_local char g_err[512] = "";

void set_err(const char* what, cudaError_t e) {
  snprintf(g_err, sizeof(g_err), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

#define QG_TRY(call)                               \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      set_err(#call, e_);                          \
      return e_ == cudaErrorMemoryAllocation ? QG_ERR_OOM : QG_ERR_CUDA; \
    }                                              \
  } while (0)

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2h(int v) {
  int k = 0;
  while ((1 << k) < v) ++k;
  return k;
}

// Twiddle table in the pass-by-pass layout fft_pass reads: for forward pass
// i (block length L, radix R, m = L / R) the entries (r - 1) m + j,
// r = 1..R-1, j = 0..m-1, hold w_L^{j r} = w[j r n / L] (w the natural table
// exp(-2 pi i k / n)).  The last pass has m = 1 and needs none; the layout
// has at most n - 1 entries and is padded with 1 to n.
void pass_twiddles(const FftPlan& p, const std::vector<double2>& w, std::vector<double2>& out) {
  const int n = p.n;
  out.assign(n, make_double2(1.0, 0.0));
  int L = n, off = 0;
  for (int i = 0; i < p.npass - 1; ++i) {
    const int R = p.radix[i], m = L / R;
    for (int r = 1; r < R; ++r)
      for (int j = 0; j < m; ++j) out[off + (r - 1) * m + j] = w[(size_t)j * r * (n / L)];
    off += (R - 1) * m;
    L /= R;
  }
}

// Frequency index held at position p after the decimation-in-frequency
// passes radix[first..]: a block of length len splits into R sub-blocks of
// length len/R; sub-block q holds the frequencies q + R f' where f' is the
// frequency at the same position inside the sub-transform.
void freq_positions(int len, const int* radix, int npass, std::vector<int>& f) {
  f.assign(len, 0);
  if (npass == 0 || len == 1) return;
  const int R = radix[0];
  const int m = len / R;
  std::vector<int> sub;
  freq_positions(m, radix + 1, npass - 1, sub);
  for (int q = 0; q < R; ++q)
    for (int pp = 0; pp < m; ++pp) f[q * m + pp] = q + R * sub[pp];
}

// w = exp(sgn 2 pi i num / den) in Linzer and Feig's factored form: w = s (1
// + i t) (form 0, |Re w| >= |Im w|) or w = s (t + i) (form 1), so |t| <= 1.
// cos and sin are evaluated in long double on at most an eighth of a turn
// and rotated by an exact multiple of a quarter turn; t is divided out in
// long double before rounding.
void lf_factor(long long num, long long den, int sgn, double2* st, unsigned* form) {
  num %= den;
  if (num < 0) num += den;
  const long long q = (4 * num + den / 2) / den;   // nearest quarter turn
  const long double two_pi = 6.283185307179586476925286766559005768L;
  const long double a = two_pi * (long double)(4 * num - q * den) / (4.0L * (long double)den);
  long double c = cosl(a), s = sinl(a);
  for (long long r = 0; r < (q & 3); ++r) {   // times i
    const long double t = c;
    c = -s;
    s = t;
  }
  if (sgn < 0) s = -s;
  if (fabsl(c) >= fabsl(s)) {
    *st = make_double2((double)c, (double)(s / c));
    *form = 0u;
  } else {
    *st = make_double2((double)s, (double)(c / s));
    *form = 1u;
  }
}

// Factor tables of the FP64 transform's Linzer-Feig passes, in the order the
// device runs them.  Forward passes 1..npass-1 (decimation in frequency with
// the twiddles taken at the input of a pass): block blk of a pass of radix R
// with nbk blocks multiplies its input r by W^r, W = exp(-2 pi i K / (nbk R)),
// K = block_frequency(blk).  Inverse passes npass-2..0 (decimation in time):
// position j of a pass with block length L multiplies input r by W^r, W =
// exp(+2 pi i j / L).  A radix-8 set holds W^4, W^2, W and zeta W (zeta =
// exp(-+2 pi i / 8), the sign of the pass), a radix-4 set W^2 and W; entry e
// of set k of a pass sits at e * nsets + k.  flg gets one word per set, bit e
// the form of entry e, in the same set order.
void lf_tables(const FftPlan& p, std::vector<double2>& ent, std::vector<unsigned>& flg) {
  const int n = p.n, np = p.npass;
  int Ls[QG_MAX_PASSES];
  for (int i = 0, L = n; i < np; ++i) {
    Ls[i] = L;
    L /= p.radix[i];
  }
  ent.clear();
  flg.clear();
  // one pass: nsets sets of E entries, set k's exponents num[e] / den[e]
  auto pass = [&](int R, int nsets, int sgn, auto&& exps) {
    const int E = R == 8 ? 4 : 2;
    const size_t base = ent.size(), fbase = flg.size();
    ent.resize(base + (size_t)E * nsets);
    flg.resize(fbase + nsets, 0u);
    for (int k = 0; k < nsets; ++k) {
      long long num[4], den[4];
      exps(k, num, den);
      for (int e = 0; e < E; ++e) {
        unsigned f = 0;
        lf_factor(num[e], den[e], sgn, &ent[base + (size_t)e * nsets + k], &f);
        flg[fbase + k] |= f << e;
      }
    }
  };
  for (int i = 1; i < np; ++i) {
    const int R = p.radix[i], nbk = n / Ls[i];
    const long long B = (long long)nbk * R;
    pass(R, nbk, -1, [&](int blk, long long* num, long long* den) {
      const long long K = block_frequency(blk, p.radix, nbk);
      const long long a[4] = {4 * K, 2 * K, K, 8 * K + B}, b[4] = {B, B, B, 8 * B};
      const int o = R == 8 ? 0 : 1;   // radix 4: W^2, W
      for (int e = 0; e + o < 4; ++e) {
        num[e] = a[e + o];
        den[e] = b[e + o];
      }
    });
  }
  for (int i = np - 2; i >= 0; --i) {
    const int R = p.radix[i];
    const long long L = Ls[i];
    pass(R, Ls[i] / R, +1, [&](int j, long long* num, long long* den) {
      const long long a[4] = {4LL * j, 2LL * j, (long long)j, 8LL * j + L}, b[4] = {L, L, L, 8 * L};
      const int o = R == 8 ? 0 : 1;
      for (int e = 0; e + o < 4; ++e) {
        num[e] = a[e + o];
        den[e] = b[e + o];
      }
    });
  }
}

// exp(-2 pi i k / n) for k = 0..n-1.  cos/sin are evaluated in long double
// on the first octant and mapped to the others by exact symmetries.
void twiddles(int n, std::vector<double2>& tw) {
  tw.resize(n);
  std::vector<long double> c(n / 8 + 1), s(n / 8 + 1);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int k = 0; k <= n / 8; ++k) {
    const long double a = two_pi * (long double)k / (long double)n;
    c[k] = cosl(a);
    s[k] = sinl(a);
  }
  for (int k = 0; k < n; ++k) {
    long double ck, sk;  // cos, sin of 2 pi k / n
    int kk = k;
    long double sgn_s = 1.0L;
    if (kk > n / 2) {  // angle = 2 pi - angle(n - k)
      kk = n - kk;
      sgn_s = -1.0L;
    }
    long double cb, sb;
    if (kk <= n / 8) {
      cb = c[kk];
      sb = s[kk];
    } else if (kk <= n / 4) {
      cb = s[n / 4 - kk];
      sb = c[n / 4 - kk];
    } else if (kk <= 3 * n / 8) {
      cb = -s[kk - n / 4];
      sb = c[kk - n / 4];
    } else {
      cb = -c[n / 2 - kk];
      sb = s[n / 2 - kk];
    }
    ck = cb;
    sk = sgn_s * sb;
    tw[k] = make_double2((double)ck, (double)(-sk));
  }
}

void default_opts(qg_solver_opts* o) {
  o->tol = 1e-12;
  o->restart = 30;
  o->max_iters = 400;
  o->reorth = 1;
  o->midpoint_epilogue = 0;
  o->true_residual = 0;
  o->inner_tol = 1e-6;
  o->max_outer = 10;
  o->solver = QG_SOLVER_GMRES;
  o->guess = QG_GUESS_EULER;
}

bool valid_opts(const qg_solver_opts& o) {
  return o.tol > 0.0 && o.restart >= 1 && o.restart <= QG_MAX_RESTART && o.max_iters >= 1 &&
         (o.reorth == 0 || o.reorth == 1) && (o.midpoint_epilogue == 0 || o.midpoint_epilogue == 1) &&
         (o.true_residual == 0 || o.true_residual == 1) && o.inner_tol > 0.0 && o.inner_tol < 1.0 &&
         o.max_outer >= 1 && o.max_outer <= 1000 &&
         (o.solver == QG_SOLVER_GMRES || (o.solver == QG_SOLVER_LANCZOS && o.restart >= 4)) &&
         (o.guess == QG_GUESS_EULER || o.guess == QG_GUESS_ZERO);
}

// Composition fractions (Sec. II C) into a fixed array (no heap): order 2 is
// the elementary step; for the recursive schemes each level maps the list L
// of order p to gamma_1 L, ..., gamma_M L with the coefficients of
// Eq. (triple_jump) or Eq. (suzukis_fractal).  QG_OPTIMAL is one
// non-recursive palindrome of Kahan and Li's coefficients (M = 9 for order 6,
// M = 17 for order 8), Suzuki's fractal for order 4.  Returns the count, or 0
// for an invalid order / scheme.
int schedule_fixed(int order, int scheme, double* out) {
  if (order < 2 || order > 8 || (order & 1)) return 0;
  if (scheme != QG_TRIPLE_JUMP && scheme != QG_SUZUKI && scheme != QG_OPTIMAL) return 0;
  if (scheme == QG_OPTIMAL && order >= 6) {
    // Kahan & Li (1997), first half of the palindrome, middle coefficient last
    static const double kl6[5] = {0.39216144400731413927925056, 0.33259913678935943859974864,
                                  -0.70624617255763935980996482, 0.08221359629355080023149045,
                                  0.79854399093482996339895035};
    static const double kl8[9] = {0.13020248308889008087881763,  0.56116298177510838456196441,
                                  -0.38947496264484728640807860, 0.15884190655515560089621075,
                                  -0.39590389413323757733623154, 0.18453964097831570709183254,
                                  0.25837438768632204729397911,  0.29501172360931029887096624,
                                  -0.60550853383003451169892108};
    const double* h = order == 6 ? kl6 : kl8;
    const int half = order == 6 ? 5 : 9, M = 2 * half - 1;
    for (int i = 0; i < M; ++i) out[i] = h[i < half ? i : M - 1 - i];
    return M;
  }
  if (scheme == QG_OPTIMAL) scheme = QG_SUZUKI;
  double tmp[QG_MAX_FRACTIONS];
  int cnt = 1;
  out[0] = 1.0;
  for (int p = 2; p < order; p += 2) {
    double g[5];
    int M;
    if (scheme == QG_TRIPLE_JUMP) {
      const double r = std::pow(2.0, 1.0 / (p + 1));
      g[0] = g[2] = 1.0 / (2.0 - r);
      g[1] = -r / (2.0 - r);
      M = 3;
    } else {
      const double r = std::pow(4.0, 1.0 / (p + 1));
      g[0] = g[1] = g[3] = g[4] = 1.0 / (4.0 - r);
      g[2] = -r / (4.0 - r);
      M = 5;
    }
    if (cnt * M > QG_MAX_FRACTIONS) return 0;
    int k = 0;
    for (int a = 0; a < M; ++a)
      for (int b = 0; b < cnt; ++b) tmp[k++] = g[a] * out[b];
    for (int b = 0; b < k; ++b) out[b] = tmp[b];
    cnt = k;
  }
  return cnt;
}

bool make_schedule(int order, int scheme, std::vector<double>& fr) {
  double buf[QG_MAX_FRACTIONS];
  const int n = schedule_fixed(order, scheme, buf);
  if (n <= 0) return false;
  fr.assign(buf, buf + n);
  return true;
}

InstDesc make_desc(const qg_state* s) {
  const qg_model* m = s->m;
  const qg_grid* g = m->g;
  InstDesc d;
  memset(&d, 0, sizeof(d));
  d.n = g->n[0];
  d.S = m->S;
  d.npass = g->plan[0].npass;
  for (int i = 0; i < QG_MAX_PASSES; ++i) d.radix[i] = g->plan[0].radix[i];
  d.h2m = 1.0 / (2.0 * m->mass[0]);
  d.dq = g->dq[0];
  d.tw = g->d_tw[0];
  d.kd = g->d_kd[0];
  d.lf = g->d_lf[0];
  d.lff = g->d_lff[0];
  d.V = m->d_V;
  d.F = m->d_F;
  d.psi = s->d_psi;
  d.work = s->d_work;
  d.restart_cap = s->restart_cap;
  d.precision = s->precision;
  d.tw32 = g->d_tw32[0];
  d.kd32 = g->d_kd32[0];
  d.V32 = m->d_V32;
  d.F32 = m->d_F32;
  d.work32 = s->d_work32;
  d.rep = m->rep;
  d.ckpt = s->adj.ckpt;
  d.nckpt = s->adj.nckpt;
  d.every = s->adj.every > 0 ? s->adj.every : 1;
  d.grad = s->adj.grad;
  d.gV = s->adj.gV;
  d.gF = s->adj.gF;
  return d;
}

Inst2D make_inst2d(const qg_state* s) {
  const qg_model* m = s->m;
  const qg_grid* g = m->g;
  Inst2D I;
  memset(&I, 0, sizeof(I));
  I.S = m->S;
  I.dv = 1.0;
  for (int d = 0; d < 2; ++d) {
    I.n[d] = g->n[d];
    I.npass[d] = g->plan[d].npass;
    for (int i = 0; i < QG_MAX_PASSES; ++i) I.radix[d][i] = g->plan[d].radix[i];
    I.h2m[d] = 1.0 / (2.0 * m->mass[d]);
    I.dv *= g->dq[d];
    I.tw[d] = g->d_tw[d];
    I.kd[d] = g->d_kd[d];
    I.lf[d] = g->d_lf[d];
    I.lff[d] = g->d_lff[d];
    I.tw32[d] = g->d_tw32[d];
    I.kd32[d] = g->d_kd32[d];
  }
  I.V = m->d_V;
  I.F = m->d_F;
  I.V32 = m->d_V32;
  I.F32 = m->d_F32;
  I.psi = s->d_psi;
  I.work = s->d_work;
  I.work32 = s->d_work32;
  I.precision = s->precision;
  I.bar = reinterpret_cast<unsigned*>(s->d_coop);
  I.err = reinterpret_cast<int*>(s->d_coop + 64);
  I.gred = reinterpret_cast<double*>(s->d_coop + 4096);
  I.ckpt = s->adj.ckpt;
  I.nckpt = s->adj.nckpt;
  I.every = s->adj.every > 0 ? s->adj.every : 1;
  I.ctas = s->launch_ctas;
  return I;
}

double grid_dv(const qg_grid* g) {
  double v = 1.0;
  for (int d = 0; d < g->D; ++d) v *= g->dq[d];
  return v;
}

}  // namespace

extern "C" {
static qg_status build_plan(int method, int order, int scheme, double dt, int64_t nsteps, const qg_solver_opts* opts,
                            StepPlan* P);
}

static qg_status upload_desc(qg_state_t s) {
  InstDesc d = make_desc(s);
  QG_TRY(cudaMemcpyAsync(s->d_inst, &d, sizeof(d), cudaMemcpyHostToDevice, s->stream));
  return QG_OK;
}

extern "C" {

void qg_default_solver_opts(qg_solver_opts* opts) {
  if (opts) default_opts(opts);
}

const char* qg_version(void) { return "qgeom 0.1 (sm_103a)"; }

const char* qg_last_error_string(void) { return g_err; }

const char* qg_status_string(qg_status st) {
  switch (st) {
    case QG_OK: return "ok";
    case QG_ERR_INVALID_ARG: return "invalid argument";
    case QG_ERR_NOT_CONVERGED: return "implicit solve did not converge";
    case QG_ERR_CUDA: return "CUDA error";
    case QG_ERR_OOM: return "out of device memory";
    case QG_ERR_TIMEOUT: return "timeout";
    case QG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

qg_status qg_create_grid(int D, const int* N, const double* qmin, const double* qmax, qg_grid_t* out) {
  if (!out || !N || !qmin || !qmax) return QG_ERR_INVALID_ARG;
  *out = nullptr;
  if (D < 1 || D > QG_MAX_D) return QG_ERR_INVALID_ARG;
  long long tot = 1;
  for (int d = 0; d < D; ++d) {
    if (!is_pow2(N[d]) || N[d] < QG_MIN_N || N[d] > QG_MAX_N) return QG_ERR_INVALID_ARG;
    if (!(qmax[d] > qmin[d]) || !std::isfinite(qmin[d]) || !std::isfinite(qmax[d])) return QG_ERR_INVALID_ARG;
    tot *= N[d];
  }
  if (D == 2 && tot > QG_MAX_2D_POINTS) return QG_ERR_INVALID_ARG;
  qg_grid* g = new (std::nothrow) qg_grid;
  if (!g) return QG_ERR_OOM;
  memset(g, 0, sizeof(*g));
  g->D = D;
  g->ntot = 1;
  cudaGetDevice(&g->device);
  for (int d = 0; d < D; ++d) {
    const int n = N[d];
    g->n[d] = n;
    g->qmin[d] = qmin[d];
    g->qmax[d] = qmax[d];
    g->dq[d] = (qmax[d] - qmin[d]) / n;
    g->ntot *= n;
    g->plan[d] = make_plan(n);
    std::vector<double2> tw_nat, tw;
    twiddles(n, tw_nat);
    pass_twiddles(g->plan[d], tw_nat, tw);
    std::vector<int> f;
    freq_positions(n, g->plan[d].radix, g->plan[d].npass, f);
    std::vector<double> kd(n);
    const double k0 = 2.0 * M_PI / (n * g->dq[d]);
    for (int p = 0; p < n; ++p) {
      const int ff = f[p] < n / 2 ? f[p] : f[p] - n;
      kd[p] = k0 * ff / n;
    }
    std::vector<float2> tw32(n);
    std::vector<float> kd32(n);
    for (int p = 0; p < n; ++p) {
      tw32[p] = make_float2((float)tw[p].x, (float)tw[p].y);
      kd32[p] = (float)kd[p];
    }
    std::vector<double2> lfe;
    std::vector<unsigned> lff;
    lf_tables(g->plan[d], lfe, lff);
    const size_t lf_bytes = lf_table_bytes(n);
    cudaError_t e = cudaMalloc(&g->d_tw[d], sizeof(double2) * n);
    if (e == cudaSuccess && lf_bytes > 0) e = cudaMalloc(&g->d_lf[d], lf_bytes);
    if (e == cudaSuccess && lf_bytes > 0) {
      g->d_lff[d] = reinterpret_cast<unsigned*>(g->d_lf[d] + lfe.size());
      e = cudaMemcpy(g->d_lf[d], lfe.data(), sizeof(double2) * lfe.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(g->d_lff[d], lff.data(), sizeof(unsigned) * lff.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&g->d_kd[d], sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_tw32[d], sizeof(float2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_kd32[d], sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_tw[d], tw.data(), sizeof(double2) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_kd[d], kd.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_tw32[d], tw32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_kd32[d], kd32.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_err("qg_create_grid", e);
      qg_destroy_grid(g);
      return e == cudaErrorMemoryAllocation ? QG_ERR_OOM : QG_ERR_CUDA;
    }
  }
  *out = g;
  return QG_OK;
}

void qg_destroy_grid(qg_grid_t g) {
  if (!g) return;
  for (int d = 0; d < 2; ++d) {
    if (g->d_tw[d]) cudaFree(g->d_tw[d]);
    if (g->d_lf[d]) cudaFree(g->d_lf[d]);
    if (g->d_kd[d]) cudaFree(g->d_kd[d]);
    if (g->d_tw32[d]) cudaFree(g->d_tw32[d]);
    if (g->d_kd32[d]) cudaFree(g->d_kd32[d]);
  }
  delete g;
}

// FP32 copies of the fields for the mixed-precision inner solves.
static cudaError_t finish_model(qg_model* m) {
  const size_t nv = (size_t)m->S * m->g->ntot;
  const size_t nf = (size_t)m->g->D * (m->S * (m->S - 1) / 2) * m->g->ntot;
  cudaError_t e = qg_launch_to_f32(m->d_V, m->d_V32, nv, 0);
  if (e == cudaSuccess) e = qg_launch_to_f32(m->d_F, m->d_F32, nf, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

static qg_status alloc_model(qg_grid_t g, int S, const double* mass, qg_model** out) {
  *out = nullptr;
  if (!g || !mass || S < 2 || S > QG_MAX_S) return QG_ERR_INVALID_ARG;
  for (int d = 0; d < g->D; ++d)
    if (!(mass[d] > 0.0) || !std::isfinite(mass[d])) return QG_ERR_INVALID_ARG;
  qg_model* m = new (std::nothrow) qg_model;
  if (!m) return QG_ERR_OOM;
  memset(m, 0, sizeof(*m));
  m->g = g;
  m->S = S;
  for (int d = 0; d < g->D; ++d) m->mass[d] = mass[d];
  const size_t nv = (size_t)S * g->ntot;
  const size_t nf = (size_t)g->D * (S * (S - 1) / 2) * g->ntot;
  cudaError_t e = cudaMalloc(&m->d_V, sizeof(double) * nv);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_F, sizeof(double) * nf);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_V32, sizeof(float) * nv);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_F32, sizeof(float) * nf);
  if (e != cudaSuccess) {
    set_err("qg_create_model", e);
    qg_destroy_model(m);
    return e == cudaErrorMemoryAllocation ? QG_ERR_OOM : QG_ERR_CUDA;
  }
  *out = m;
  return QG_OK;
}

qg_status qg_create_model(qg_grid_t g, int S, const double* mass, const double* V, const double* F, int on_device,
                          qg_model_t* out) {
  if (!out || !V || !F) return QG_ERR_INVALID_ARG;
  qg_model* m;
  qg_status st = alloc_model(g, S, mass, &m);
  if (st != QG_OK) return st;
  const size_t nv = (size_t)S * g->ntot;
  const size_t nf = (size_t)g->D * (S * (S - 1) / 2) * g->ntot;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpy(m->d_V, V, sizeof(double) * nv, k);
  if (e == cudaSuccess) e = cudaMemcpy(m->d_F, F, sizeof(double) * nf, k);
  if (e == cudaSuccess) e = finish_model(m);
  if (e != cudaSuccess) {
    set_err("qg_create_model", e);
    qg_destroy_model(m);
    return QG_ERR_CUDA;
  }
  *out = m;
  return QG_OK;
}

qg_status qg_create_model_diabatic(qg_grid_t g, int S, const double* mass, const double* W, const double* dW,
                                   int on_device, qg_model_t* out) {
  if (!out || !W || !dW) return QG_ERR_INVALID_ARG;
  if (g && g->D != 1 && S != 2) return QG_ERR_UNSUPPORTED;
  qg_model* m;
  qg_status st = alloc_model(g, S, mass, &m);
  if (st != QG_OK) return st;
  const int n = g->ntot;
  const size_t nw = (size_t)(S * (S + 1) / 2) * n;
  const size_t ndw = nw * g->D;
  double *dWd = nullptr, *ddW = nullptr, *dvec = nullptr;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    e = cudaMalloc(&dWd, sizeof(double) * nw);
    if (e == cudaSuccess) e = cudaMalloc(&ddW, sizeof(double) * ndw);
    if (e == cudaSuccess) e = cudaMemcpy(dWd, W, sizeof(double) * nw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ddW, dW, sizeof(double) * ndw, cudaMemcpyHostToDevice);
  }
  const double* w = on_device ? W : dWd;
  const double* dw = on_device ? dW : ddW;
  // O(q) is kept for the changes of representation (Eq. psi_diab2adiab)
  if (e == cudaSuccess) e = cudaMalloc(&dvec, sizeof(double) * (size_t)S * S * n);
  if (e == cudaSuccess) {
    if (S == 2)
      e = qg_launch_fields2(w, dw, n, g->D, m->d_V, m->d_F, dvec, 0);
    else
      e = qg_launch_fieldsS(w, dw, n, S, m->d_V, m->d_F, dvec, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = finish_model(m);
  if (dWd) cudaFree(dWd);
  if (ddW) cudaFree(ddW);
  if (e == cudaSuccess) {
    m->d_O = dvec;
  } else if (dvec) {
    cudaFree(dvec);
  }
  if (e != cudaSuccess) {
    set_err("qg_create_model_diabatic", e);
    qg_destroy_model(m);
    return QG_ERR_CUDA;
  }
  *out = m;
  return QG_OK;
}

qg_status qg_create_model_diabatic_rep(qg_grid_t g, int S, const double* mass, const double* W, int on_device,
                                       qg_model_t* out) {
  if (!out || !W) return QG_ERR_INVALID_ARG;
  if (g && g->D != 1) return QG_ERR_UNSUPPORTED;
  qg_model* m;
  qg_status st = alloc_model(g, S, mass, &m);
  if (st != QG_OK) return st;
  const int n = g->ntot;
  const size_t nw = (size_t)(S * (S + 1) / 2) * n;
  double* dWd = nullptr;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    e = cudaMalloc(&dWd, sizeof(double) * nw);
    if (e == cudaSuccess) e = cudaMemcpy(dWd, W, sizeof(double) * nw, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = qg_launch_diabatic_fields(on_device ? W : dWd, n, S, m->d_V, m->d_F, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = finish_model(m);
  if (dWd) cudaFree(dWd);
  if (e != cudaSuccess) {
    set_err("qg_create_model_diabatic_rep", e);
    qg_destroy_model(m);
    return QG_ERR_CUDA;
  }
  m->rep = 1;
  *out = m;
  return QG_OK;
}

static qg_status rotate_state(qg_model_t m, const void* in, void* out, int on_device, int to_adiabatic) {
  if (!m || !in || !out) return QG_ERR_INVALID_ARG;
  if (!m->d_O || m->g->D != 1) return QG_ERR_UNSUPPORTED;
  const int n = m->g->ntot, S = m->S;
  const size_t bytes = sizeof(double2) * (size_t)S * n;
  double2 *di = nullptr, *dout = nullptr;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    e = cudaMalloc(&di, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dout, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(di, in, bytes, cudaMemcpyHostToDevice);
  }
  const double2* src = on_device ? (const double2*)in : di;
  double2* dst = on_device ? (double2*)out : dout;
  double2* tmp = nullptr;
  if (e == cudaSuccess && on_device && src == dst) {   // in place: rotate into a copy
    e = cudaMalloc(&tmp, bytes);
    if (e == cudaSuccess) dst = tmp;
  }
  if (e == cudaSuccess) e = qg_launch_rotate(m->d_O, src, dst, n, S, to_adiabatic, 0);
  if (e == cudaSuccess && tmp) e = cudaMemcpy(out, tmp, bytes, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && !on_device) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (di) cudaFree(di);
  if (dout) cudaFree(dout);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) {
    set_err("representation change", e);
    return QG_ERR_CUDA;
  }
  return QG_OK;
}

qg_status qg_diabatic_to_adiabatic(qg_model_t m, const void* psi_diab, void* psi_adiab, int on_device) {
  return rotate_state(m, psi_diab, psi_adiab, on_device, 1);
}

qg_status qg_adiabatic_to_diabatic(qg_model_t m, const void* psi_adiab, void* psi_diab, int on_device) {
  return rotate_state(m, psi_adiab, psi_diab, on_device, 0);
}

qg_status qg_interpolate(qg_state_t src, qg_state_t dst) {
  if (!src || !dst) return QG_ERR_INVALID_ARG;
  const qg_grid* gs = src->m->g;
  const qg_grid* gd = dst->m->g;
  if (gs->D != 1 || gd->D != 1) return QG_ERR_UNSUPPORTED;
  if (src->m->S != dst->m->S) return QG_ERR_INVALID_ARG;
  const int S = src->m->S;
  double2* coef = nullptr;
  cudaError_t e = cudaStreamSynchronize(src->stream);
  if (e == cudaSuccess) e = cudaMalloc(&coef, sizeof(double2) * (size_t)S * gs->n[0]);
  if (e == cudaSuccess)
    e = qg_launch_interpolate(src->d_psi, gs->n[0], gs->qmin[0], gs->qmax[0] - gs->qmin[0], coef, dst->d_psi,
                              gd->n[0], gd->qmin[0], gd->dq[0], S, dst->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(dst->stream);
  if (coef) cudaFree(coef);
  if (e != cudaSuccess) {
    set_err("qg_interpolate", e);
    return QG_ERR_CUDA;
  }
  return QG_OK;
}

qg_status qg_model_fields(qg_model_t m, double* V, double* F, int on_device) {
  if (!m) return QG_ERR_INVALID_ARG;
  const size_t nv = (size_t)m->S * m->g->ntot;
  const size_t nf = (size_t)m->g->D * (m->S * (m->S - 1) / 2) * m->g->ntot;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (V) QG_TRY(cudaMemcpy(V, m->d_V, sizeof(double) * nv, k));
  if (F) QG_TRY(cudaMemcpy(F, m->d_F, sizeof(double) * nf, k));
  return QG_OK;
}

void qg_destroy_model(qg_model_t m) {
  if (!m) return;
  if (m->d_V) cudaFree(m->d_V);
  if (m->d_F) cudaFree(m->d_F);
  if (m->d_V32) cudaFree(m->d_V32);
  if (m->d_F32) cudaFree(m->d_F32);
  if (m->d_O) cudaFree(m->d_O);
  delete m;
}

qg_status qg_create_state(qg_model_t m, int precision, qg_state_t* out) {
  if (!out || !m) return QG_ERR_INVALID_ARG;
  *out = nullptr;
  if (precision != QG_C128 && precision != QG_C64_MIXED) return QG_ERR_INVALID_ARG;
  qg_state* s = new (std::nothrow) qg_state;
  if (!s) return QG_ERR_OOM;
  memset(s, 0, sizeof(*s));
  s->m = m;
  s->restart_cap = QG_MAX_RESTART;
  s->precision = precision;
  s->stream = 0;
  const size_t len = (size_t)m->S * m->g->ntot;
  cudaError_t e = cudaMalloc(&s->d_psi, sizeof(double2) * len);
  if (e == cudaSuccess) e = cudaMemset(s->d_psi, 0, sizeof(double2) * len);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_work, sizeof(double2) * len * (size_t)(s->restart_cap + 5));
  if (e == cudaSuccess && precision == QG_C64_MIXED)
    e = cudaMalloc(&s->d_work32, sizeof(float2) * len * (size_t)(s->restart_cap + 4));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_stats, sizeof(qg_step_stats));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_scalars, sizeof(double) * 64);
  if (e == cudaSuccess && m->g->D == 2) e = cudaMalloc(&s->d_coop, 4096 + sizeof(double) * 2 * 1024 * 32);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_inst, sizeof(InstDesc));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_counter, sizeof(int));
  if (e != cudaSuccess) {
    set_err("qg_create_state", e);
    qg_destroy_state(s);
    return e == cudaErrorMemoryAllocation ? QG_ERR_OOM : QG_ERR_CUDA;
  }
  qg_status st = upload_desc(s);
  if (st == QG_OK) {
    cudaError_t e2 = cudaStreamSynchronize(s->stream);
    if (e2 != cudaSuccess) {
      set_err("qg_create_state", e2);
      st = QG_ERR_CUDA;
    }
  }
  if (st != QG_OK) {
    qg_destroy_state(s);
    return st;
  }
  *out = s;
  return QG_OK;
}

void qg_destroy_state(qg_state_t s) {
  if (!s) return;
  if (s->d_psi) cudaFree(s->d_psi);
  if (s->d_work) cudaFree(s->d_work);
  if (s->d_work32) cudaFree(s->d_work32);
  if (s->d_coop) cudaFree(s->d_coop);
  if (s->d_stats) cudaFree(s->d_stats);
  if (s->d_scalars) cudaFree(s->d_scalars);
  if (s->d_inst) cudaFree(s->d_inst);
  if (s->d_counter) cudaFree(s->d_counter);
  delete s;
}

qg_status qg_state_set_cluster(qg_state_t s, int G) {
  if (!s || G < 0) return QG_ERR_INVALID_ARG;
  if (G > 0) {
    const qg_grid* g = s->m->g;
    if (g->D != 1 || s->precision != QG_C128 || s->m->rep) return QG_ERR_UNSUPPORTED;
    if (qg_cluster_smem(g->n[0], s->m->S, G, 4) == 0) return QG_ERR_UNSUPPORTED;
  }
  s->cluster = G;
  return QG_OK;
}

qg_status qg_state_set_launch_width(qg_state_t s, int ctas) {
  if (!s || ctas < 0) return QG_ERR_INVALID_ARG;
  s->launch_ctas = ctas;
  return QG_OK;
}

qg_status qg_state_autotune(qg_state_t s, int method, int order, int scheme, double dt, int64_t trial_steps,
                            const qg_solver_opts* opts, double* ms_out) {
  if (!s || trial_steps < 1) return QG_ERR_INVALID_ARG;
  if (s->m->g->D != 2) return QG_OK;   // 1-D states run on one CTA: nothing to tune
  StepPlan P;
  qg_status st = build_plan(method, order, scheme, dt, trial_steps, opts, &P);
  if (st != QG_OK) return st;
  if (P.restart > QG_MAX_RESTART - 1) return QG_ERR_UNSUPPORTED;
  const size_t len = (size_t)s->m->S * s->m->g->ntot;
  double2* save = nullptr;
  QG_TRY(cudaMalloc(&save, sizeof(double2) * len));
  s->launch_ctas = 0;
  const int gmax = qg_grid2d_ctas(make_inst2d(s));
  const int cand[3] = {gmax, gmax / 2 > 0 ? gmax / 2 : 1, gmax / 4 > 0 ? gmax / 4 : 1};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(save, s->d_psi, sizeof(double2) * len, cudaMemcpyDeviceToDevice, s->stream);
  double best = 1e300;
  int bi = 0;
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
    s->launch_ctas = cand[c];
    e = cudaEventRecord(e0, s->stream);
    if (e == cudaSuccess) e = qg_launch_propagate2d(make_inst2d(s), P, s->d_stats, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = -1.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out) ms_out[c] = ms;
    if (ms > 0.f && ms < best) {
      best = ms;
      bi = c;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->d_psi, save, sizeof(double2) * len, cudaMemcpyDeviceToDevice, s->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(save);
  if (e != cudaSuccess) {
    set_err("qg_state_autotune", e);
    return QG_ERR_CUDA;
  }
  s->launch_ctas = cand[bi];
  return QG_OK;
}

qg_status qg_state_set_stream(qg_state_t s, void* stream) {
  if (!s) return QG_ERR_INVALID_ARG;
  s->stream = (cudaStream_t)stream;
  return QG_OK;
}

qg_status qg_set_state(qg_state_t s, const void* psi, int on_device) {
  if (!s || !psi) return QG_ERR_INVALID_ARG;
  const size_t bytes = sizeof(double2) * (size_t)s->m->S * s->m->g->ntot;
  QG_TRY(cudaMemcpyAsync(s->d_psi, psi, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         s->stream));
  if (!on_device) QG_TRY(cudaStreamSynchronize(s->stream));
  return QG_OK;
}

qg_status qg_get_state(qg_state_t s, void* psi, int on_device) {
  if (!s || !psi) return QG_ERR_INVALID_ARG;
  const size_t bytes = sizeof(double2) * (size_t)s->m->S * s->m->g->ntot;
  QG_TRY(cudaMemcpyAsync(psi, s->d_psi, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         s->stream));
  if (!on_device) QG_TRY(cudaStreamSynchronize(s->stream));
  return QG_OK;
}

qg_status qg_set_gaussian(qg_state_t s, int surface, const double* q0, const double* p0, const double* sigma0) {
  if (!s || !q0 || !p0 || !sigma0) return QG_ERR_INVALID_ARG;
  const qg_grid* g = s->m->g;
  if (surface < 0 || surface >= s->m->S) return QG_ERR_INVALID_ARG;
  for (int d = 0; d < g->D; ++d)
    if (!(sigma0[d] > 0.0) || !std::isfinite(q0[d]) || !std::isfinite(p0[d])) return QG_ERR_INVALID_ARG;
  if (g->D == 2) {
    QG_TRY(qg_launch_gaussian2d(s->d_psi, g->n, s->m->S, surface, g->qmin, g->dq, q0, p0, sigma0, s->stream));
    return QG_OK;
  }
  QG_TRY(qg_launch_gaussian(s->d_psi, g->n[0], s->m->S, surface, g->qmin[0], g->dq[0], q0[0], p0[0], sigma0[0],
                            s->stream));
  return QG_OK;
}

qg_status qg_apply_h(qg_state_t s, void* out, int on_device) {
  if (!s || !out) return QG_ERR_INVALID_ARG;
  const qg_grid* g = s->m->g;
  const size_t len = (size_t)s->m->S * g->ntot;
  double2* dst = on_device ? (double2*)out : s->d_work + 2 * len;  // B slot as staging
  if (g->D == 2) {
    QG_TRY(qg_launch_apply_h2d(make_inst2d(s), dst, nullptr, s->stream));
  } else {
    QG_TRY(qg_launch_apply_h(s->d_inst, dst, g->n[0], s->m->S, s->stream));
  }
  if (!on_device) {
    QG_TRY(cudaMemcpyAsync(out, dst, sizeof(double2) * len, cudaMemcpyDeviceToHost, s->stream));
    QG_TRY(cudaStreamSynchronize(s->stream));
  }
  return QG_OK;
}

static qg_status build_plan(int method, int order, int scheme, double dt, int64_t nsteps, const qg_solver_opts* opts,
                            StepPlan* P) {
  qg_solver_opts o;
  default_opts(&o);
  if (opts) o = *opts;
  if (!valid_opts(o)) return QG_ERR_INVALID_ARG;
  if (method < QG_TRAPEZOIDAL || method > QG_SOD) return QG_ERR_INVALID_ARG;
  if (!std::isfinite(dt) || nsteps < 0) return QG_ERR_INVALID_ARG;
  std::vector<double> fr;
  if (method >= QG_EXPLICIT_EULER) {
    // the elementary comparison methods: one step of size dt, never composed
    if (order != (method == QG_SOD ? 2 : 1)) return QG_ERR_INVALID_ARG;
    fr.assign(1, 1.0);
  } else if (!make_schedule(order, scheme, fr)) {
    return QG_ERR_INVALID_ARG;
  }
  memset(P, 0, sizeof(*P));
  P->method = method;
  P->nfrac = (int)fr.size();
  for (size_t i = 0; i < fr.size(); ++i) P->frac[i] = fr[i];
  P->dt = dt;
  P->nsteps = nsteps;
  P->tol = o.tol;
  P->restart = o.restart;
  P->max_iters = o.max_iters;
  P->reorth = o.reorth;
  P->mid_epi = o.midpoint_epilogue;
  P->true_res = o.true_residual;
  P->inner_tol = o.inner_tol;
  P->max_outer = o.max_outer;
  P->solver = o.solver;
  P->guess = o.guess;
  return QG_OK;
}

static qg_status check_run(int run, const StepPlan& P, const qg_state* s) {
  if (run != QG_RUN_FORWARD && run != QG_RUN_CHECKPOINT && run != QG_RUN_ADJOINT) return QG_ERR_INVALID_ARG;
  if (run == QG_RUN_CHECKPOINT && (!s->adj.ckpt || s->adj.every < 1 || s->adj.nckpt < 1)) return QG_ERR_INVALID_ARG;
  if (run == QG_RUN_ADJOINT &&
      (!s->adj.grad || !s->adj.gV || !s->adj.gF || P.restart > QG_MAX_RESTART - 4 || s->adj.every < 1 ||
       P.method >= QG_EXPLICIT_EULER || s->m->rep))
    return QG_ERR_INVALID_ARG;
  return QG_OK;
}

qg_status qg_state_set_adjoint(qg_state_t s, void* checkpoints, int64_t ncheckpoints, int64_t every, void* grad,
                               double* grad_V, double* grad_F) {
  if (!s || every < 1 || ncheckpoints < 0 || (ncheckpoints > 0 && !checkpoints)) return QG_ERR_INVALID_ARG;
  s->adj.ckpt = (double2*)checkpoints;
  s->adj.nckpt = ncheckpoints;
  s->adj.every = every;
  s->adj.grad = (double2*)grad;
  s->adj.gV = grad_V;
  s->adj.gF = grad_F;
  return upload_desc(s);
}

qg_status qg_propagate_ex(qg_state_t s, int run, int method, int order, int scheme, double dt, int64_t nsteps,
                          const qg_solver_opts* opts, qg_step_stats* stats) {
  if (!s) return QG_ERR_INVALID_ARG;
  StepPlan P;
  qg_status st = build_plan(method, order, scheme, dt, nsteps, opts, &P);
  if (st != QG_OK) return st;
  st = check_run(run, P, s);
  if (st != QG_OK) return st;
  P.run = run;
  const qg_grid* g = s->m->g;
  if (g->D == 2) {
    if (run == QG_RUN_ADJOINT || P.restart > QG_MAX_RESTART - 1) return QG_ERR_UNSUPPORTED;
    QG_TRY(qg_launch_propagate2d(make_inst2d(s), P, s->d_stats, s->stream));
  } else if (s->cluster > 0 && run == QG_RUN_FORWARD) {
    const size_t smem = qg_cluster_smem(g->n[0], s->m->S, s->cluster, P.restart);
    if (smem == 0) return QG_ERR_UNSUPPORTED;
    QG_TRY(qg_launch_cluster(s->cluster, s->d_inst, 1, P, s->d_stats, smem, s->stream));
  } else {
    QG_TRY(qg_launch_propagate(s->d_inst, 1, P, s->d_counter, s->d_stats, g->n[0], s->m->S, s->stream));
  }
  qg_step_stats h;
  QG_TRY(cudaMemcpyAsync(&h, s->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  QG_TRY(cudaStreamSynchronize(s->stream));
  if (stats) *stats = h;
  return (qg_status)h.status;
}

qg_status qg_propagate(qg_state_t s, int method, int order, int scheme, double dt, int64_t nsteps,
                       const qg_solver_opts* opts, qg_step_stats* stats) {
  if (!s) return QG_ERR_INVALID_ARG;
  StepPlan P;
  qg_status st = build_plan(method, order, scheme, dt, nsteps, opts, &P);
  if (st != QG_OK) return st;
  const qg_grid* g = s->m->g;
  if (g->D == 2) {
    if (P.restart > QG_MAX_RESTART - 1) return QG_ERR_UNSUPPORTED;
    QG_TRY(qg_launch_propagate2d(make_inst2d(s), P, s->d_stats, s->stream));
  } else if (s->cluster > 0) {
    const size_t smem = qg_cluster_smem(g->n[0], s->m->S, s->cluster, P.restart);
    if (smem == 0) return QG_ERR_UNSUPPORTED;
    QG_TRY(qg_launch_cluster(s->cluster, s->d_inst, 1, P, s->d_stats, smem, s->stream));
  } else {
    QG_TRY(qg_launch_propagate(s->d_inst, 1, P, s->d_counter, s->d_stats, g->n[0], s->m->S, s->stream));
  }
  qg_step_stats h;
  QG_TRY(cudaMemcpyAsync(&h, s->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  QG_TRY(cudaStreamSynchronize(s->stream));
  if (stats) *stats = h;
  return (qg_status)h.status;
}

qg_status qg_step_implicit(qg_state_t s, int method, int order, int scheme, double dt, const qg_solver_opts* opts,
                           qg_step_stats* stats) {
  return qg_propagate(s, method, order, scheme, dt, 1, opts, stats);
}

qg_status qg_batch_create(qg_state_t* states, int nstates, qg_batch_t* out) {
  if (!out || !states || nstates < 1) return QG_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < nstates; ++i) {
    if (!states[i]) return QG_ERR_INVALID_ARG;
    if (states[i]->m->g->D != 1) return QG_ERR_UNSUPPORTED;
  }
  qg_batch* b = new (std::nothrow) qg_batch;
  if (!b) return QG_ERR_OOM;
  memset(b, 0, sizeof(*b));
  b->n = nstates;
  b->stream = states[0]->stream;
  b->order = new (std::nothrow) int[nstates];
  if (!b->order) {
    delete b;
    return QG_ERR_OOM;
  }
  std::vector<InstDesc> descs(nstates);
  std::vector<double> cost(nstates);
  b->all_fp64 = 1;
  std::vector<int> ns(nstates), ss(nstates);
  for (int i = 0; i < nstates; ++i) {
    const InstDesc d = make_desc(states[i]);
    if (d.n > b->max_n) b->max_n = d.n;
    if (d.S > b->max_S) b->max_S = d.S;
    if (d.precision != QG_C128 || d.rep) b->all_fp64 = 0;   // the cluster form is adiabatic FP64 only
    ns[i] = d.n;
    ss[i] = d.S;
    // work estimate of one H psi: S transforms of n log2 n
    cost[i] = (double)d.S * d.n * (ilog2h(d.n) + 1);
    b->order[i] = i;
  }
  b->adjoint_ready = true;
  for (int i = 0; i < nstates; ++i) {
    const qg_state_adjoint& ad = states[i]->adj;
    if (!ad.grad || !ad.gV || !ad.gF || !ad.ckpt || ad.nckpt < 1 || ad.every < 1 || states[i]->m->rep)
      b->adjoint_ready = false;
  }
  // grid-size classes, largest N first; within a class longest estimated
  // work first, so the persistent CTAs of a class launch finish together
  std::stable_sort(b->order, b->order + nstates, [&](int x, int y) {
    if (ns[x] != ns[y]) return ns[x] > ns[y];
    return cost[x] > cost[y];
  });
  b->nclass = 0;
  for (int k = 0; k < nstates; ++k) {
    const int i = b->order[k];
    const int c = b->nclass;
    if (k == 0 || ns[i] != b->cls_n[c - 1]) {
      if (c == QG_MAX_CLASSES) {
        delete[] b->order;
        delete b;
        return QG_ERR_UNSUPPORTED;
      }
      b->cls_start[c] = k;
      b->cls_count[c] = 0;
      b->cls_n[c] = ns[i];
      b->cls_S[c] = 0;
      b->cls_ctas[c] = 1;
      b->cls_nb[c] = 0;
      b->cls_cluster[c] = 0;
      b->nclass++;
    }
    const int cc = b->nclass - 1;
    b->cls_count[cc]++;
    if (ss[i] > b->cls_S[cc]) b->cls_S[cc] = ss[i];
  }
  for (int k = 0; k < nstates; ++k) descs[k] = make_desc(states[b->order[k]]);
  cudaError_t e = cudaSuccess;
  if (b->stream == 0) {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamDefault);
    b->own_stream = (e == cudaSuccess);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_desc, sizeof(InstDesc) * nstates);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_stats, sizeof(qg_step_stats) * nstates);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int) * QG_MAX_CLASSES);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int c = 0; c < b->nclass && e == cudaSuccess; ++c) {
    e = cudaStreamCreateWithFlags(&b->cls_stream[c], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->cls_done[c], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_stats, sizeof(qg_step_stats) * nstates);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_desc, descs.data(), sizeof(InstDesc) * nstates, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_err("qg_batch_create", e);
    qg_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? QG_ERR_OOM : QG_ERR_CUDA;
  }
  *out = b;
  return QG_OK;
}

void qg_batch_destroy(qg_batch_t b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_stats) cudaFree(b->d_stats);
  if (b->d_counter) cudaFree(b->d_counter);
  for (int c = 0; c < QG_MAX_CLASSES; ++c) {
    if (b->cls_stream[c]) cudaStreamDestroy(b->cls_stream[c]);
    if (b->cls_done[c]) cudaEventDestroy(b->cls_done[c]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->h_stats) cudaFreeHost(b->h_stats);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete[] b->order;
  delete b;
}

static qg_status batch_collect(qg_batch_t b, int32_t* statuses, qg_step_stats* stats) {
  QG_TRY(cudaMemcpyAsync(b->h_stats, b->d_stats, sizeof(qg_step_stats) * b->n, cudaMemcpyDeviceToHost, b->stream));
  QG_TRY(cudaStreamSynchronize(b->stream));
  qg_status ret = QG_OK;
  for (int k = 0; k < b->n; ++k) {
    const int i = b->order[k];
    if (statuses) statuses[i] = b->h_stats[k].status;
    if (stats) stats[i] = b->h_stats[k];
    if (b->h_stats[k].status != QG_OK) ret = QG_ERR_NOT_CONVERGED;
  }
  return ret;
}

// Dynamic shared memory of class c in the cluster form of size G (0 if an
// instance of the class does not fit).
static size_t class_cluster_smem(const qg_batch* b, int c, int G, int restart) {
  if (!b->all_fp64) return 0;
  size_t best = 0;
  for (int S = 2; S <= b->cls_S[c]; ++S) {
    const size_t t = qg_cluster_smem(b->cls_n[c], S, G, restart);
    if (t == 0) return 0;
    best = std::max(best, t);
  }
  return best;
}

// The persistent launch of one class with a given shape (the cluster form
// for forward runs when cluster > 0, else the one-CTA form).  ninst = 0 only
// sets function attributes.
static cudaError_t class_launch(qg_batch* b, int c, const StepPlan& P, bool all, int ctas_per_sm, int nb_pref,
                                int cluster, cudaStream_t stream) {
  const InstDesc* d = b->d_desc + b->cls_start[c];
  qg_step_stats* st = b->d_stats + b->cls_start[c];
  const int ninst = all ? b->cls_count[c] : 0;
  if (cluster > 0 && P.run == QG_RUN_FORWARD) {
    const size_t smem = class_cluster_smem(b, c, cluster, P.restart);
    if (smem == 0) return cudaErrorInvalidConfiguration;
    return qg_launch_cluster(cluster, d, ninst, P, st, smem, stream);
  }
  return qg_launch_propagate_tuned(d, ninst, P, b->d_counter + c, st, b->cls_n[c], b->cls_S[c], ctas_per_sm, nb_pref,
                                   stream);
}

// Every class, one persistent launch each: a single class runs in the
// batch's stream; several run concurrently in their own streams, forked from
// and joined back into the batch's stream, so that one class's tail overlaps
// the others' work.
static cudaError_t batch_launch(qg_batch* b, const StepPlan& P, bool all) {
  if (b->nclass == 1 || !all)
    for (int c = 0; c < b->nclass; ++c) {
      const cudaError_t e = class_launch(b, c, P, all, b->cls_ctas[c], b->cls_nb[c], b->cls_cluster[c], b->stream);
      if (e != cudaSuccess) return e;
    }
  if (b->nclass == 1 || !all) return cudaSuccess;
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (int c = 0; c < b->nclass && e == cudaSuccess; ++c) {
    e = cudaStreamWaitEvent(b->cls_stream[c], b->fork, 0);
    if (e == cudaSuccess)
      e = class_launch(b, c, P, all, b->cls_ctas[c], b->cls_nb[c], b->cls_cluster[c], b->cls_stream[c]);
    if (e == cudaSuccess) e = cudaEventRecord(b->cls_done[c], b->cls_stream[c]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->cls_done[c], 0);
  }
  return e;
}

qg_status qg_batch_run(qg_batch_t b, int method, int order, int scheme, double dt, int64_t nsteps,
                       const qg_solver_opts* opts, int32_t* statuses, qg_step_stats* stats) {
  if (!b) return QG_ERR_INVALID_ARG;
  StepPlan P;
  qg_status st = build_plan(method, order, scheme, dt, nsteps, opts, &P);
  if (st != QG_OK) return st;
  QG_TRY(batch_launch(b, P, true));
  return batch_collect(b, statuses, stats);
}

qg_status qg_batch_run_ex(qg_batch_t b, int run, int method, int order, int scheme, double dt, int64_t nsteps,
                          const qg_solver_opts* opts, int32_t* statuses, qg_step_stats* stats) {
  if (!b) return QG_ERR_INVALID_ARG;
  StepPlan P;
  qg_status st = build_plan(method, order, scheme, dt, nsteps, opts, &P);
  if (st != QG_OK) return st;
  if (run != QG_RUN_FORWARD && run != QG_RUN_CHECKPOINT && run != QG_RUN_ADJOINT) return QG_ERR_INVALID_ARG;
  if (run == QG_RUN_ADJOINT && P.restart > QG_MAX_RESTART - 4) return QG_ERR_INVALID_ARG;
  if (run != QG_RUN_FORWARD && !b->adjoint_ready) return QG_ERR_INVALID_ARG;
  P.run = run;
  QG_TRY(batch_launch(b, P, true));
  return batch_collect(b, statuses, stats);
}

qg_status qg_batch_capture(qg_batch_t b, int method, int order, int scheme, double dt, int64_t nsteps,
                           const qg_solver_opts* opts) {
  if (!b) return QG_ERR_INVALID_ARG;
  StepPlan P;
  qg_status st = build_plan(method, order, scheme, dt, nsteps, opts, &P);
  if (st != QG_OK) return st;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  // function attributes are set here, outside the capture, by a zero-instance
  // launch that the kernel leaves immediately
  QG_TRY(batch_launch(b, P, false));
  QG_TRY(cudaStreamSynchronize(b->stream));
  cudaGraph_t g = nullptr;
  QG_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = batch_launch(b, P, true);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_err("qg_batch_capture", e);
    b->graph = nullptr;
    return QG_ERR_CUDA;
  }
  return QG_OK;
}

qg_status qg_batch_autotune(qg_batch_t b, int method, int order, int scheme, double dt, int64_t trial_steps,
                            const qg_solver_opts* opts, double* ms_out /* 6 entries or NULL */) {
  if (!b || trial_steps < 1) return QG_ERR_INVALID_ARG;
  StepPlan P;
  qg_status st = build_plan(method, order, scheme, dt, trial_steps, opts, &P);
  if (st != QG_OK) return st;
  // save every state, time each candidate launch shape of each grid-size
  // class on the class's own instances, restore the states after each trial
  std::vector<InstDesc> descs(b->n);
  QG_TRY(cudaMemcpy(descs.data(), b->d_desc, sizeof(InstDesc) * b->n, cudaMemcpyDeviceToHost));
  size_t total = 0;
  for (const InstDesc& d : descs) total += (size_t)d.S * d.n;
  double2* save = nullptr;
  QG_TRY(cudaMalloc(&save, sizeof(double2) * total));
  auto copy_class = [&](int c, bool to_save) -> cudaError_t {
    size_t off = 0;
    for (int k = 0; k < b->n; ++k) {
      const InstDesc& d = descs[k];
      const size_t len = (size_t)d.S * d.n;
      if (c < 0 || (k >= b->cls_start[c] && k < b->cls_start[c] + b->cls_count[c])) {
        cudaError_t e = to_save ? cudaMemcpyAsync(save + off, d.psi, sizeof(double2) * len,
                                                  cudaMemcpyDeviceToDevice, b->stream)
                                : cudaMemcpyAsync(d.psi, save + off, sizeof(double2) * len,
                                                  cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) return e;
      }
      off += len;
    }
    return cudaSuccess;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = copy_class(-1, true);
  for (int c = 0; c < b->nclass && e == cudaSuccess; ++c) {
    // {CTAs per SM, surfaces per FFT batch, cluster size}: the one-CTA form
    // in four shapes, then the cluster form at the smallest cluster size that
    // holds the class and at twice that size
    int g0 = 0;
    for (int G = 1; G <= 16 && !g0; G *= 2)
      if (class_cluster_smem(b, c, G, P.restart) > 0) g0 = G;
    const int cand[6][3] = {{1, 0, 0}, {1, 1, 0}, {2, 0, 0}, {2, 1, 0}, {1, 0, g0},
                            {1, 0, g0 > 0 && g0 < 16 ? 2 * g0 : 0}};
    double best = 1e300;
    int bi = 0;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
      float ms = -1.f;
      if (k >= 4 && (cand[k][2] == 0 || class_cluster_smem(b, c, cand[k][2], P.restart) == 0)) {
        if (ms_out && c == 0) ms_out[k] = -1.0;
        continue;
      }
      e = cudaEventRecord(e0, b->stream);
      cudaError_t el = class_launch(b, c, P, true, cand[k][0], cand[k][1], cand[k][2], b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (el == cudaSuccess && e == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
      } else if (el == cudaErrorInvalidConfiguration) {
        cudaGetLastError();   // shape does not fit: skip it
        ms = -1.f;
      } else if (e == cudaSuccess) {
        e = el;
      }
      if (ms_out && c == 0) ms_out[k] = ms;
      if (ms > 0.f && ms < best) {
        best = ms;
        bi = k;
      }
      if (e == cudaSuccess) e = copy_class(c, false);
    }
    b->cls_ctas[c] = cand[bi][0];
    b->cls_nb[c] = cand[bi][1];
    b->cls_cluster[c] = cand[bi][2];
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(save);
  if (e != cudaSuccess) {
    set_err("qg_batch_autotune", e);
    return QG_ERR_CUDA;
  }
  if (b->graph) {   // a captured graph used the old launch shapes
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return QG_OK;
}

qg_status qg_batch_tuning(qg_batch_t b, int* ctas_per_sm, int* surfaces_per_fft) {
  if (!b) return QG_ERR_INVALID_ARG;
  if (ctas_per_sm) *ctas_per_sm = b->cls_ctas[0];
  if (surfaces_per_fft) *surfaces_per_fft = b->cls_nb[0];
  return QG_OK;
}

qg_status qg_batch_classes(qg_batch_t b, int* nclass, int* grid_n, int* count, int* ctas_per_sm,
                           int* surfaces_per_fft, int* cluster) {
  if (!b || !nclass) return QG_ERR_INVALID_ARG;
  *nclass = b->nclass;
  for (int c = 0; c < b->nclass; ++c) {
    if (grid_n) grid_n[c] = b->cls_n[c];
    if (count) count[c] = b->cls_count[c];
    if (ctas_per_sm) ctas_per_sm[c] = b->cls_ctas[c];
    if (surfaces_per_fft) surfaces_per_fft[c] = b->cls_nb[c];
    if (cluster) cluster[c] = b->cls_cluster[c];
  }
  return QG_OK;
}

qg_status qg_batch_set_cluster(qg_batch_t b, int G) {
  if (!b || G < 0) return QG_ERR_INVALID_ARG;
  for (int c = 0; c < b->nclass && G > 0; ++c)
    if (class_cluster_smem(b, c, G, QG_MAX_RESTART) == 0 && class_cluster_smem(b, c, G, 4) == 0)
      return QG_ERR_UNSUPPORTED;
  for (int c = 0; c < b->nclass; ++c) b->cls_cluster[c] = G;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return QG_OK;
}

qg_status qg_batch_cluster(qg_batch_t b, int* G) {
  if (!b || !G) return QG_ERR_INVALID_ARG;
  *G = b->cls_cluster[0];
  return QG_OK;
}

int qg_cluster_size(int N, int S, int restart) {
  for (int G = 1; G <= 16; G *= 2)
    if (qg_cluster_smem(N, S, G, restart) > 0) return G;
  return 0;
}

qg_status qg_batch_replay(qg_batch_t b) {
  if (!b || !b->graph) return QG_ERR_INVALID_ARG;
  QG_TRY(cudaGraphLaunch(b->graph, b->stream));
  return QG_OK;
}

qg_status qg_batch_stats(qg_batch_t b, int32_t* statuses, qg_step_stats* stats) {
  if (!b) return QG_ERR_INVALID_ARG;
  return batch_collect(b, statuses, stats);
}

void* qg_batch_stream(qg_batch_t b) { return b ? (void*)b->stream : nullptr; }

qg_status qg_batch_propagate(qg_state_t* states, int nstates, int method, int order, int scheme, double dt,
                             int64_t nsteps, const qg_solver_opts* opts, int32_t* statuses, qg_step_stats* stats) {
  qg_batch_t b = nullptr;
  qg_status st = qg_batch_create(states, nstates, &b);
  if (st != QG_OK) return st;
  st = qg_batch_run(b, method, order, scheme, dt, nsteps, opts, statuses, stats);
  qg_batch_destroy(b);
  return st;
}

qg_status qg_norm(qg_state_t s, double* out) {
  if (!s || !out) return QG_ERR_INVALID_ARG;
  double pop[QG_MAX_S];
  qg_status st = qg_population(s, pop);
  if (st != QG_OK) return st;
  double t = 0.0;
  for (int i = 0; i < s->m->S; ++i) t += pop[i];
  *out = std::sqrt(t);
  return QG_OK;
}

qg_status qg_population(qg_state_t s, double* out) {
  if (!s || !out) return QG_ERR_INVALID_ARG;
  const qg_grid* g = s->m->g;
  QG_TRY(qg_launch_populations(s->d_psi, g->ntot, s->m->S, grid_dv(g), s->d_scalars, s->stream));
  QG_TRY(cudaMemcpyAsync(out, s->d_scalars, sizeof(double) * s->m->S, cudaMemcpyDeviceToHost, s->stream));
  QG_TRY(cudaStreamSynchronize(s->stream));
  return QG_OK;
}

qg_status qg_energy(qg_state_t s, double* out) {
  if (!s || !out) return QG_ERR_INVALID_ARG;
  const qg_grid* g = s->m->g;
  if (g->D == 2) {
    QG_TRY(qg_launch_apply_h2d(make_inst2d(s), s->d_work + (size_t)2 * s->m->S * g->ntot, s->d_scalars,
                               s->stream));
  } else {
    QG_TRY(qg_launch_energy(s->d_inst, s->d_scalars, g->n[0], s->m->S, s->stream));
  }
  double v[2];
  QG_TRY(cudaMemcpyAsync(v, s->d_scalars, sizeof(v), cudaMemcpyDeviceToHost, s->stream));
  QG_TRY(cudaStreamSynchronize(s->stream));
  *out = v[0];
  return QG_OK;
}

qg_status qg_overlap(qg_state_t a, qg_state_t b, double* out) {
  if (!a || !b || !out) return QG_ERR_INVALID_ARG;
  if (a->m->S != b->m->S || a->m->g->ntot != b->m->g->ntot) return QG_ERR_INVALID_ARG;
  const size_t len = (size_t)a->m->S * a->m->g->ntot;
  QG_TRY(cudaStreamSynchronize(b->stream));
  QG_TRY(qg_launch_overlap(a->d_psi, b->d_psi, (int)len, grid_dv(a->m->g), a->d_scalars, a->stream));
  QG_TRY(cudaMemcpyAsync(out, a->d_scalars, sizeof(double) * 2, cudaMemcpyDeviceToHost, a->stream));
  QG_TRY(cudaStreamSynchronize(a->stream));
  return QG_OK;
}


qg_status qg_propagate_noalloc(int N, double qmin, double qmax, int S, double mass, const double* V, const double* F,
                               void* psi, int method, int order, int scheme, double dt, int64_t nsteps,
                               const qg_solver_opts* opts, qg_step_stats* stats, void* stream) {
  if (!V || !F || !psi) {
    snprintf(g_err, sizeof(g_err), "qg_propagate_noalloc: V, F and psi must be device pointers");
    return QG_ERR_INVALID_ARG;
  }
  if (!is_pow2(N) || N < QG_MIN_N || N > QG_NA_MAX_N || S < 2 || S > QG_MAX_S || (int64_t)S * N > QG_NA_MAX_LEN) {
    snprintf(g_err, sizeof(g_err),
             "qg_propagate_noalloc: N = %d, S = %d outside the fixed scratch capacity "
             "(N a power of two in [%d, %d], 2 <= S <= %d, S*N <= %d)",
             N, S, QG_MIN_N, QG_NA_MAX_N, QG_MAX_S, QG_NA_MAX_LEN);
    return QG_ERR_INVALID_ARG;
  }
  if (!(qmax > qmin) || !std::isfinite(qmin) || !std::isfinite(qmax) || !(mass > 0.0) || !std::isfinite(mass) ||
      !std::isfinite(dt) || nsteps < 0 || (method != QG_TRAPEZOIDAL && method != QG_MIDPOINT)) {
    snprintf(g_err, sizeof(g_err), "qg_propagate_noalloc: invalid grid, mass, method or step");
    return QG_ERR_INVALID_ARG;
  }
  qg_solver_opts o;
  default_opts(&o);
  o.restart = QG_NA_MAX_RESTART;
  if (opts) o = *opts;
  if (!valid_opts(o) || o.restart > QG_NA_MAX_RESTART) {
    snprintf(g_err, sizeof(g_err), "qg_propagate_noalloc: invalid solver options (restart must be <= %d)",
             QG_NA_MAX_RESTART);
    return QG_ERR_INVALID_ARG;
  }
  StepPlan P;
  memset(&P, 0, sizeof(P));
  P.nfrac = schedule_fixed(order, scheme, P.frac);
  if (P.nfrac == 0) {
    snprintf(g_err, sizeof(g_err), "qg_propagate_noalloc: invalid order or scheme");
    return QG_ERR_INVALID_ARG;
  }
  P.method = method;
  P.dt = dt;
  P.nsteps = nsteps;
  P.tol = o.tol;
  P.restart = o.restart;
  P.max_iters = o.max_iters;
  P.reorth = o.reorth;
  P.mid_epi = o.midpoint_epilogue;
  P.true_res = o.true_residual;
  P.inner_tol = o.inner_tol;
  P.max_outer = o.max_outer;
  P.solver = o.solver;
  P.guess = o.guess;
  const FftPlan plan = make_plan(N);
  qg_step_stats h;
  memset(&h, 0, sizeof(h));
  cudaError_t e = qg_noalloc_launch(N, qmin, qmax, S, mass, V, F, (double2*)psi, plan, P, &h, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_err("qg_propagate_noalloc", e);
    return QG_ERR_CUDA;
  }
  if (stats) *stats = h;
  return (qg_status)h.status;
}

qg_status qg_selftest_barrier_timeout(int* timed_out, int* passed) {
  int* d = nullptr;
  QG_TRY(cudaMalloc(&d, 4 * sizeof(int)));
  cudaError_t e = qg_selftest_barrier(d, timed_out, passed);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_err("qg_selftest_barrier_timeout", e);
    return QG_ERR_CUDA;
  }
  return (timed_out && *timed_out) ? QG_ERR_TIMEOUT : QG_OK;
}

}  // extern "C"
