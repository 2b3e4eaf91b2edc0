// Small kernels of libqgeom -- the Hamiltonian action, the energy,
// observables, the Gaussian initial state, the diabatic -> adiabatic field
// builders, FP64 -> FP32 copies -- and the host launch wrappers, including the
// occupancy dispatch of the persistent propagator.
#include <cuda_runtime.h>

#include <mutex>
#include <utility>
#include <vector>

#include "qg_cluster.cuh"
#include "qg_dom1d.cuh"

namespace qg {

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
// O(q) of Eq. (..._orthogonal_transformation) with columns in ascending
// order: ground = (-Delta, W12) / norm (the paper's state 2), excited =
// (W12, Delta) / norm (state 1), Delta = V_1 - W11 = dW/2 + r taken as
// W12^2 / (r - dW/2) when dW < 0 (no cancellation); O is written when given.
__global__ void fields2_kernel(const double* __restrict__ W, const double* __restrict__ dW, int n, int D, double* V,
                               double* F, double* O) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double w11 = W[j], w12 = W[n + j], w22 = W[2 * n + j];
  const double dw = w22 - w11;
  const double wbar = 0.5 * (w11 + w22);
  const double r = hypot(0.5 * dw, w12);
  V[j] = wbar - r;
  V[n + j] = wbar + r;
  if (O) {
    const double del = dw >= 0.0 ? 0.5 * dw + r : (r - 0.5 * dw > 0.0 ? w12 * w12 / (r - 0.5 * dw) : 0.0);
    const double nrm = hypot(del, w12);
    double* o = O + (size_t)j * 4;   // o[r * 2 + i]: component r of state i
    if (nrm > 0.0) {
      o[0] = -del / nrm;
      o[2] = w12 / nrm;
      o[1] = w12 / nrm;
      o[3] = del / nrm;
    } else {   // uncoupled with W22 < W11: the ground state is diabatic state 1
      o[0] = 0.0;
      o[2] = 1.0;
      o[1] = 1.0;
      o[3] = 0.0;
    }
  }
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

// Diabatic representation: V = the diagonal of W, F = its upper triangle
// (pairs s < t in lexicographic order, as for the adiabatic couplings).
__global__ void diabatic_fields_kernel(const double* __restrict__ W, int n, int S, double* V, double* F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int t = 0, p = 0;
  for (int a = 0; a < S; ++a)
    for (int b = a; b < S; ++b) {
      const double w = W[(size_t)t * n + j];
      if (a == b)
        V[(size_t)a * n + j] = w;
      else
        F[(size_t)(p++) * n + j] = w;
      ++t;
    }
}

// out = O^T in (to_adiabatic, Eq. psi_diab2adiab) or O in at every point.
__global__ void rotate_kernel(const double* __restrict__ O, const double2* __restrict__ in, double2* out, int n, int S,
                              int to_adiabatic) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double* o = O + (size_t)j * S * S;
  double2 v[QG_MAX_S];
  for (int r = 0; r < S; ++r) v[r] = in[(size_t)r * n + j];
  for (int i = 0; i < S; ++i) {
    double2 acc = make_double2(0.0, 0.0);
    for (int r = 0; r < S; ++r) {
      const double c = to_adiabatic ? o[r * S + i] : o[i * S + r];
      acc = caxpy_r(c, v[r], acc);
    }
    out[(size_t)i * n + j] = acc;
  }
}

// Trigonometric interpolation (Appendix B), step 1: the DFT coefficients
// c_k = sum_j v_j exp(-2 pi i j k / n) of every surface by direct sums (the
// phase from the exact integer j k mod n).
__global__ void interp_coef_kernel(const double2* __restrict__ src, int n, int S, double2* coef) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * n) return;
  const int s = idx / n, k = idx - s * n;
  const double2* v = src + (size_t)s * n;
  double2 acc = make_double2(0.0, 0.0);
  long long ph = 0;
  for (int j = 0; j < n; ++j) {
    double sn, cs;
    sincospi(-2.0 * (double)ph / (double)n, &sn, &cs);
    acc = caxpy(make_double2(cs, sn), v[j], acc);
    ph += k;
    if (ph >= n) ph -= n;
  }
  coef[idx] = acc;
}

// Step 2: p(q) = (1/n) sum_k c_k exp(i k' 2 pi (q - qmin) / L), k' the signed
// frequency, the Nyquist coefficient taken as a cosine (split between +-n/2).
__global__ void interp_eval_kernel(const double2* __restrict__ coef, int ns, double qmin_s, double len_s,
                                   double2* dst, int nd, double qmin_d, double dq_d, int S) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * nd) return;
  const int s = idx / nd, i = idx - s * nd;
  const double x = (qmin_d + dq_d * i - qmin_s) / len_s;
  const double2* c = coef + (size_t)s * ns;
  double2 acc = make_double2(0.0, 0.0);
  for (int k = 0; k < ns; ++k) {
    const int m = k < ns / 2 ? k : k - ns;
    double t = (double)m * x;
    t -= rint(t);
    double sn, cs;
    if (k == ns / 2) {
      cs = cospi(2.0 * t);
      sn = 0.0;
    } else {
      sincospi(2.0 * t, &sn, &cs);
    }
    acc = caxpy(make_double2(cs, sn), c[k], acc);
  }
  dst[idx] = cscale(1.0 / ns, acc);
}

__global__ void to_f32_kernel(const double* __restrict__ in, float* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
}  // namespace qg
// ---------------------------------------------------------------------------
// Host-side launch wrappers.

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
  // staging may use what one CTA per SM leaves free (227 KB less the static
  // arrays), or the 2-CTA budget
  const int stage = stage_plan(max_n, max_S, ctas_per_sm >= 2 ? 110 * 1024 : 224 * 1024, &smem);
  if (ninst == 0)   // attributes only
    return ctas_per_sm >= 2
               ? qg_launch_propagate_minb<2>(d_insts, 0, plan, d_counter, d_stats, max_n, max_S, nb, stage, smem, 0, st)
               : qg_launch_propagate_minb<1>(d_insts, 0, plan, d_counter, d_stats, max_n, max_S, nb, stage, smem, 0, st);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slots = sms * (ctas_per_sm >= 2 ? 2 : 1);
  const int grid = ninst < slots ? ninst : slots;
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (ctas_per_sm >= 2)
    return qg_launch_propagate_minb<2>(d_insts, ninst, plan, d_counter, d_stats, max_n, max_S, nb, stage, smem, grid,
                                       st);
  return qg_launch_propagate_minb<1>(d_insts, ninst, plan, d_counter, d_stats, max_n, max_S, nb, stage, smem, grid, st);
}

cudaError_t qg_launch_propagate(const InstDesc* d_insts, int ninst, const StepPlan& plan, int* d_counter,
                                qg_step_stats* d_stats, int max_n, int max_S, cudaStream_t st) {
  return qg_launch_propagate_tuned(d_insts, ninst, plan, d_counter, d_stats, max_n, max_S, 1, 0, st);
}

cudaError_t qg_allow_max_smem(const void* fn, bool cluster) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> hold(mu);
  for (const auto& d : done)
    if (d.first == fn && d.second == dev) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess && cluster) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) done.push_back({fn, dev});
  return e;
}

cudaError_t qg_launch_apply_h(const InstDesc* d_inst, double2* d_out, int n, int S, cudaStream_t st) {
  size_t smem;
  const int nb = nb_capacity(n, S, 1, &smem);
  cudaError_t e = qg_allow_max_smem((const void*)qg::apply_h_kernel);
  if (e != cudaSuccess) return e;
  qg::apply_h_kernel<<<1, QG_THREADS, smem, st>>>(d_inst, d_out, nb);
  return cudaGetLastError();
}

cudaError_t qg_launch_energy(const InstDesc* d_inst, double* d_out, int n, int S, cudaStream_t st) {
  size_t smem;
  const int nb = nb_capacity(n, S, 1, &smem);
  cudaError_t e = qg_allow_max_smem((const void*)qg::energy_kernel);
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
                              double* d_O, cudaStream_t st) {
  qg::fields2_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_W, d_dW, n, D, d_V, d_F, d_O);
  return cudaGetLastError();
}

cudaError_t qg_launch_diabatic_fields(const double* d_W, int n, int S, double* d_V, double* d_F, cudaStream_t st) {
  qg::diabatic_fields_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_W, n, S, d_V, d_F);
  return cudaGetLastError();
}

cudaError_t qg_launch_rotate(const double* d_O, const double2* in, double2* out, int n, int S, int to_adiabatic,
                             cudaStream_t st) {
  qg::rotate_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_O, in, out, n, S, to_adiabatic);
  return cudaGetLastError();
}

cudaError_t qg_launch_interpolate(const double2* src, int ns, double qmin_s, double len_s, double2* coef,
                                  double2* dst, int nd, double qmin_d, double dq_d, int S, cudaStream_t st) {
  qg::interp_coef_kernel<<<(S * ns + 127) / 128, 128, 0, st>>>(src, ns, S, coef);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  qg::interp_eval_kernel<<<(S * nd + 127) / 128, 128, 0, st>>>(coef, ns, qmin_s, len_s, dst, nd, qmin_d, dq_d, S);
  return cudaGetLastError();
}

cudaError_t qg_launch_cluster(int G, const InstDesc* d_insts, int ninst, const StepPlan& plan, qg_step_stats* d_stats,
                              size_t smem, cudaStream_t st) {
  switch (G) {
    case 1:
      return qg_launch_cluster_g<1>(d_insts, ninst, plan, d_stats, smem, st);
    case 2:
      return qg_launch_cluster_g<2>(d_insts, ninst, plan, d_stats, smem, st);
    case 4:
      return qg_launch_cluster_g<4>(d_insts, ninst, plan, d_stats, smem, st);
    case 8:
      return qg_launch_cluster_g<8>(d_insts, ninst, plan, d_stats, smem, st);
    case 16:
      return qg_launch_cluster_g<16>(d_insts, ninst, plan, d_stats, smem, st);
    default:
      return cudaErrorInvalidValue;
  }
}

size_t qg_cluster_smem(int n, int S, int G, int restart) {
  if (G < 1 || G > 16 || (G & (G - 1)) || n % G || n / G < 8 || S < 2 || S > QG_MAX_S) return 0;
  // local vectors of at most kClusterLocal values, split evenly into the
  // G shares of the centre phase
  if ((long long)S * (n / G) > qg::kClusterLocal || (S * (n / G)) % G) return 0;
  const size_t t = qg::cluster_smem_layout(n / G, S, G, restart).total;
  return t <= (size_t)227 * 1024 ? t : 0;
}
