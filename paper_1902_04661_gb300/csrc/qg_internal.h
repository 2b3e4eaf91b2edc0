// Internal declarations shared by the host API and the kernels of libqgeom.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qgeom.h"

#define QG_MAX_S 4
#define QG_MAX_D 2
#define QG_MAX_2D_POINTS (1 << 20)
#define QG_MAX_RESTART 64
#define QG_MAX_PASSES 8
#define QG_MAX_FRACTIONS 128
#define QG_MAX_CLASSES 12
#define QG_MIN_N 8
#define QG_MAX_N 8192
#define QG_THREADS 256
// Capacity of the no-allocation entry point (qg_propagate_noalloc).
#define QG_NA_MAX_LEN 8192
#define QG_NA_MAX_N 8192
#define QG_NA_MAX_RESTART 16

// Radix plan of one power-of-two FFT length.  Passes run in the listed order
// for the forward (decimation-in-frequency) transform and in reverse order
// for the inverse (decimation-in-time) transform.
struct FftPlan {
  int n;
  int npass;
  int radix[QG_MAX_PASSES];
};

// Radix sequence for n = 2^k (k >= 2): as many radix-8 passes as possible,
// the remainder as one or two radix-4 passes.
__host__ __device__ inline FftPlan make_plan(int n) {
  FftPlan p;
  p.n = n;
  p.npass = 0;
  int k = 0;
  while ((1 << k) < n) ++k;
  int a = k / 3;
  const int rem = k % 3;
  if (rem == 1) a -= 1;
  for (int i = 0; i < a; ++i) p.radix[p.npass++] = 8;
  if (rem == 2) p.radix[p.npass++] = 4;
  if (rem == 1) {
    p.radix[p.npass++] = 4;
    p.radix[p.npass++] = 4;
  }
  return p;
}

// Accumulated frequency K of block blk of a forward pass preceded by the
// passes radix[0..] that made nbk blocks: the block index read as
// mixed-radix digits (first pass most significant), digits reversed.
__host__ __device__ inline int block_frequency(int blk, const int* radix, int nbk) {
  int K = 0, mult = 1, rem = blk, size = nbk, i = 0;
  while (size > 1) {
    const int R = radix[i++];
    size /= R;
    const int d = rem / size;
    rem -= d * size;
    K += d * mult;
    mult *= R;
  }
  return K;
}

// Sizes of the Linzer-Feig factor tables of the FP64 transform of a plan
// (qg_api.cu, lf_tables): one set of factors per block of forward passes
// 1..npass-1 and per position of inverse passes 0..npass-2, 4 double2
// entries per radix-8 set and 2 per radix-4 set, one word of form bits per
// set.
__host__ __device__ inline void lf_counts(const int* radix, int npass, int n, int* entries, int* sets) {
  int e = 0, s = 0, L = n;
  for (int i = 0; i < npass; ++i) {
    const int R = radix[i], E = R == 8 ? 4 : 2;
    if (i >= 1) {
      e += E * (n / L);
      s += n / L;
    }
    if (i <= npass - 2) {
      e += E * (L / R);
      s += L / R;
    }
    L /= R;
  }
  *entries = e;
  *sets = s;
}

// Bytes of those tables for n points (entries, then form words, padded to 16).
__host__ __device__ inline size_t lf_table_bytes(int n) {
  const FftPlan p = make_plan(n);
  int e = 0, s = 0;
  lf_counts(p.radix, p.npass, n, &e, &s);
  return ((size_t)e * 16 + (size_t)s * 4 + 15) & ~(size_t)15;
}

struct qg_grid {
  int D;
  int n[2];
  double qmin[2], qmax[2], dq[2];
  int ntot;
  FftPlan plan[2];
  double2* d_tw[2];  // tw[k] = exp(-2 pi i k / n), k = 0..n-1
  double2* d_lf[2];  // Linzer-Feig factor tables of the FP64 transform (entries, then the form words)
  unsigned* d_lff[2];  // the form words (inside the d_lf allocation)
  double* d_kd[2];   // k of the frequency held at digit-reversed position p, divided by n
  float2* d_tw32[2];  // the same tables rounded to FP32 (mixed-precision inner solves)
  float* d_kd32[2];
  int device;
};

struct qg_model {
  qg_grid* g;
  int S;
  double mass[2];
  double* d_V;  // S * ntot
  double* d_F;  // D * S(S-1)/2 * ntot (upper triangle)
  float* d_V32;  // FP32 copies for the mixed-precision inner solves
  float* d_F32;
  int rep;       // 0: adiabatic (V, F); 1: diabatic representation (V = diag W, F = upper triangle of W)
  double* d_O;   // adiabatic models built from W: O(q) per point, O[(j S + r) S + i] = component r of
                 // adiabatic state i (ascending), or null
};

struct InstDesc;

struct qg_state_adjoint {
  double2* ckpt;
  long long nckpt;
  long long every;
  double2* grad;
  double* gV;
  double* gF;
};

struct qg_state {
  qg_model* m;
  InstDesc* d_inst;         // this state's instance descriptor (device)
  int* d_counter;           // work counter of the persistent kernel (device)
  double2* d_psi;    // S * ntot
  double2* d_work;   // (restart_cap + 5) vectors of S * ntot
  float2* d_work32;  // mixed precision: (restart_cap + 4) FP32 vectors, else null
  int precision;     // QG_C128 or QG_C64_MIXED
  int restart_cap;
  cudaStream_t stream;
  qg_step_stats* d_stats;   // one record
  double* d_scalars;        // small device scratch for observables
  qg_state_adjoint adj;     // caller-owned adjoint buffers (or nulls)
  unsigned char* d_coop;    // 2-D grids: barrier words, error flag, partial sums
  int launch_ctas;          // 2-D grids: cooperative launch width (0 = automatic)
  int cluster;              // 1-D grids: > 0 selects the shared-memory cluster form with this many CTAs
};

// Everything one CTA needs to work on one instance (a state with its model
// and grid), in device memory.
struct InstDesc {
  int n;          // grid points
  int S;          // surfaces
  int npass;
  int radix[QG_MAX_PASSES];
  double h2m;     // hbar^2 / (2 m)
  double dq;
  const double2* tw;
  const double* kd;
  const double2* lf;     // Linzer-Feig factor tables (FP64 transform), or null: the
  const unsigned* lff;   // transform then runs its twiddle passes from tw
  const double* V;
  const double* F;
  double2* psi;
  double2* work;  // U, B, X, P0, then basis V_0..V_m (each S * n)
  int restart_cap;
  int precision;  // QG_C128 or QG_C64_MIXED
  const float2* tw32;
  const float* kd32;
  const float* V32;
  const float* F32;
  float2* work32;  // mixed: U32, r32, d32, then inner basis (each S * n)
  // adjoint buffers (caller-owned device memory, optional)
  double2* ckpt;       // checkpoints: nckpt vectors of S * n
  long long nckpt;
  long long every;     // composed steps between checkpoints
  double2* grad;       // in: dL/dpsi(t_f); out: dL/dpsi(0)   (S * n)
  double* gV;          // += dL/dV   (S * n)
  double* gF;          // += dL/dF   (S(S-1)/2 * n)
  int rep;             // 1: diabatic representation (see qg_model)
};

// One instance on a 2-D grid (all CTAs of a cooperative launch share it).
struct Inst2D {
  int n[2];
  int S;
  int npass[2];
  int radix[2][QG_MAX_PASSES];
  double h2m[2];
  double dv;
  const double2* tw[2];
  const double* kd[2];
  const double2* lf[2];     // Linzer-Feig factor tables of each dimension's FP64 transform, or null
  const unsigned* lff[2];
  const float2* tw32[2];
  const float* kd32[2];
  const double* V;     // S * N
  const double* F;     // 2 * S(S-1)/2 * N
  const float* V32;
  const float* F32;
  double2* psi;
  double2* work;       // U, T, B, X, P0, basis (m + 1)
  float2* work32;      // U, T, r, d, basis (m + 1)
  int precision;
  unsigned* bar;       // grid barrier: count, generation
  int* err;            // barrier time-out flag
  double* gred;        // 2 x gridDim x 32 partial sums
  double2* ckpt;
  long long nckpt;
  long long every;
  int ctas;            // cooperative launch width (0 = automatic)
};

// Parameters of one propagate launch (passed by value).
struct StepPlan {
  int method;
  int nfrac;
  double dt;
  long long nsteps;
  double tol;
  int restart;
  int max_iters;
  int reorth;
  int mid_epi;
  int true_res;
  double inner_tol;
  int max_outer;
  int run;   // QG_RUN_FORWARD, QG_RUN_CHECKPOINT or QG_RUN_ADJOINT
  int solver;  // QG_SOLVER_GMRES or QG_SOLVER_LANCZOS
  int guess;   // QG_GUESS_EULER or QG_GUESS_ZERO
  double frac[QG_MAX_FRACTIONS];
};

struct qg_batch {
  int n;
  int max_n, max_S;
  cudaStream_t stream;      // the states' stream, or a private stream when that is the legacy stream
  bool own_stream;
  InstDesc* d_desc;         // instance table, longest estimated work first
  int* order;               // order[k] = index (into the caller's list) of table entry k
  qg_step_stats* d_stats;   // per table entry
  int* d_counter;
  qg_step_stats* h_stats;   // pinned, per table entry
  cudaGraphExec_t graph;    // captured run, or null
  bool adjoint_ready;       // every state has checkpoint and gradient buffers
  int all_fp64;             // every state is adiabatic QG_C128 (the cluster form needs it)
  // Grid-size classes: the table is ordered by N (then S) descending, and
  // entries [cls_start[c], cls_start[c] + cls_count[c]) share N = cls_n[c]
  // (cls_S[c] = their largest S).  Each class is one persistent launch with
  // its own shape: CTAs per SM, surfaces per FFT batch, cluster size (> 0:
  // the shared-memory cluster form); qg_batch_autotune picks them.
  int nclass;
  int cls_start[QG_MAX_CLASSES], cls_count[QG_MAX_CLASSES], cls_n[QG_MAX_CLASSES], cls_S[QG_MAX_CLASSES];
  int cls_ctas[QG_MAX_CLASSES], cls_nb[QG_MAX_CLASSES], cls_cluster[QG_MAX_CLASSES];
  // the classes run concurrently: one stream per class, forked from and
  // joined back into the batch's stream with events
  cudaStream_t cls_stream[QG_MAX_CLASSES];
  cudaEvent_t cls_done[QG_MAX_CLASSES];
  cudaEvent_t fork;
};

// Raises a kernel's dynamic shared-memory limit to the device maximum, once
// per kernel and device (thread-safe, qg_kernels.cu).  Launches of any
// smaller size then need no further attribute call, so launches issued from
// several host threads cannot lower the limit under one another.
// cluster: also allow non-portable cluster sizes (more than 8 CTAs).
cudaError_t qg_allow_max_smem(const void* fn, bool cluster = false);

// Launch wrappers (qg_kernels.cu).
size_t qg_smem_bytes(int max_n, int max_S, int restart);
cudaError_t qg_launch_propagate(const InstDesc* d_insts, int ninst, const StepPlan& plan, int* d_counter,
                                qg_step_stats* d_stats, int max_n, int max_S, cudaStream_t st);
// The persistent propagator built for MINB CTAs per SM (one translation unit
// each); grid 0 only sets the kernel's shared-memory attribute.
template <int MINB>
cudaError_t qg_launch_propagate_minb(const InstDesc* d_insts, int ninst, const StepPlan& plan, int* d_counter,
                                     qg_step_stats* d_stats, int max_n, int max_S, int nb, int stage, size_t smem,
                                     int grid, cudaStream_t st);
template <>
cudaError_t qg_launch_propagate_minb<1>(const InstDesc*, int, const StepPlan&, int*, qg_step_stats*, int, int, int, int,
                                        size_t, int, cudaStream_t);
template <>
cudaError_t qg_launch_propagate_minb<2>(const InstDesc*, int, const StepPlan&, int*, qg_step_stats*, int, int, int, int,
                                        size_t, int, cudaStream_t);
cudaError_t qg_launch_propagate_tuned(const InstDesc* d_insts, int ninst, const StepPlan& plan, int* d_counter,
                                      qg_step_stats* d_stats, int max_n, int max_S, int ctas_per_sm, int nb_pref,
                                      cudaStream_t st);
// The shared-memory cluster form of the 1-D propagator, one translation unit
// per cluster size G (qg_propagate_cluster.cu); qg_launch_cluster dispatches
// on G (1, 2, 4, 8, 16).
template <int G>
cudaError_t qg_launch_cluster_g(const InstDesc* d_insts, int ninst, const StepPlan& plan, qg_step_stats* d_stats,
                                size_t smem, cudaStream_t st);
template <>
cudaError_t qg_launch_cluster_g<1>(const InstDesc*, int, const StepPlan&, qg_step_stats*, size_t, cudaStream_t);
template <>
cudaError_t qg_launch_cluster_g<2>(const InstDesc*, int, const StepPlan&, qg_step_stats*, size_t, cudaStream_t);
template <>
cudaError_t qg_launch_cluster_g<4>(const InstDesc*, int, const StepPlan&, qg_step_stats*, size_t, cudaStream_t);
template <>
cudaError_t qg_launch_cluster_g<8>(const InstDesc*, int, const StepPlan&, qg_step_stats*, size_t, cudaStream_t);
template <>
cudaError_t qg_launch_cluster_g<16>(const InstDesc*, int, const StepPlan&, qg_step_stats*, size_t, cudaStream_t);
cudaError_t qg_launch_cluster(int G, const InstDesc* d_insts, int ninst, const StepPlan& plan, qg_step_stats* d_stats,
                              size_t smem, cudaStream_t st);
// Dynamic shared memory of the cluster form for an instance of n points and
// S surfaces on clusters of G CTAs, or 0 if that shape is not supported.
size_t qg_cluster_smem(int n, int S, int G, int restart);
cudaError_t qg_launch_apply_h(const InstDesc* d_inst, double2* d_out, int n, int S, cudaStream_t st);
cudaError_t qg_launch_energy(const InstDesc* d_inst, double* d_out, int n, int S, cudaStream_t st);
cudaError_t qg_launch_populations(const double2* d_psi, int n, int S, double dq, double* d_out, cudaStream_t st);
cudaError_t qg_launch_overlap(const double2* d_a, const double2* d_b, int len, double dq, double* d_out,
                              cudaStream_t st);
cudaError_t qg_launch_gaussian(double2* d_psi, int n, int S, int surface, double qmin, double dq, double q0,
                               double p0, double sigma0, cudaStream_t st);
cudaError_t qg_noalloc_launch(int n, double qmin, double qmax, int S, double mass, const double* V, const double* F,
                              double2* psi, const FftPlan& plan, const StepPlan& P, qg_step_stats* host_stats,
                              cudaStream_t st);
// Host stub of the 2-D propagator kernel for one precision form (0:
// complex128, 1: mixed), one translation unit each.
template <int PREC>
const void* qg_propagate2d_fn();
template <>
const void* qg_propagate2d_fn<0>();
template <>
const void* qg_propagate2d_fn<1>();
cudaError_t qg_launch_propagate2d(const Inst2D& I, const StepPlan& P, qg_step_stats* d_stats, cudaStream_t st);
int qg_grid2d_ctas(const Inst2D& I);
cudaError_t qg_launch_apply_h2d(const Inst2D& I, double2* d_out, double* d_energy, cudaStream_t st);
cudaError_t qg_launch_gaussian2d(double2* d_psi, const int* n, int S, int surface, const double* qmin,
                                 const double* dq, const double* q0, const double* p0, const double* s0,
                                 cudaStream_t st);
cudaError_t qg_selftest_barrier(int* d_words, int* h_timed_out, int* h_passed);
cudaError_t qg_launch_to_f32(const double* d_in, float* d_out, size_t n, cudaStream_t st);
cudaError_t qg_launch_fieldsS(const double* d_W, const double* d_dW, int n, int S, double* d_V, double* d_F,
                              double* d_vec, cudaStream_t st);
cudaError_t qg_launch_fields2(const double* d_W, const double* d_dW, int n, int D, double* d_V, double* d_F,
                              double* d_O, cudaStream_t st);
cudaError_t qg_launch_diabatic_fields(const double* d_W, int n, int S, double* d_V, double* d_F, cudaStream_t st);
cudaError_t qg_launch_rotate(const double* d_O, const double2* in, double2* out, int n, int S, int to_adiabatic,
                             cudaStream_t st);
cudaError_t qg_launch_interpolate(const double2* src, int ns, double qmin_s, double len_s, double2* coef,
                                  double2* dst, int nd, double qmin_d, double dq_d, int S, cudaStream_t st);
