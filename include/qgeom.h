/*
 * qgeom.h -- C-ABI of the GB300 (sm_103a) library for composed implicit
 * propagation of multi-surface nuclear wavepackets on Fourier grids in the
 * adiabatic representation (Choi & Vanicek, arXiv:1902.04661).
 *
 * The method: the time-dependent Schroedinger equation (Eq. tdse) with the
 * adiabatic molecular Hamiltonian (Eq. adiab_mol_ham)
 *     H = 1/2 [p 1 - i hbar F(q)]^dagger . m^{-1} . [p 1 - i hbar F(q)] + V(q)
 * is propagated by the trapezoidal rule (Eq. trap_rule) or the implicit
 * midpoint method (Eq. imp_midpoint), each the product of an explicit Euler
 * (Eq. exp_euler) and an implicit Euler (Eq. imp_euler) half step.  Every
 * implicit half step solves (1 + i tau H) x = b, tau = dt / (2 hbar), with
 * restarted GMRES started from the explicit-Euler guess (Sec. II B).  The
 * elementary steps are composed recursively and symmetrically by the triple
 * jump (Eq. triple_jump) or Suzuki's fractal (Eq. suzukis_fractal) to orders
 * 2, 4, 6, 8 (Sec. II C).  H psi is evaluated by the dynamic Fourier method
 * (Sec. II D): 4 D Fourier transforms per surface.
 *
 * Units: Hartree atomic units, hbar = 1.  Times in atomic units of time.
 *
 * Conventions shared by every entry point:
 *  - Grid: dimension d has N_d points q_j = qmin_d + j dq_d, j = 0..N_d-1,
 *    dq_d = (qmax_d - qmin_d) / N_d (periodic).  N_d must be a power of two,
 *    8 <= N_d <= 8192.  Only D = 1 grids are accepted by this version.
 *  - Wave numbers k_j = 2 pi / (N dq) (j for j < N/2, j - N otherwise).
 *  - Inner product <a|b> = prod_d dq_d * sum_s sum_j conj(a_s(q_j)) b_s(q_j).
 *  - A molecular state is S * prod(N_d) complex values (double2 = {re, im}),
 *    surface-major: element (s, j) at index s * prod(N_d) + j, grid points in
 *    C order.
 *  - Adiabatic surfaces are ordered by ascending energy (0 = ground).
 *  - V is S * prod(N_d) doubles (surface-major).  F is the upper triangle of
 *    the real antisymmetric coupling matrices: D * S(S-1)/2 * prod(N_d)
 *    doubles, dimension-major, pairs (i < j) in lexicographic order
 *    (01, 02, 12 for S = 3); F_ji = -F_ij and F_ii = 0 are implied.
 *  - Diabatic W is the upper triangle including the diagonal:
 *    S(S+1)/2 * prod(N_d) doubles, pairs (i <= j) lexicographic
 *    (00, 01, 11 for S = 2); dW is D * S(S+1)/2 * prod(N_d) doubles of
 *    dW/dq_d.
 *
 * Ownership: the library owns every handle and the device workspaces behind
 * it; the caller owns every buffer it passes.  A buffer flagged on_device is
 * a device pointer of the current device and is read or written in stream
 * order on the state's stream; a host buffer is copied synchronously.
 *
 * Errors: every call returns a qg_status and never throws across the ABI.
 * A propagation that fails (GMRES not converged within the iteration cap)
 * restores the state it was given and returns QG_ERR_NOT_CONVERGED with the
 * statistics filled in.  Invalid handles or sizes return QG_ERR_INVALID_ARG
 * before any device work.  CUDA errors return QG_ERR_CUDA
 * (qg_last_error_string() gives the CUDA message).
 */
#ifndef QGEOM_H
#define QGEOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QG_OK = 0,
  QG_ERR_INVALID_ARG = 1,
  QG_ERR_NOT_CONVERGED = 2,
  QG_ERR_CUDA = 3,
  QG_ERR_OOM = 4,
  QG_ERR_TIMEOUT = 5,
  QG_ERR_UNSUPPORTED = 6
} qg_status;

/* Elementary second-order methods (Sec. II B), composable (Sec. II C). */
enum { QG_TRAPEZOIDAL = 0,   /* U_impl(dt/2) U_expl(dt/2), Eq. (trap_rule)    */
       QG_MIDPOINT = 1,      /* U_expl(dt/2) U_impl(dt/2), Eq. (imp_midpoint) */
/* The elementary comparison methods of Sec. II B, never composed.  Pass
 * order 1 for the Euler methods and order 2 for SOD (the scheme is ignored);
 * each step has size dt:
 *   QG_EXPLICIT_EULER  psi' = (1 - i dt H) psi, Eq. (exp_euler): norm grows,
 *                      unstable for every dt (Eq. exp_eu_stability);
 *   QG_IMPLICIT_EULER  (1 + i dt H) psi' = psi, Eq. (imp_euler): one implicit
 *                      solve with tau = dt per step, norm decays;
 *   QG_SOD             psi(t + dt) = psi(t - dt) - 2 i dt H psi(t),
 *                      Eq. (sod_method): stable only for dt < 1 / E_max
 *                      (Eq. sod_critical_timestep).  Every call starts from
 *                      psi(-dt) approximated by one two-stage Runge-Kutta
 *                      step backward from the state (Sec. III), so nsteps in
 *                      one call differ from the same steps split over calls.
 * None of them is available for adjoint runs or qg_propagate_noalloc. */
       QG_EXPLICIT_EULER = 2,
       QG_IMPLICIT_EULER = 3,
       QG_SOD = 4 };
/* Composition schemes (Sec. II C). */
enum { QG_TRIPLE_JUMP = 0,   /* Eq. (triple_jump), M = 3, C = 3^(order/2-1)     */
       QG_SUZUKI = 1,        /* Eq. (suzukis_fractal), M = 5, C = 5^(order/2-1) */
       /* the non-recursive "optimal" schemes of Sec. II C: Kahan and Li's
        * minimal max|gamma_n| compositions, C = 9 for order 6 and C = 17 for
        * order 8 (coefficients from Kahan & Li 1997, which the paper cites
        * but does not print); order 4 is Suzuki's fractal, which Sec. II C
        * names the optimal fourth-order scheme; order 2 the elementary step */
       QG_OPTIMAL = 2 };
/* State precision: the state is always stored in complex128.  QG_C128 solves
 * every implicit step in FP64.  QG_C64_MIXED runs the Krylov iterations in
 * complex64 and refines in FP64: r = b - (1 + i tau H) x is evaluated in FP64,
 * (1 + i tau H) d = r is solved in complex64 GMRES to inner_tol, x += d, until
 * ||r|| <= tol ||b|| (FP64 residual), so the result meets the same tolerance
 * -- or until the FP64 residual stops falling (less than halved by a
 * refinement step) within 256 DBL_EPSILON ||b|| (5.7e-14 ||b||), the rounding level of an
 * FP64 residual; max_residual of the statistics reports what was reached.
 * Compositions, the state update and the observables stay FP64. */
enum { QG_C128 = 0, QG_C64_MIXED = 1 };

typedef struct qg_grid* qg_grid_t;
typedef struct qg_model* qg_model_t;
typedef struct qg_state* qg_state_t;
typedef struct qg_batch* qg_batch_t;

/* Linear-solver options for the implicit half steps (Sec. II B).
 * tol: stop when the GMRES residual estimate |g_{j+1}| <= tol * ||b||
 *      (relative residual in the inner-product norm), default 1e-12.
 * restart: Krylov dimension m of GMRES(m), 1..64, default 30.
 * max_iters: cap on the total Arnoldi iterations of one implicit solve
 *      (all restarts), default 400; exceeding it is QG_ERR_NOT_CONVERGED.
 * reorth: 1 = classical Gram-Schmidt with one re-orthogonalisation pass
 *      (CGS2, default), 0 = single pass.
 * midpoint_epilogue: 0 = psi' = 2 chi - psi (default; equal to the explicit
 *      half step up to the solver residual), 1 = psi' = chi - i tau H chi as
 *      written in Eq. (imp_midpoint) (one more H psi per step).
 * true_residual: 1 = recompute ||b - A x|| after convergence and restart if
 *      it exceeds tol (one more H psi per solve); default 0.
 * inner_tol: QG_C64_MIXED only -- relative tolerance of each complex64 inner
 *      solve, default 1e-6; a refinement step whose residual rho is already
 *      close to the target uses max(inner_tol, tol ||b|| / (4 rho)).
 * max_outer: QG_C64_MIXED only -- cap on FP64 refinement steps per implicit
 *      solve, default 10; exceeding it is QG_ERR_NOT_CONVERGED.
 * solver: QG_SOLVER_GMRES (default; restarted GMRES with Arnoldi/CGS as in
 *      Sec. II B) or QG_SOLVER_LANCZOS (the same minimal-residual iterates by
 *      the three-term recurrence that the Hermitian H allows: 5 work vectors,
 *      O(1) vector passes per iteration; needs restart >= 4).
 * guess: QG_GUESS_EULER (default) starts each implicit solve from the
 *      explicit-Euler step (1 - i tau H) b, as in Sec. II B; QG_GUESS_ZERO
 *      starts from zero, so the first residual is b and no H psi is spent on
 *      the guess or its residual.  For a minimal-residual solver the zero
 *      start after k + 2 iterations searches K_{k+2}(H, b), a space that
 *      contains everything the Euler start reaches after k iterations at the
 *      same H psi count; both stop at the same tolerance. */
enum { QG_SOLVER_GMRES = 0, QG_SOLVER_LANCZOS = 1 };
enum { QG_GUESS_EULER = 0, QG_GUESS_ZERO = 1 };
typedef struct {
  double tol;
  int restart;
  int max_iters;
  int reorth;
  int midpoint_epilogue;
  int true_residual;
  double inner_tol;
  int max_outer;
  int solver;
  int guess;
} qg_solver_opts;

/* Statistics of one propagate / step call (summed over all sub-steps). */
typedef struct {
  int64_t n_hpsi;          /* H psi evaluations                                */
  int64_t n_krylov;        /* Arnoldi iterations (I summed over sub-steps)     */
  int64_t n_substeps;      /* elementary steps taken (C per composed step)     */
  int32_t max_krylov;      /* largest I of one implicit solve                  */
  int32_t status;          /* qg_status of the call                            */
  double max_residual;     /* largest final relative residual estimate         */
  int64_t failed_step;     /* composed-step index that failed, or -1           */
  int64_t n_ortho;         /* sum over Arnoldi iterations j of (j + 1): basis
                              vectors orthogonalised against, per pass          */
  int64_t n_update;        /* basis vectors summed into the solution           */
  int64_t n_restart;       /* GMRES restarts and true-residual re-checks (one
                              H psi each)                                       */
  int64_t n_hpsi32;        /* complex64 H psi evaluations (QG_C64_MIXED)       */
  int64_t n_outer;         /* FP64 refinement steps (QG_C64_MIXED)             */
} qg_step_stats;

/* Fill opts with the defaults listed above. */
void qg_default_solver_opts(qg_solver_opts* opts);

/* Grid of D dimensions (Sec. II D; Sec. III uses D = 1, N = 2048 on
 * [3.8, 47.0) a.u.).  N, qmin, qmax: arrays of D entries, qmax > qmin.
 * Builds the FP64 twiddle and wave-number tables on the current device. */
qg_status qg_create_grid(int D, const int* N, const double* qmin, const double* qmax,
                         qg_grid_t* out);
void qg_destroy_grid(qg_grid_t g);

/* Adiabatic model from its fields (Eq. adiab_mol_ham): S surfaces (2..4),
 * mass: D nuclear masses (electron masses), V and F in the layouts above.
 * on_device: 1 = V, F are device pointers (copied device-to-device),
 * 0 = host pointers.  The grid must outlive the model. */
qg_status qg_create_model(qg_grid_t g, int S, const double* mass, const double* V,
                          const double* F, int on_device, qg_model_t* out);

/* Adiabatic model from a diabatic matrix W(q) and its derivative (Sec. II E),
 * computed on the device per grid point.  S = 2: V_{1,2} = Wbar +-
 * sqrt((dW/2)^2 + W12^2) (Eq. pot_diab2adiab with the orthogonal matrix of
 * Eq. ..._orthogonal_transformation) and the coupling of Eq. (nonadiab_c); the
 * paper labels the upper surface 1, this library stores surfaces ascending,
 * so V[0] is the ground and F[0] = F_{ground,excited} = -F_12 (paper).
 * S = 3, 4: the same definitions V = O^T W O, F = O^T O' taken numerically:
 * Jacobi eigen-decomposition per point (ascending), F_ij = <phi_i|W'|phi_j> /
 * (V_j - V_i), eigenvector signs fixed by continuity along the grid (largest
 * component positive at the first point).  Only D = 1 grids. */
qg_status qg_create_model_diabatic(qg_grid_t g, int S, const double* mass, const double* W,
                                   const double* dW, int on_device, qg_model_t* out);
/* Model in the diabatic representation (Sec. II E):
 *     H_diab = 1/2 p^T m^{-1} p 1 + W(q),
 * no vector coupling; W is the real symmetric diabatic matrix in the upper-
 * triangle layout above (S(S+1)/2 * N doubles).  H psi takes 2 transforms per
 * surface (the second derivative) and the pointwise W; all propagation
 * methods, solvers and the mixed precision form apply.  Only D = 1 grids; not
 * available in the cluster form, adjoint runs or qg_propagate_noalloc.
 * qg_model_fields returns V = the diagonal of W and F = its upper triangle. */
qg_status qg_create_model_diabatic_rep(qg_grid_t g, int S, const double* mass, const double* W, int on_device,
                                       qg_model_t* out);
/* Changes of representation with the O(q) of an adiabatic model built by
 * qg_create_model_diabatic (D = 1): psi = O(q)^T psi_diab (Eq.
 * psi_diab2adiab) and its inverse psi_diab = O(q) psi.  O's columns are the
 * adiabatic states in ascending order -- for S = 2 the paper's closed form
 * (Eq. ..._orthogonal_transformation) with its columns swapped, for S >= 3 the
 * sign-continuous eigenvectors -- consistent with the model's F = O^T O'.
 * Buffers are S * N complex128 (host or device per on_device; may be the
 * same buffer); synchronous.  QG_ERR_UNSUPPORTED for models without O. */
qg_status qg_diabatic_to_adiabatic(qg_model_t m, const void* psi_diab, void* psi_adiab, int on_device);
qg_status qg_adiabatic_to_diabatic(qg_model_t m, const void* psi_adiab, void* psi_diab, int on_device);

/* Copy the model's V and F (layouts above) to host (on_device = 0) or device
 * buffers. */
qg_status qg_model_fields(qg_model_t m, double* V, double* F, int on_device);
void qg_destroy_model(qg_model_t m);

/* Molecular wavepacket for a model (owns S * prod(N_d) complex128 values and
 * the solver workspace).  precision: QG_C128 or QG_C64_MIXED. */
qg_status qg_create_state(qg_model_t m, int precision, qg_state_t* out);
void qg_destroy_state(qg_state_t s);
/* Stream (cudaStream_t) on which the state's work is ordered; NULL = the
 * legacy default stream. */
qg_status qg_state_set_stream(qg_state_t s, void* stream);
/* 2-D grids: number of CTAs of the cooperative launch that carries the
 * state (0 = automatic: the largest power of two not above the SM count and
 * the shorter grid side).  qg_state_autotune times trial_steps composed steps
 * at the automatic width and at 1/2 and 1/4 of it (restoring psi after each
 * trial), keeps the fastest and writes the three trial times (ms) to ms_out
 * (may be NULL).  No effect on 1-D states, which run on one CTA each. */
qg_status qg_state_set_launch_width(qg_state_t s, int ctas);
/* 1-D grids: the launch form of the state's propagations (not in the paper;
 * the same arithmetic as the default form).  G = 0 (default): one CTA owns
 * the instance and keeps its vectors in global memory.  G = 1, 2, 4, 8, 16:
 * the shared-memory cluster form -- a thread-block cluster of G CTAs owns the
 * instance, CTA r holds the grid points j = r + G n2 of every surface, every
 * solver vector lives in shared memory, the spectral derivative (Sec. II D)
 * takes a length-N/G transform in each CTA plus length-G transforms across
 * the cluster through distributed shared memory, and sums over the state are
 * combined across the cluster in a fixed order.  Needs a QG_C128 state,
 * S * N / G <= 1024, N / G >= 8; applies to forward runs (checkpoint and
 * adjoint runs keep the one-CTA form).  QG_ERR_UNSUPPORTED otherwise.
 * qg_cluster_size gives the smallest G that holds an instance of N points and
 * S surfaces (0: none). */
qg_status qg_state_set_cluster(qg_state_t s, int G);
int qg_cluster_size(int N, int S, int restart);
qg_status qg_state_autotune(qg_state_t s, int method, int order, int scheme, double dt, int64_t trial_steps,
                            const qg_solver_opts* opts, double* ms_out);
qg_status qg_set_state(qg_state_t s, const void* psi, int on_device);
qg_status qg_get_state(qg_state_t s, void* psi, int on_device);
/* Gaussian wavepacket on one surface, zero on the others (Sec. III):
 * psi(q) = prod_d exp(-(q_d - q0_d)^2 / (4 sigma0_d^2) + i p0_d (q_d - q0_d)),
 * normalised on the grid.  q0, p0, sigma0: D entries each. */
qg_status qg_set_gaussian(qg_state_t s, int surface, const double* q0, const double* p0,
                          const double* sigma0);

/* Trigonometric interpolation (Appendix B compares wavepackets on grids of
 * different density this way): dst's state becomes the trigonometric
 * interpolant of src's state, p(q) = (1/N) sum_k c_k exp(i k (q - qmin)),
 * c the DFT of src's samples, the Nyquist term a cosine, evaluated at dst's
 * grid points; points of dst outside src's interval see the periodic
 * extension.  Both 1-D with the same S; the grids may differ in N and range.
 * O(N_src (N_src + N_dst)) direct sums on the device; synchronous. */
qg_status qg_interpolate(qg_state_t src, qg_state_t dst);

/* out = H psi (Eq. adiab_mol_ham by the dynamic Fourier method, Sec. II D);
 * out: S * prod(N_d) complex128, host or device per on_device. */
qg_status qg_apply_h(qg_state_t s, void* out, int on_device);

/* One composed time step dt (Secs. II B, II C): method QG_TRAPEZOIDAL or
 * QG_MIDPOINT, order 2/4/6/8, scheme QG_TRIPLE_JUMP or QG_SUZUKI.  opts may
 * be NULL (defaults); stats may be NULL.
 * Cost in H psi per elementary step (Table I counts 3 + I, I Krylov
 * iterations): trapezoidal 3 + I; midpoint with psi' = 2 chi - psi and the
 * explicit-Euler start 1 + I, plus one exact H psi per composed step, since
 * H psi' = 2 H chi - H psi with H chi = i (chi - psi) / tau is carried from
 * one elementary step to the next (QG_C64_MIXED also carries H^2 psi: two
 * FP64 H psi per elementary step). */
qg_status qg_step_implicit(qg_state_t s, int method, int order, int scheme, double dt,
                           const qg_solver_opts* opts, qg_step_stats* stats);
/* nsteps composed steps in one device launch. */
qg_status qg_propagate(qg_state_t s, int method, int order, int scheme, double dt,
                       int64_t nsteps, const qg_solver_opts* opts, qg_step_stats* stats);

/* Reverse-mode differentiation through a propagation (not in the paper; it
 * relies on the unitarity and exact time reversibility of the composed
 * Cayley maps, Sec. II A-C).
 * qg_state_set_adjoint attaches caller-owned device buffers to a state:
 *   checkpoints: ncheckpoints vectors of S*N complex128 (may be NULL);
 *   every: composed steps between checkpoints (>= 1);
 *   grad: S*N complex128, dL/dpsi at the final time on entry to an adjoint
 *         run, dL/dpsi(0) on exit (torch convention dL = Re sum conj(g) dpsi);
 *   grad_V: S*N doubles and grad_F: S(S-1)/2*N doubles, ACCUMULATED (+=)
 *         with dL/dV_s(q_j) and dL/dF_ab(q_j) (upper-triangle layout).
 * Attach before qg_batch_create when the state is used in a batch.
 * Run kinds for qg_propagate_ex / qg_batch_run_ex:
 *   QG_RUN_FORWARD     plain propagation (= qg_propagate);
 *   QG_RUN_CHECKPOINT  propagation that stores psi before every `every`-th
 *                      composed step into the checkpoints;
 *   QG_RUN_ADJOINT     from psi(t_f) (the state) and grad, steps backward
 *                      nsteps composed steps: psi is re-propagated with
 *                      U(-dt) and reset to the stored checkpoints, the
 *                      adjoint is propagated with U^dagger = U(-dt), and the
 *                      field gradients are accumulated; on exit the state is
 *                      psi(0) and grad is dL/dpsi(0).  FP64 solves; restart
 *                      must be <= 60. */
enum { QG_RUN_FORWARD = 0, QG_RUN_CHECKPOINT = 1, QG_RUN_ADJOINT = 2 };
qg_status qg_state_set_adjoint(qg_state_t s, void* checkpoints, int64_t ncheckpoints, int64_t every, void* grad,
                               double* grad_V, double* grad_F);
qg_status qg_propagate_ex(qg_state_t s, int run, int method, int order, int scheme, double dt, int64_t nsteps,
                          const qg_solver_opts* opts, qg_step_stats* stats);
qg_status qg_batch_run_ex(qg_batch_t b, int run, int method, int order, int scheme, double dt, int64_t nsteps,
                          const qg_solver_opts* opts, int32_t* statuses, qg_step_stats* stats);

/* Observables (Sec. II A): norm ||psi||, energy <psi|H|psi>, populations
 * P_s = ||psi_s||^2 (out: S doubles), overlap <a|b> (out: {re, im}).
 * Results are written to host memory; the call synchronises the stream. */
qg_status qg_norm(qg_state_t s, double* out);
qg_status qg_energy(qg_state_t s, double* out);
qg_status qg_population(qg_state_t s, double* out);
qg_status qg_overlap(qg_state_t a, qg_state_t b, double* out);

/* Batched form: nstates independent states (each with its own model and
 * grid) propagated in ONE persistent launch; each CTA takes instances from
 * an on-device work counter.  statuses / stats: per-instance outputs of
 * nstates entries on the host (either may be NULL).  The stream of states[0]
 * is used.  Returns QG_ERR_NOT_CONVERGED if any instance failed (those
 * instances are restored; the others advance). */
qg_status qg_batch_propagate(qg_state_t* states, int nstates, int method, int order, int scheme,
                             double dt, int64_t nsteps, const qg_solver_opts* opts,
                             int32_t* statuses, qg_step_stats* stats);

/* Reusable batch: the device instance table, work counter and per-instance
 * statistics for a fixed list of states, built once so that repeated
 * qg_batch_run calls allocate nothing.  The states must outlive the batch
 * and keep their models; the stream of states[0] is used. */
qg_status qg_batch_create(qg_state_t* states, int nstates, qg_batch_t* out);
/* Same semantics as qg_batch_propagate on the batch's states.  The batch
 * hands instances to the persistent CTAs longest estimated work first. */
qg_status qg_batch_run(qg_batch_t b, int method, int order, int scheme, double dt, int64_t nsteps,
                       const qg_solver_opts* opts, int32_t* statuses, qg_step_stats* stats);
/* Capture one batch run (the work-counter reset and the single persistent
 * launch of nsteps composed steps) as a CUDA graph, replayed by
 * qg_batch_replay (asynchronous, in the batch's stream); qg_batch_stats then
 * copies the statuses and statistics of the last run to the host
 * (synchronises; same return convention as qg_batch_run).  When the states'
 * stream is the legacy default stream the batch uses a private stream,
 * returned by qg_batch_stream. */
qg_status qg_batch_capture(qg_batch_t b, int method, int order, int scheme, double dt, int64_t nsteps,
                           const qg_solver_opts* opts);
qg_status qg_batch_replay(qg_batch_t b);
/* Autotuner of the batched launch (not in the paper).  A batch is split into
 * grid-size classes (instances of equal N; largest N first), each run as its
 * own persistent launch in the batch's stream, one after another.  For every
 * class the autotuner times trial_steps composed steps of the class's
 * instances under each candidate launch shape -- {1, 2} CTAs per SM x {all
 * surfaces of an instance per shared-memory FFT batch, one surface at a time}
 * for the one-CTA form, then the shared-memory cluster form (see
 * qg_state_set_cluster) at the smallest cluster size that holds the class
 * and at twice that size -- restoring the states after each trial, and keeps
 * the fastest shape per class for later qg_batch_run / qg_batch_capture
 * calls (a captured graph is dropped).  ms_out (6 doubles, may be NULL)
 * receives the trial times of the first class (the largest grid) in that
 * order, -1 for a shape that does not fit.  qg_batch_tuning reports the
 * first class's one-CTA shape (surfaces_per_fft 0 = all), qg_batch_cluster
 * its cluster size (0 = the one-CTA form); qg_batch_classes reports every
 * class (arrays of up to 12 entries, any may be NULL): grid size, instance
 * count and chosen shape.  qg_batch_set_cluster sets the cluster form for
 * every class by hand (QG_ERR_UNSUPPORTED if a class does not fit it). */
qg_status qg_batch_autotune(qg_batch_t b, int method, int order, int scheme, double dt, int64_t trial_steps,
                            const qg_solver_opts* opts, double* ms_out);
qg_status qg_batch_tuning(qg_batch_t b, int* ctas_per_sm, int* surfaces_per_fft);
qg_status qg_batch_cluster(qg_batch_t b, int* G);
qg_status qg_batch_classes(qg_batch_t b, int* nclass, int* grid_n, int* count, int* ctas_per_sm,
                           int* surfaces_per_fft, int* cluster);
qg_status qg_batch_set_cluster(qg_batch_t b, int G);
qg_status qg_batch_stats(qg_batch_t b, int32_t* statuses, qg_step_stats* stats);
void* qg_batch_stream(qg_batch_t b);
void qg_batch_destroy(qg_batch_t b);

/* Propagation without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that are not allowed to allocate GPU
 * memory -- for example a plug-in running inside a host application whose
 * own allocator owns the device memory, or code that must not allocate after
 * start-up.  It propagates one state like qg_propagate but takes every input
 * as a raw pointer (no handles), and keeps all of its scratch (FFT tables,
 * GMRES workspace, statistics) in one fixed device array of about 3 MB that
 * lives in the library for the life of the process on every GPU that loads
 * it.  It calls no cudaMalloc / cudaFree and no allocating library routine.
 *   N: grid points (power of two, 8..8192) on [qmin, qmax); S: 2..4
 *   surfaces, with S * N <= 8192; mass: nuclear mass (electron masses);
 *   V (S*N doubles) and F (S(S-1)/2 * N doubles): device pointers in the
 *   layouts above; psi: device pointer to S*N complex128, read and
 *   overwritten in place; method / order / scheme / dt / nsteps as in
 *   qg_propagate; opts may be NULL (defaults with restart 16; a restart
 *   above 16 is rejected); stats (host) may be NULL; stream: cudaStream_t
 *   (NULL = legacy default stream).  The call returns after the stream has
 *   finished the propagation.
 * The first call on a device looks up the array's device address and builds
 * the FFT tables; make that first call before any stream capture.  Sizes
 * beyond the capacity return QG_ERR_INVALID_ARG with a message in
 * qg_last_error_string().  Every call shares the one array, whose contents
 * persist between calls (nothing in it needs to start at zero: each call
 * rewrites what it reads).  Calls that overlapped on the GPU would race on
 * the array and corrupt each other's results; the library holds a per-device
 * lock from the start of a call until its stream has finished, so calls
 * from several host threads of one process run one after another. */
qg_status qg_propagate_noalloc(int N, double qmin, double qmax, int S, double mass, const double* V,
                               const double* F, void* psi, int method, int order, int scheme, double dt,
                               int64_t nsteps, const qg_solver_opts* opts, qg_step_stats* stats,
                               void* stream);

/* Failure-path self-test of the bounded grid barrier used by 2-D grids (not
 * in the paper): a small cooperative launch in which one CTA never arrives;
 * every other CTA must give up after its wait limit (about a second), raise
 * the error flag and leave.  Returns QG_ERR_TIMEOUT with *timed_out = 1 and
 * *passed = 0 when the time-out path works. */
qg_status qg_selftest_barrier_timeout(int* timed_out, int* passed);

/* FP64 throughput probe of the current device (not in the paper; the
 * denominator of the FP64 roofline): chains of fused multiply-adds and of
 * adds on registers over 8 CTAs per SM, timed with CUDA events, the SM clock
 * read inside the kernel (clock64 against the global timer).  Writes the
 * achieved rates in TFLOP/s (a fused multiply-add counts 2 flops, an add 1),
 * the instructions per SM per clock of each, and the SM clock (GHz) during
 * the FMA run; any pointer may be NULL.  Synchronous, about 0.2 s. */
qg_status qg_probe_fp64(double* fma_tflops, double* add_tflops, double* fma_per_sm_clk, double* add_per_sm_clk,
                        double* sm_ghz);

/* Human-readable name of a status; message of the last CUDA error seen by
 * this thread. */
const char* qg_status_string(qg_status st);
const char* qg_last_error_string(void);
/* Library version string. */
const char* qg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QGEOM_H */
