/*
 * rve.h -- C ABI of the GB300 finite-strain FFT homogenisation solver.
 *
 * The library solves the mechanical equilibrium of a periodic cell on a
 * regular voxel grid with the method of de Geus, Vondrejc, Zeman, Peerlings
 * and Geers, "Finite strain FFT-based non-linear solvers made simple"
 * (CMAME 318, 2017):
 *
 *   G : P(F) = 0,  <F> = F-bar                      (Eq. weak:discr:FFT, Sec. 3.1)
 *
 * by Newton iterations (Algorithm 1) whose linear systems
 *
 *   G : K_(i) : dF = rhs                             (Eq. iter:system, Eq. bc:lin)
 *
 * are solved matrix-free by conjugate gradients.  G is applied in Fourier
 * space with the closed-form G-hat of Eq. G; the per-voxel stress P and
 * tangent K come from the constitutive model (Sec. 4 Saint Venant-Kirchhoff,
 * Sec. 5 finite-strain J2 plasticity).
 *
 * Conventions (all calls):
 *  - Grids are nx x ny x nz voxels, n = nx*ny*nz, voxel v = (x*ny + y)*nz + z
 *    (z fastest).  Eq. G is stated for odd sizes; an axis of even size gets
 *    the treatment of Appendix C: G-hat is zero at every frequency vector
 *    with a Nyquist component (the deformation gradient stays compatible).
 *  - Second-order tensor fields are [9][n] float64, component 3*i+j holding
 *    A_ij; F_ij = dx_i/dX_j (Appendix A).  Fourth-order tangents are [81][n]
 *    with component ((i*3+j)*3+k)*3+l holding K_ijkl in the convention of
 *    Eq. iter:varP:  dP_ji = K_ijkl dF_kl.
 *  - Every function returns RVE_OK (0) or a negative RVE_ERR_* code; the
 *    text of the last error of a handle is returned by rve_last_error().
 *  - Pointers passed with an "_on_device" flag of 0 are host memory, with 1
 *    device memory of the current CUDA device.  Inputs are copied during the
 *    call; the caller keeps ownership of every array it passes.
 *  - All device work of a handle is enqueued on the stream given in
 *    rve_options.stream.  Calls that return host data synchronise that stream.
 *  - The handle owns its device memory: either one block it allocates with
 *    cudaMalloc, or the caller's block given in rve_options.workspace (which
 *    must stay valid until rve_destroy).
 *  - A handle is not thread safe; distinct handles are independent.
 */
#ifndef RVE_H
#define RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RVE_OK 0
#define RVE_ERR_INVALID (-1)      /* bad argument: grid, model, pointer, option */
#define RVE_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define RVE_ERR_NOMEM (-3)        /* device allocation failed / workspace too small */
#define RVE_ERR_CG_MAXIT (-4)     /* CG reached max_cg iterations */
#define RVE_ERR_CG_BREAKDOWN (-5) /* p.Ap = 0 exactly */
#define RVE_ERR_NEWTON_MAXIT (-6) /* Newton reached max_newton iterations */
#define RVE_ERR_NONFINITE (-7)    /* NaN or Inf in a residual, norm or stress */
#define RVE_ERR_DETF (-8)         /* det F <= 0 in some voxel of a converged state */
#define RVE_ERR_TIMEOUT (-9)      /* a bounded device wait gave up */
#define RVE_ERR_UNSUPPORTED (-10) /* valid request the library does not implement */

/* constitutive models */
#define RVE_SVK 0 /* Saint Venant-Kirchhoff (Sec. 4); params per phase: K, mu */
#define RVE_J2 1  /* finite-strain J2 plasticity (Sec. 5); params: K, mu, tau_y0, H */

/* precision of the CG operator */
#define RVE_FP64 0  /* everything in float64 */
#define RVE_MIXED 1 /* CG operator and vectors in float32; residual G:P(F), F and all
                       reductions in float64 (Newton acts as iterative refinement) */

/* storage of the tangent used by the CG operator */
#define RVE_TAN_AUTO 0      /* library choice (RECOMPUTE for SVK, SYM45 for J2) */
#define RVE_TAN_FULL81 1    /* K_ijkl stored, 81 reals per voxel */
#define RVE_TAN_RECOMPUTE 2 /* SVK: dP = dF.S + F.dS recomputed from F (and S) */
#define RVE_TAN_SYM45 3     /* K stored as the upper triangle of the symmetric 9x9 matrix
                               dP_ij/dF_kl (major symmetry K_ijkl = K_lkji of both
                               models), 45 reals per voxel */

/* CG preconditioner (not in the paper, which uses plain CG) */
#define RVE_PRECOND_NONE 0      /* plain CG (Algorithm 1) */
#define RVE_PRECOND_REFERENCE 1 /* reference-medium preconditioner M = G:K0:G, K0 isotropic
                                   with the voxel averages of the Lame parameters; applied as
                                   the inverse acoustic tensor of K0 per frequency in the x
                                   pass; MIXED precision and x lengths with a four-step DFT
                                   kernel (15, 21, 27, 33, 45, 63, 125, 243, 315) only */

/* arithmetic of the mixed path's float64-accuracy transforms */
#define RVE_RES_FLOATFLOAT 0 /* float-float on the float32 pipe: hi + lo float pairs,
                                ~48-bit significand, float64 inputs and outputs */
#define RVE_RES_FP64 1       /* hardware float64 */

typedef struct rve_s* rve_t;

typedef struct {
  int precision;        /* RVE_FP64 (default) or RVE_MIXED */
  int tangent;          /* RVE_TAN_* (default AUTO) */
  int max_newton;       /* default 50 */
  int max_cg;           /* default 10000 */
  double cg_tol_floor;  /* MIXED only: CG tolerance used = max(tol_cg, floor); default 1e-5.
                           MIXED CG also stops after 200 iterations without a 10% drop of
                           ||r|| (float32 accuracy limit); Newton's float64 residual then
                           decides */
  double cg_atol;       /* absolute CG floor: stop when ||r|| <= max(tol ||b||, atol); default 0 */
  int mixed_refine;     /* MIXED only: extra Newton iterations after the convergence test
                           first passes (further refinement with the float64 residual);
                           default 0 */
  int residual;         /* MIXED only: arithmetic of the float64-accuracy transforms (the
                           residual G:P and the projection of dF) and of the SVK
                           constitutive update with the recomputed tangent:
                           RVE_RES_FLOATFLOAT (default) or RVE_RES_FP64 */
  int autotune;         /* MIXED only: 1 = time the float32 CG iteration's kernel
                           variants (DFT engine per axis, z-pass grid and staging) at
                           rve_create on this grid and keep the fastest; the choice
                           is cached per (grid, device, tangent) for the process;
                           default 0 */
  int precond;          /* RVE_PRECOND_* (default NONE).  REFERENCE: every CG solve
                           (Newton, predictor, adjoint, homogenised tangent) runs the
                           preconditioned recurrence z = M^+ r with one transform round
                           trip per iteration, as plain CG; it stops at
                           sqrt(r.z) <= max(tol sqrt(r0.z0), cg_atol), the M^-1-norm of
                           the residual instead of its 2-norm.  The converged Newton
                           state is the same; CG needs fewer iterations as the phase
                           contrast grows */
  void* stream;         /* cudaStream_t; NULL = legacy default stream */
  void* workspace;      /* optional caller-owned device memory (see rve_workspace_size) */
  size_t workspace_bytes;
} rve_options;

#define RVE_MAX_NEWTON_LOG 64

typedef struct {
  int status;                              /* return code of the increment */
  int newton_iters;                        /* linear solves (Algorithm 1 iterations) */
  int cg_iters_total;
  int cg_iters[RVE_MAX_NEWTON_LOG];        /* per Newton iteration */
  double rel_update[RVE_MAX_NEWTON_LOG];   /* ||dF|| / ||F|| per Newton iteration */
  double residual[RVE_MAX_NEWTON_LOG];     /* ||G:P(F)||, float64, after each update */
  double elapsed_ms;                       /* device time of the increment (CUDA events) */
  int substeps;                            /* rve_solve_step: increments solved */
  int cuts;                                /* rve_solve_step: halvings after a failure */
  double substep_to[RVE_MAX_NEWTON_LOG];   /* rve_solve_step / rve_solve_mixed: fraction of
                                              the step reached after each solved increment */
  int macro_iters;                         /* rve_solve_mixed: increments solved as iterates
                                              of the Newton loop on the free F-bar components */
  int tangent_solves;                      /* rve_solve_mixed: linear solves for columns of
                                              the homogenised tangent */
} rve_stats;

/* Fills *opt with the defaults listed above. */
void rve_default_options(rve_options* opt);

/* Device bytes a handle of this grid/model/options needs (for
 * rve_options.workspace).  Returns RVE_ERR_INVALID for unsupported grids. */
int rve_workspace_size(int nx, int ny, int nz, int model, const rve_options* opt, size_t* bytes);

/* Creates a solver for an nx x ny x nz periodic cell with F = I everywhere
 * (Algorithm 1, first line) and evaluates the constitutive model there.
 *  phase        : [n] uint8 phase index per voxel (host), or NULL
 *  nphase       : rows of phase_params (1..256)
 *  phase_params : [nphase][nparam] float64 (host), nparam = 2 (SVK: K, mu)
 *                 or 4 (J2: K, mu, tau_y0, H); K is the bulk modulus
 *                 (lambda = K - 2 mu / 3, Eq. elas:C)
 *  voxel_params : [nparam][n] float64 per-voxel parameters, used when phase
 *                 is NULL; host memory, or device memory of the current
 *                 device (detected; converted on the device without a
 *                 copy through the host)
 *  opt          : may be NULL (defaults)
 * Errors: RVE_ERR_INVALID (non-positive sizes, bad model, phase index
 * >= nphase, missing parameters), RVE_ERR_NOMEM, RVE_ERR_CUDA. */
int rve_create(rve_t* out, int nx, int ny, int nz, int model, int nphase, const uint8_t* phase,
               const double* phase_params, const double* voxel_params, const rve_options* opt);

/* Releases all device memory of the handle (not a caller workspace). */
void rve_destroy(rve_t h);

/* Prescribes the macroscopic deformation gradient F-bar (row-major, host).
 * The next increment applies dF-bar = F-bar - <F> (Sec. 3.1). */
int rve_set_macro_F(rve_t h, const double Fbar[9]);

/* One load increment (Algorithm 1): tangent of the last converged state,
 * predictor G:K:dF = -G:K:dF-bar (Eq. bc:lin), then Newton iterations
 * dF from G:K:dF = -G:P (Eq. iter:system) until ||dF||/||F|| < tol_newton
 * after at least two linear solves; each CG solve stops at
 * ||r|| <= max(tol_cg ||b||, cg_atol).  On success the state is committed;
 * on failure F and the history return to the last committed state and the
 * error code is returned.  st may be NULL. */
int rve_solve_increment(rve_t h, double tol_newton, double tol_cg, rve_stats* st);

/* A load step to the absolute macroscopic F-bar (row-major, host) solved as
 * one or more increments of rve_solve_increment along the straight path from
 * the last committed F-bar: when an increment fails (Newton divergence or
 * max iterations, CG failure, non-finite values, det F <= 0) the state has
 * been rolled back and the increment is retried with half the step; after
 * two successes in a row at one step size the step doubles again (up to the
 * remainder).  Newton is declared diverged when ||dF||/||F|| > 0.5 or the
 * update grew in two consecutive equilibrium iterations.  The step never
 * falls below 2^-max_cuts of the load step (the call fails there); st (may
 * be NULL) accumulates the iterations of all attempts and counts the
 * halvings in st->cuts.  Not in the paper (its
 * examples use fixed small increments, Sec. 5.5); the elasto-plastic switch
 * of Sec. 5.3 makes full Newton steps diverge when an increment crosses the
 * yield point by far. */
int rve_solve_step(rve_t h, const double Fbar[9], double tol_newton, double tol_cg, int max_cuts,
                   rve_stats* st);

/* A load step under mixed macroscopic control.  mask[c] != 0 (c = 3i+j)
 * prescribes P-bar_ij = Pbar[c] and leaves F-bar_ij free; mask[c] == 0
 * prescribes F-bar_ij = Fbar[c] (Fbar and Pbar row-major, host; entries
 * that are not prescribed are ignored).  Not in the paper, which prescribes
 * the full F-bar (Sec. 3.1) and leaves other boundary conditions to the
 * literature.  Each increment seeks the equilibrium G:P(F) = 0 from the
 * committed state with <F>_c = F-bar_c on the strain-controlled and
 * <P>_c = P*_c on the stress-controlled components, by Newton on the free
 * F-bar components (starting at their committed values): every iterate is an
 * increment as in rve_solve_increment (not committed in between), and the
 * Jacobian is the homogenised tangent
 *   dP-bar_a/dF-bar_b = <K : (E_b + dF_b)>_a,  G:K:dF_b = -G:K:E_b
 * (Eq. bc:lin with dF-bar = E_b, the uniform unit tensor of component b;
 * one CG solve per stress-controlled component), evaluated at the first
 * iterate and whenever the stress residual fell by less than 4x, with
 * Broyden's rank-one update otherwise.  The increment has converged when
 * ||P-bar_S - P*_S|| <= tol_stress ||P-bar|| after an iterate (Frobenius
 * norms over the stress-controlled, resp. all, components); at most 30
 * iterates.  Sub-stepping as in rve_solve_step: the prescribed values move
 * on the straight path from the committed F-bar and P-bar, and a failed
 * increment is retried with half the step, at most max_cuts times in a row
 * (max_cuts = 0: one increment).  Without stress-controlled components the
 * call is rve_solve_step.  st (may be NULL): accumulated iterations,
 * macro_iters, tangent_solves, substeps, cuts; elapsed_ms is the wall time
 * of the call.  Errors as rve_solve_increment, plus RVE_ERR_INVALID for
 * non-finite prescribed values or a homogenised tangent that is singular on
 * the stress-controlled components (e.g. a rotation left free at zero
 * stress); the state is then the last committed one. */
int rve_solve_mixed(rve_t h, const double Fbar[9], const double Pbar[9], const int mask[9],
                    double tol_stress, double tol_newton, double tol_cg, int max_cuts,
                    rve_stats* st);

/* F-bar of the last committed state (row-major, host). */
int rve_macro_F(rve_t h, double Fbar[9]);

/* Copies F, P (each [9][n] float64) or the tangent K ([81][n] float64,
 * evaluated in float64 at the current F) to dst (host or device). */
int rve_get_F(rve_t h, double* dst, int dst_on_device);
int rve_get_P(rve_t h, double* dst, int dst_on_device);
int rve_get_K4(rve_t h, double* dst, int dst_on_device);

/* J2 only: committed history, [7][n] float64 = (Cp^-1)_00, _11, _22, _01,
 * _02, _12 and the accumulated plastic strain eps_p (Sec. 5.2), to dst
 * (host or device).  RVE_ERR_INVALID for models without history. */
int rve_get_history(rve_t h, double* dst, int dst_on_device);

/* Gradient of J = W : P-bar (W row-major, host) with respect to the
 * per-voxel shear moduli mu at fixed bulk moduli, at the current converged
 * state, by one adjoint solve (not in the paper; derived from its
 * equilibrium G:P = 0, Eq. weak:discr:FFT): the adjoint field lambda solves
 * G:K:lambda = G:(K:W)/n with the same CG operator (K is symmetric for
 * Saint Venant-Kirchhoff), and
 *   dJ/dmu_v = (1/n) W : (dP/dmu)_v - lambda_v : (dP/dmu)_v,
 *   dP/dmu = F . (2 dev E).
 * The linear solve stops at ||r|| <= tol_cg ||b|| (float32 handles refine
 * float32 CG solutions against the float64 residual).  grad: [n] float64
 * (host or device).  cg_iters (may be NULL) receives the CG iterations.
 * J2: see rve_adjoint_grad_params. */
int rve_adjoint_grad_mu(rve_t h, const double W[9], double tol_cg, double* grad, int grad_on_device,
                        int* cg_iters);

/* As rve_adjoint_grad_mu, and with the same adjoint field also the gradient
 * with respect to the per-voxel bulk moduli K at fixed shear moduli:
 *   dJ/dK_v = (1/n) W : (dP/dK)_v - lambda_v : (dP/dK)_v,
 *   dP/dK = F . (tr(E) I)   (S = (K - 2 mu/3) tr(E) I + 2 mu E, Eq. elas:S, elas:C).
 * grad_K, grad_mu: [n] float64 each (host or device), either may be NULL. */
int rve_adjoint_grad(rve_t h, const double W[9], double tol_cg, double* grad_K, double* grad_mu,
                     int grads_on_device, int* cg_iters);

/* Gradient of J = W : P-bar with respect to every per-voxel material
 * parameter, from one adjoint field: grads [nparam][n] float64 (host or
 * device) in the order of rve_create's parameters -- SVK: K, mu (as
 * rve_adjoint_grad); J2: K, mu, tau_y0, H.  Not in the paper.  J2 (Sec. 5)
 * is path dependent: the derivative is that of the last committed increment
 * with the history at its start held fixed -- the adjoint system uses the
 * consistent tangent of that increment (symmetric), and at fixed F and
 * history
 *   dtau/dK = tr(eps) I,  ds/dmu = 2 e - 3 (dgamma + mu (2 q H + 3 tau_y)/(3 mu + H)^2) e/q,
 *   ds/dtau_y0 = 3 mu/(3 mu + H) e/q,  ds/dH = 3 mu (eps_p + dgamma)/(3 mu + H) e/q
 * in the principal basis of the trial elastic strain (e its deviator,
 * q = sqrt(3/2 e:e), tau_y = tau_y0 + H eps_p; elastic voxels: 2 e for mu,
 * 0 for tau_y0, H), dP = dtau F^-T.  Exact for a path of one increment from
 * the virgin state; for longer paths the contribution of the last increment
 * only (the adjoint through the history of earlier increments is not built).
 * MIXED J2 handles solve the adjoint system in float32 without float64
 * refinement (their tangent is stored in float32), relative accuracy about
 * the CG tolerance floor. */
int rve_adjoint_grad_params(rve_t h, const double W[9], double tol_cg, double* grads,
                            int grads_on_device, int* cg_iters);

/* Path tape of a J2 handle (not in the paper): enable != 0 starts recording,
 * at every committed increment, its converged F and the history at its
 * start (16 float64 per voxel per increment, device memory allocated per
 * increment); 0 stops and frees it.  Any call clears the previous tape, as
 * does rve_set_F.  RVE_ERR_UNSUPPORTED for SVK (path independent).
 * rve_tape_length returns the increments recorded. */
int rve_tape(rve_t h, int enable);
int rve_tape_length(rve_t h);

/* Gradient of J = W : P-bar after the taped path with respect to the
 * per-voxel J2 parameters K, mu, tau_y0, H, through the history of every
 * taped increment (grads [4][n], host or device): a reverse sweep over the
 * increments m = M..1 with a_m = dJ/dh_m (a_M = 0) --
 *   G K_m G lambda_m = G ((1/n) K_M W [m = M] + (dH/dF)^T a_m),
 *   c_m = (1/n) W [m = M] - lambda_m,
 *   dJ/dp += c_m : dP/dp + (dH/dp)^T a_m,   a_{m-1} = c_m : dP/dh + (dH/dh)^T a_m,
 * K_m, P and the new history H at (F_m, h_{m-1}); the return map's
 * derivatives by central differences per voxel (step 1e-7).  The taped path
 * must start at the state the parameters act from (the virgin state, or
 * the state of rve_set_F, which clears the tape) and end at the current
 * state.  Float64 J2 handles only (RVE_ERR_UNSUPPORTED otherwise);
 * RVE_ERR_INVALID for an empty tape. */
int rve_adjoint_grad_path(rve_t h, const double W[9], double tol_cg, double* grads,
                          int grads_on_device, int* cg_iters);

/* Homogenised first Piola-Kirchhoff stress P-bar = <P> (voxel average),
 * row-major, host. */
int rve_homogenized_P(rve_t h, double Pbar[9]);

/* Replaces the deformation field F ([9][n] float64) and re-evaluates P and
 * K there.  The new field becomes the committed state. */
int rve_set_F(rve_t h, const double* F, int src_on_device);

/* out = G : (K : dF) -- one application of the CG operator with the current
 * tangent, in the handle's CG precision (float32 when MIXED).  dF and out are
 * [9][n] float64, both on the host or both on the device. */
int rve_apply_operator(rve_t h, const double* dF, double* out, int on_device);

/* out = G : A in float64 (Eq. weak:discr:FFT-intermediate): hardware
 * float64, or for MIXED handles the arithmetic of rve_options.residual (the
 * transform the mixed path applies to its residual).  A and out are [9][n]
 * float64, both on the host or both on the device. */
int rve_project(rve_t h, const double* A, double* out, int on_device);

/* ---------------------------------------------------------------------------
 * Batches of independent cells of uneven size, solved together: each cell has
 * its own state (as a handle); their CG iterations run as parallel branches
 * of one CUDA graph and their Newton steps in lockstep, converged cells
 * dropping out.  Not in the paper (one cell per run there).
 * ------------------------------------------------------------------------- */
typedef struct rve_batch_s* rve_batch_t;

/* nrve cells; dims [nrve][3]; per cell a phase map (host [n_c] uint8), its
 * number of phases and its parameter table [nphase_c][nparam] (host).  All
 * cells share model and options (opt->workspace must be NULL: every cell
 * allocates its own memory; opt->stream is not used: the batch runs on
 * streams of its own and its calls return after they are idle). */
int rve_batch_create(rve_batch_t* out, int nrve, const int* dims, int model, const int* nphase,
                     const uint8_t* const* phase, const double* const* phase_params,
                     const rve_options* opt);
void rve_batch_destroy(rve_batch_t b);

/* One load increment of every cell to its own F-bar (Fbar [nrve][9],
 * row-major, host).  Same algorithm and tolerances as rve_solve_increment.
 * stats: [nrve] or NULL.  Returns RVE_OK if every cell converged, else the
 * first failure code (failed cells are rolled back; see their stats). */
int rve_batch_solve(rve_batch_t b, const double* Fbar, double tol_newton, double tol_cg,
                    rve_stats* stats);
/* As rve_batch_solve, with the increment cutting of rve_solve_step applied
 * per cell (cells whose increment failed are retried together with half
 * their step, same step control as rve_solve_step); stats[c].substeps / cuts /
 * substep_to report each cell's path. */
int rve_batch_solve_step(rve_batch_t b, const double* Fbar, double tol_newton, double tol_cg,
                         int max_cuts, rve_stats* stats);

int rve_batch_size(rve_batch_t b);
/* Handle of cell i (owned by the batch; use it for rve_get_* calls). */
rve_t rve_batch_cell(rve_batch_t b, int i);
/* P-bar of every cell, [nrve][9] host. */
int rve_batch_homogenized_P(rve_batch_t b, double* Pbar);
int rve_batch_launch_count(rve_batch_t b, long long* count);
const char* rve_batch_last_error(rve_batch_t b);

/* Text of the last error of h (never NULL); rve_status_string maps a code. */
const char* rve_last_error(rve_t h);
const char* rve_status_string(int code);

/* Checkpoint of the converged state (the paper keeps the converged state and
 * history between increments, Algorithm 1): F, the committed F, P, the
 * tangent data, the J2 history, the material in its internal form, F-bar
 * and the kernel variants, written to `path` (host byte order).
 * rve_load creates a new handle from such a file: every solver option comes
 * from the file; opt (may be NULL) supplies only stream and workspace (NULL
 * workspace: the library allocates).  Continuing from a loaded handle gives
 * bit-identical results to continuing the saved one.  The J2 path tape
 * (rve_tape) is not saved: a loaded handle starts without one.
 * RVE_ERR_INVALID for unreadable or malformed files. */
int rve_save(rve_t h, const char* path);
int rve_load(rve_t* out, const char* path, const rve_options* opt);

/* The handle's constitutive model (RVE_SVK, RVE_J2), or RVE_ERR_INVALID
 * for a null handle. */
int rve_model(rve_t h);

/* Grid sizes of a handle. */
int rve_grid(rve_t h, int dims[3]);

/* Kernel variants in use (not in the paper; set by rve_options.autotune or
 * the defaults): knobs[0..5] = four-step z pass, blocks per SM of the
 * persistent z passes, four-step y pass, four-step x pass, composite radices
 * in the Stockham plans, TMA-staged first z pass (1 = on); knobs[6] = 1 if
 * they were autotuned; knobs[7], knobs[8] = tile height of the four-step x
 * and y passes (0: the default number of kz values per tile, 1: half of it,
 * twice the tiles).  Returns RVE_OK. */
int rve_tuning(rve_t h, int knobs[9]);

/* Sets the kernel variants of a handle explicitly (not in the paper), in the
 * layout of rve_tuning (knobs[6] is ignored): e.g. a tuning found by the
 * autotuner in an earlier process.  Values outside 0/1 (1..3 for knobs[1])
 * give RVE_ERR_INVALID; the handle's later calls use the new variants. */
int rve_set_tuning(rve_t h, const int knobs[9]);

/* Instrumentation: number of kernels this handle has launched, and optional
 * CUDA-event timing of every launch of one kernel family
 * (0 zfwd, 1 fft_y fwd, 2 fft_x+projection, 3 fft_y inv, 4 zinv, 5 cg_update;
 * the float32 CG iteration of RVE_MIXED has no family 5: its vector update
 * is fused into families 0 and 4).
 * rve_kernel_time returns the summed milliseconds and launches since the
 * timing was enabled (synchronises the stream). */
int rve_launch_count(rve_t h, long long* count);
int rve_kernel_timing(rve_t h, int family, int enable);
int rve_kernel_time(rve_t h, double* total_ms, long long* launches);

/* Failure-test setting (the paper has no counterpart): the number of polls a
 * thread block's bounded wait on its own asynchronous (TMA) copies makes
 * before it gives up, marks the solver state and lets the call end with
 * RVE_ERR_TIMEOUT after rolling back to the committed state.  The default
 * is 1 << 20 polls (far longer than a copy takes); 0 makes every first wait
 * give up at once, which exercises the timeout path without a fault: after
 * giving up a block still waits (bounded) for its copies to land before it
 * touches the staged data again.  Applies to the handle's later calls.
 * Returns RVE_OK, or RVE_ERR_INVALID for a null handle. */
int rve_set_wait_polls(rve_t h, unsigned polls);

/* ---------------------------------------------------------------------------
 * Allocation-free projection.  (The paper has no counterpart: this entry
 * point exists for callers of this library that cannot allocate device
 * memory -- plugins of a host program that owns every device allocation
 * itself and hands out only its own buffers, and real-time paths where an
 * allocation, with the implicit device synchronisation it may bring, is not
 * allowed.)
 *
 * out = G : A in float64, the same operation as rve_project, without a
 * handle and without allocating anything: its scratch (the float64 half
 * spectrum, 9*nx*ny*(nz/2+1 rounded up to a multiple of 4) complex values,
 * plus the twiddle tables) lives in one fixed device array of
 * RVE_NOALLOC_SCRATCH_BYTES that the library reserves on every GPU that
 * loads it, for the life of the process.  Odd and even sizes are accepted
 * (even axes take G-hat = 0 at their Nyquist frequency, Appendix C).
 *  A, out : [9][n] float64 in device memory of the current device; out may
 *           equal A.  The caller owns both; the library cannot check their
 *           lengths, so each must hold 9*nx*ny*nz values.
 *  stream : cudaStream_t (NULL = legacy default stream).  The call only
 *           enqueues work; synchronise the stream before reading out.
 * The first call on a device does the set-up for that device, with it
 * current: one cudaGetSymbolAddress for the array's device address (cached
 * for the process) and the kernels' shared-memory attributes.  Make that
 * first call before any stream capture.  cudaDeviceReset invalidates the
 * cached address: do not use this entry point after resetting a device.
 * All calls on a device share the one array and it keeps the last call's
 * contents (each call rewrites everything it reads, so nothing is cleared):
 * calls whose work overlaps on the GPU (different streams without ordering,
 * or concurrent host threads) race on it.
 * Errors: RVE_ERR_INVALID (null pointer, a size below 1 or above 2047, or
 * a line too long for the transform kernels' shared-memory tiles),
 * RVE_ERR_NOMEM (the grid's scratch exceeds RVE_NOALLOC_SCRATCH_BYTES, e.g.
 * 63^3), RVE_ERR_UNSUPPORTED (device ordinal 64 or above), RVE_ERR_CUDA. */
#define RVE_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int rve_project_noalloc(int nx, int ny, int nz, const double* A, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RVE_H */
