/*
 * fse.h -- C ABI of the GB300-native FSE-Shooting hot path.
 *
 * FSE-Shooting (Fourier-series-expansion shooting, arXiv 2508.06302) finds a
 * quasi-periodic response of  M q'' + D q' + K q + f_nl(q) = sum_i F_i cos(w_i t)
 * (Eq. 1 with Theta = I, Eq. 25) as the Fourier coefficients Z(0) of the
 * (d-1)-torus of trajectory start points that satisfy the coupling residual
 *     R(Z(0), w) = (I_2n (x) R(rho)) Z(2 pi) - Z(0)                   (Eq. 16)
 * evaluated by  Z(0) -i-DFT-> zbar(0) -Newmark-> zbar(2 pi) -DFT-> Z(2 pi)
 * (Eq. 17, Eq. 20, Eq. 21, App. E).
 *
 * Conventions shared by every entry point
 *  - Real numbers are IEEE double unless stated.  Matrices are dense,
 *    row-major.  All pointers without a _dev suffix are HOST pointers; the
 *    library copies what it needs and never keeps a caller pointer.
 *  - The state is z = [q; u] with u = dq/dphi_1 = qdot / w_1 (App. E, Eq. E8).
 *  - Z vectors are state-major: Z[i * U + c] is coefficient c of state i,
 *    i < 2n, in the basis of Eq. (11) [1, cos k_1.phi, sin k_1.phi, ...].
 *  - The frequency ratios rho_j = w_j / w_1 (j = 2..d) are fixed per context,
 *    so the torus rotation and the forcing phases do not depend on w_1.
 *  - Return value: FSE_OK (0) or a negative FSE_E* code; fse_last_error()
 *    gives a one-line text.  The library never aborts or traps; every device
 *    loop has a fixed bound.
 *  - A context is not thread-safe; distinct contexts may be used from
 *    distinct host threads.  All work of a context runs on its stream.
 */
#ifndef FSE_H
#define FSE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FSE_OK 0
#define FSE_EINVAL (-1)        /* bad size / pointer / Nyquist rule / option */
#define FSE_ENOMEM (-2)        /* device allocation failed                   */
#define FSE_ENOCONV (-3)       /* per-step Newton hit its iteration limit    */
#define FSE_ENONPOS_PIVOT (-4) /* effective stiffness not positive definite  */
#define FSE_ENAN (-5)          /* non-finite value in a result               */
#define FSE_ECUDA (-6)         /* CUDA runtime error                         */
#define FSE_ENOJAC (-7)        /* no Jacobian stored in the context yet      */

/* Nonlinear element types of f_nl(q, qdot) (Eq. 1).  Only FSE_NL_VDP depends on qdot: its
 * velocity tangent C_t = d f / d qdot enters the effective stiffness as w_1 (2/Delta) C_t and
 * the sensitivity recurrence of App. E. */
#define FSE_NL_CUBIC_GROUND 1  /* f[d0] += p0 q[d0]^3                          */
#define FSE_NL_CUBIC_DIFF 2    /* s = q[d0]-q[d1]: f[d0] += p0 s^3, f[d1] -= p0 s^3 */
#define FSE_NL_VK_BEAM 3       /* 2-node von Karman beam, dofs (u1,w1,th1,u2,w2,th2),
                                  p0 = EA, p1 = length; force = gradient of
                                  EA/2 int (u' w'^2 + w'^4/4) dx; dof -1 = clamped */
#define FSE_NL_VDP 4           /* self-excited (van der Pol) damper:
                                  f[d0] += p0 (q[d0]^2 - 1) qdot[d0]                */

/* Precision of the sensitivity (monodromy) propagation.  The trajectory
 * state, the per-step Newton residual and test, the coupling residual and
 * the outer solve are FP64 in every mode. */
#define FSE_FP64 0             /* plain: sensitivities FP64                    */
#define FSE_MIXED_FP32 1       /* sensitivities + factorisation FP32           */

typedef struct {
    int type;                  /* FSE_NL_*                                     */
    int dof[6];                /* global dof indices, -1 = unused / clamped    */
    double p[6];               /* parameters, see FSE_NL_*                     */
} fse_nl_elem;

typedef struct {
    int n;                     /* number of dofs                               */
    const double* M;           /* n x n mass, symmetric positive definite      */
    const double* D;           /* n x n viscous damping, symmetric             */
    const double* K;           /* n x n linear stiffness, symmetric            */
    int n_nl;                  /* number of nonlinear elements (>= 0)          */
    const fse_nl_elem* nl;     /* n_nl records                                 */
    int e;                     /* number of forcing components, 1 <= e <= d    */
    const double* F;           /* e x n amplitudes: e(t) = sum_i F_i cos(w_i t) */
} fse_model;

typedef struct {
    int d;                     /* base frequencies, 2 <= d <= 4                */
    const int* S;              /* d-1 sample counts S_j; N = prod S_j          */
    const int* H;              /* d-1 highest harmonics; S_j >= 2 H_j + 1      */
    const double* rho;         /* d-1 fixed ratios rho_j = w_j / w_1           */
    int S1;                    /* Newmark steps per period T_1 = 2 pi / w_1    */
    double newton_tol;         /* per-step Newton: ||dq||_inf <= tol ||q||_inf;
                                  tol <= 0 runs exactly newton_maxit iterations */
    int newton_maxit;          /* 1..64                                        */
    int precision;             /* FSE_FP64 or FSE_MIXED_FP32                   */
} fse_opts;

typedef struct fse_ctx fse_ctx;

/* fse_setup -- validate and copy the model and options to the GPU, build the
 * harmonic table (App. B), the sample grid and Gamma / Gamma^-1 (App. D), the
 * rotation R(rho) (Eq. 14) and the banded forms of M, D, K (the half-bandwidth
 * b is detected from the exact zeros of M, D, K and the element dof spans).
 * Allocates all device memory of the context.  Errors: FSE_EINVAL for bad
 * sizes, the sampling rule S_j >= 2 H_j + 1 (Sec. 3.1), e > d, an element dof
 * out of range or a non-positive-definite M (FSE_ENONPOS_PIVOT); FSE_ENOMEM.
 * FSE_EINVAL also when the model exceeds the kernels' on-chip working set
 * (message "n or half-bandwidth too large for the on-chip working set"):
 * b > 224, or b > 96 with FSE_FP64 tangents (the solves keep b + 32 solved rows
 * of 128 or 256 columns in shared memory), or n beyond the state kernel's
 * shared-memory vectors (about n > 3600 mixed, n > 2700 FP64, at b near 90).
 * On error *out is NULL.  device < 0 uses the current device. */
int fse_setup(const fse_model* model, const fse_opts* opts, int device, fse_ctx** out);

/* fse_setup for a trajectory shard: the context integrates only samples s_begin .. s_end - 1
 * of the N-sample grid of opts (sample order of Eq. D1), with the grid's phases and the Gamma /
 * Gamma^-1 entries of those samples (Eq. D2, D3, normalised by the whole N).  Trajectories are
 * independent within an evaluation, so the shards of a torus can run on different GPUs; only the
 * DFT sums over samples (Eq. 21, 22, 23) couple them.  On a shard context the residual, J v,
 * dR/dw_1 and the hyper-time residual are completed by the reduction set with fse_set_reduce:
 * the library forms this shard's partial sum, hands it to the reduction (which must return the
 * sum over all shards in the same buffer) and subtracts Z0 / v afterwards.  Without a reduction
 * those outputs are the partial sums (nothing subtracted).  Entry points that need every
 * monodromy in one place (fse_jacobian_dense, the dense outer solve, fse_lyapunov*,
 * fse_monodromy) return FSE_EINVAL on a shard.  Errors as fse_setup; FSE_EINVAL for a range
 * outside [0, N). */
int fse_setup_shard(const fse_model* model, const fse_opts* opts, int s_begin, int s_end, int device,
                    fse_ctx** out);

/* Reduction of partial DFT sums across shards: called synchronously (the context's stream has
 * finished) with `count` doubles of this shard's partial sums in device memory at buf_dev; it
 * must leave the sum over all shards (the same count, every shard's buffer in the same
 * order) in buf_dev before returning, and return 0 (non-zero aborts the call with FSE_ECUDA).
 * stream is the context's stream (a cudaStream_t). */
typedef int (*fse_reduce_fn)(void* user, double* buf_dev, size_t count, void* stream);

/* Set (or clear with fn = NULL) the reduction of a shard context.  FSE_EINVAL on a context that is
 * not a shard. */
int fse_set_reduce(fse_ctx* ctx, fse_reduce_fn fn, void* user);

/* Wait for the context's work, free all its device memory and the handle.
 * NULL is ignored. */
void fse_destroy(fse_ctx* ctx);

/* Text of the last error of ctx (or of the last failed fse_setup if ctx is NULL). */
const char* fse_last_error(const fse_ctx* ctx);

/* Sizes: unknowns 2 n U~, U~ = prod (2 H_j + 1), N = prod S_j, n, half-bandwidth b. */
int fse_sizes(const fse_ctx* ctx, int* n_unknowns, int* U_tilde, int* N, int* n, int* band);

/* Harmonic table K~^d of App. B (Eq. B1-B2): (U~+1)/2 rows of d-1 ints,
 * rows k~_1..k~_L first, the zero row last.  ktilde is caller-owned. */
int fse_harmonics(const fse_ctx* ctx, int* ktilde);

/* fse_residual_jacobian -- one evaluation of Eq. (16) at (Z0, w_1).
 *  Z0      host, 2 n U~ doubles (state-major)
 *  R_out   host, 2 n U~ doubles: R = (I (x) R(rho)) Z(2 pi) - Z0
 *  want_jacobian: 0 = residual only; 1 = also propagate the sensitivities
 *          and keep the monodromy blocks Phi_s = d zbar_s(2 pi)/d zbar_s(0)
 *          (Eq. E8) and d zbar(2 pi)/d w_1 on the device for
 *          fse_jacobian_apply / _domega / _dense / fse_monodromy.
 *  traj_status host, N ints or NULL: per-trajectory 0 = ok, FSE_ENOCONV,
 *          FSE_ENONPOS_PIVOT, FSE_ENAN.
 *  newton_iters host, N ints or NULL: total per-step Newton iterations.
 * Returns the worst per-trajectory status (FSE_OK if all converged). */
int fse_residual_jacobian(fse_ctx* ctx, const double* Z0, double omega1, double* R_out,
                          int want_jacobian, int* traj_status, int* newton_iters);

/* Same on device memory: Z0_dev / R_dev are device pointers (2 n U~ doubles)
 * and the call is asynchronous with respect to the host.  `stream` (a
 * cudaStream_t, NULL = the legacy default stream) is ordered before the
 * evaluation and waits for its end; the work itself runs on the context's
 * two streams (state path and sensitivities overlap).  The status of the run
 * is read with fse_status(). */
int fse_residual_jacobian_dev(fse_ctx* ctx, const double* Z0_dev, double omega1, double* R_dev,
                              int want_jacobian, void* stream);

/* Waits for the context stream and returns the worst trajectory status of
 * the last evaluation (copied to traj_status / newton_iters when non-NULL). */
int fse_status(fse_ctx* ctx, int* traj_status, int* newton_iters);

/* Eq. (22) applied without forming J:  Jv = (I (x) R Gamma^-1) blockdiag(Phi_s)
 * (I (x) Gamma) v - v for nvec vectors of 2 n U~ doubles each (host, packed). */
int fse_jacobian_apply(fse_ctx* ctx, const double* v, double* Jv, int nvec);

/* Eq. (23), i = 1, rho fixed: dR/dw_1 = (I (x) R Gamma^-1) d zbar(2 pi)/d w_1. */
int fse_jacobian_domega(fse_ctx* ctx, double* dRdw1);

/* Dense dR/dZ(0) of Eq. (22), (2 n U~)^2 doubles, row-major.  FSE_EINVAL if
 * the matrix would exceed 2^31 entries. */
int fse_jacobian_dense(fse_ctx* ctx, double* J);

/* Copy the monodromy blocks Phi_s (N x 2n x 2n, row-major) and
 * d zbar_s(2 pi)/d w_1 (N x 2n) of the last evaluation (either may be NULL). */
int fse_monodromy(fse_ctx* ctx, double* Phi, double* dz_dw);

/* The monodromy block Phi_s (2n x 2n, row-major) and d zbar_s(2 pi)/d w_1 (2n)
 * of trajectory s of the last evaluation (either may be NULL): one block of
 * fse_monodromy without copying all N.  FSE_EINVAL for s outside [0, N). */
int fse_monodromy_traj(fse_ctx* ctx, int s, double* Phi, double* dz_dw);

/* One Newton-Raphson update of Z(0) at fixed w_1 (Sec. 3.3 step 6): evaluates
 * R and J at Z0, solves J dZ = -R on the GPU with the solver chosen by
 * fse_set_linear_solver (dense LU up to 16384 unknowns, matrix-free GMRES
 * above by default) and overwrites Z0 <- Z0 + dZ.  res_norm_out receives
 * ||R(Z0_in)||_2.  Returns the evaluation status, FSE_ENOCONV also when GMRES
 * stops above its tolerance (the update is still applied). */
int fse_newton_step(fse_ctx* ctx, double* Z0, double omega1, double* res_norm_out);

/* Outer linear solver of fse_newton_step and fse_continue (Sec. 3.3 step 6,
 * J dZ = -R with J of Eq. 22).  FSE_LIN_DENSE: the dense J is formed on the
 * GPU and factorised by LU with partial pivoting (2 n U~ <= 16384);
 * FSE_LIN_GMRES: restarted GMRES(restart) in FP64 on the structured products
 * J v = (I (x) R Gamma^-1) blockdiag(Phi_s) (I (x) Gamma) v - v, which read the
 * monodromies in place (no dense J), stopped at ||J dZ + R|| <= rel_tol ||R||
 * or after max_iters products; FSE_LIN_AUTO (default): dense up to 16384
 * unknowns, GMRES above.  Defaults rel_tol 1e-8, restart 40, max_iters 400.
 * The GMRES basis ((restart + 1) x 2 n U~ doubles) is allocated on first use
 * and kept by the context.  Returns FSE_EINVAL for an unknown kind or
 * restart outside [1, 256]. */
#define FSE_LIN_AUTO 0
#define FSE_LIN_DENSE 1
#define FSE_LIN_GMRES 2
int fse_set_linear_solver(fse_ctx* ctx, int kind, double rel_tol, int restart, int max_iters);

/* Kernels of the banded tangent solves (App. E: the 2n+1 sensitivity columns of every
 * trajectory through the factor L L^T of K_eff, forward L Y' = Y then backward L^T X = Y' with
 * the Newmark update of V).  FSE_SOLVE_SIMT: blocked substitution on the FP32/FP64 FMA pipes.
 * FSE_SOLVE_TC: the FP32 tangents on the TF32 tensor cores (tcgen05, accumulators in tensor
 * memory) with both operands split into a TF32 high part and an FP32 remainder and three
 * products per pair, which keeps FP32-level products; only for FSE_MIXED_FP32 contexts with
 * half-bandwidth b <= 96.  The tensor cores accumulate with truncation, so the TC tangents carry
 * a biased error of a few FP32 ulps per block solve that grows along the period: about ten times
 * the SIMT error on short periods, 1e-2 relative on the monodromy of the 1872-dof shell's
 * 1000-step period, where Newton no longer converges quadratically.  FSE_SOLVE_AUTO (default):
 * the SIMT solves.
 * Returns FSE_EINVAL for an unknown kind or FSE_SOLVE_TC where it does not apply. */
#define FSE_SOLVE_AUTO 0
#define FSE_SOLVE_SIMT 1
#define FSE_SOLVE_TC 2
int fse_set_tangent_solve(fse_ctx* ctx, int kind);

/* Statistics of the last outer linear solve: Krylov iterations (0 for the
 * dense solve) and the relative residual ||J dZ + R|| / ||R|| it reached
 * (GMRES estimate; 0 for the dense solve). */
int fse_linear_stats(const fse_ctx* ctx, int* iters, double* rel_res);

/* ------------------------------------------------------------------------
 * A priori unknown base frequencies (Sec. 3.2).  With e forcing components and d > e
 * base frequencies, w_i for i > e is set by no forcing (a self-excited oscillation): it
 * joins Z(0) as an unknown (Eq. Cont1), and the torus, which any shift along phi_i
 * maps to another solution, is pinned by one phase condition per unknown (Eq. 18 with
 * the gradient of Eq. 19).  w_1 stays fixed; w_i = rho_{i-1} w_1.
 * ------------------------------------------------------------------------ */

/* Set the frequency ratios rho_j = w_{j+1} / w_1 (d-1 doubles, host): rebuilds the rotation
 * R(rho) of Eq. 14 and the tables that hold it, and drops the stored Jacobian.  Contexts in a
 * graph batch must be re-batched after a change. */
int fse_set_rho(fse_ctx* ctx, const double* rho);

/* One Newton update of (Z(0), w_u) at fixed w_1 (Sec. 3.3 step 6 for Eq. Cont1):
 * unknown (d-1 ints, host): unknown[j] != 0 makes w_{j+2} an unknown (FSE_EINVAL if forcing
 * component j+1 moves with it, i.e. j + 1 < e); rho (d-1 doubles, host, in/out) holds the current
 * ratios and receives the updated ones; Z0 (host, in/out) as for fse_newton_step.  The system is
 *   [ J       dR/dw_u ] [dZ  ]     [R]
 *   [ G_u^T   0       ] [dw_u] = - [0]
 * with J of Eq. 22, dR/dw_u = (2 pi / w_1) (I (x) Upsilon_u) (I (x) R(rho)) Z(2 pi) (Eq. 23, 24,
 * rotation term only: no trajectory moves with an unforced w_u) and the phase-condition rows
 * G_u = (I (x) grad_u) Z0 (Eq. 18, 19), solved by dense LU (2 n U~ + u <= 16384) or GMRES on the
 * bordered products, per fse_set_linear_solver.  res_norm_out (nullable): ||R(Z0_in)||_2.
 * Returns as fse_newton_step. */
int fse_newton_step_unknown(fse_ctx* ctx, double* Z0, double omega1, double* rho, const int* unknown,
                            double* res_norm_out);

/* ------------------------------------------------------------------------
 * FSE-Shooting in the hyper-time domain (Sec. 3.4, Eq. FSES_T).  The unknowns are the
 * start points zbar(0, phi~_s) of the N trajectories themselves, stored sample-major
 * (N x 2n doubles, row s = [q; u] of trajectory s, the sample order of Eq. D1), instead of
 * their Fourier coefficients.  The residual maps the end points back through the
 * band-limited interpolant of the context's harmonics and rotates them:
 *     R_T = (I_2n (x) Gamma R(rho) Gamma^-1) zbar(2 pi) - zbar(0),
 * with Jacobian J_T = (I (x) Gamma R Gamma^-1) blockdiag(Phi_s) - I.  N may exceed U~ (more
 * samples than coefficients); where zbar(0) = (I (x) Gamma) Z(0) the residual is
 * (I (x) Gamma) R(Z(0)) of Eq. (16), so both forms share their tori.  The integration, the
 * stored monodromies, the precision and the outer-solver settings are the context's.
 * ------------------------------------------------------------------------ */

/* One evaluation of R_T at (zbar0, w_1): zbar0 and RT_out host, N x 2n doubles;
 * want_jacobian, traj_status and newton_iters as for fse_residual_jacobian (the stored
 * monodromies also serve fse_jacobian_apply and friends).  Returns the worst trajectory
 * status, FSE_ENOMEM if the form's buffers (4 N 2n + 2n U~ + N^2 doubles, allocated on first
 * use and kept by the context) cannot be allocated. */
int fse_residual_jacobian_hypertime(fse_ctx* ctx, const double* zbar0, double omega1, double* RT_out,
                                    int want_jacobian, int* traj_status, int* newton_iters);

/* J_T v for nvec vectors of N x 2n doubles (host, packed), from the monodromies of the last
 * evaluation with want_jacobian (FSE_ENOJAC if there is none). */
int fse_jacobian_apply_hypertime(fse_ctx* ctx, const double* v, double* Jv, int nvec);

/* One Newton update of zbar0 (host, N x 2n, in/out) at fixed w_1: evaluates R_T and J_T,
 * solves J_T dz = -R_T with the solver of fse_set_linear_solver (dense J_T and LU with partial
 * pivoting up to 16384 unknowns, else GMRES on the products above) and adds dz.  res_norm_out
 * (nullable) receives ||R_T(zbar0_in)||_2.  Returns the evaluation status, FSE_ENOCONV also when
 * GMRES stops above its tolerance (the update is still applied). */
int fse_newton_step_hypertime(fse_ctx* ctx, double* zbar0, double omega1, double* res_norm_out);

/* First-order Lyapunov exponents (App. F) of the torus at (Z0, w_1), 1/s,
 * from the monodromy by-product: Psi_s = diag(I, w_1 I) Phi_s diag(I, I/w_1)
 * (Eq. F3), trigonometric interpolation of Psi over phi~ with the context
 * harmonics at phi~ = 2 (i-1) pi rho, QR re-orthonormalisation for
 * i = 1..N_Ly, sigma_j = sum_i ln|R_i[j,j]| / (N_Ly T_1), j < h.
 * Re-evaluates the Jacobian at Z0 in the context precision (create the
 * context with FSE_FP64 for the certified exponents).  1 <= h <= min(64, 2n).
 * sigma_out: h doubles (host). */
int fse_lyapunov(fse_ctx* ctx, const double* Z0, double omega1, int N_Ly, int h,
                 double* sigma_out);

/* Size limits of fse_lyapunov_noalloc: 2 n h doubles for each of its Q and A
 * blocks, and N trajectories. */
#define FSE_NOALLOC_MAX_QH 262144
#define FSE_NOALLOC_MAX_N 65536

/* fse_lyapunov without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc or cudaFree
 * while they run -- a process that gives all device memory to its own pool at
 * start-up and allows no other allocation, or a latency-bound loop that cannot
 * take the device-wide synchronisation cudaFree implies.  Arguments, result and
 * status are those of fse_lyapunov; the trajectory buffers are the context's
 * (allocated once by fse_setup) and the propagation scratch is one static
 * device array of 4.5 MiB that every GPU loading this library holds until the
 * process exits.  Limits: h <= 64, 2 n h <= FSE_NOALLOC_MAX_QH,
 * N <= FSE_NOALLOC_MAX_N; a larger size returns FSE_EINVAL (message in
 * fse_last_error) before anything runs.  The first call on a device looks up
 * the array's device address and caches it: make that first call before any
 * stream capture on that device.  Every call in the process shares the array,
 * which keeps the last call's contents (each call re-initialises what it
 * needs); calls that overlap on the GPU -- from other contexts, streams or
 * host threads -- race on it, so the caller must serialise them. */
int fse_lyapunov_noalloc(fse_ctx* ctx, const double* Z0, double omega1, int N_Ly, int h,
                         double* sigma_out);

typedef struct fse_batch fse_batch;

/* Several contexts evaluated together (the paper evaluates one point at a time;
 * this runs the residual and Jacobian of Eq. 16 / Eq. 22 for a set of
 * continuation points, possibly of different N and H, concurrently).  All
 * contexts must be on one device and distinct; the batch does not own them
 * (destroy the batch before its contexts).  use_graph = 0: the evaluations are
 * enqueued back to back on the contexts' own streams and overlap on the GPU.
 * use_graph = 1: the evaluations of all contexts (every Newmark step of their
 * two-stream loops) are captured once into one CUDA graph on the batch's own
 * stream and replayed by later calls with the same w_1 values and
 * want_jacobian; a change of either re-captures it.  Per-kernel profiling of
 * the contexts must be off in graph mode. */
int fse_batch_create(fse_ctx* const* ctxs, int count, int use_graph, fse_batch** out);
/* Free the batch (its stream, events and graph; not the contexts). */
void fse_batch_destroy(fse_batch* batch);
/* Text of the last batch error. */
const char* fse_batch_last_error(const fse_batch* batch);
/* Evaluate every context of the batch: Z0[i] (host, 2 n_i U~_i doubles, the
 * layout of fse_residual_jacobian) at omega1[i] -> R_out[i] (host); the
 * Jacobian (monodromies and the w_1 column) stays in each context as after
 * fse_residual_jacobian with want_jacobian.  status_out (nullable, count ints)
 * receives each context's status.  Returns FSE_OK, FSE_ENOCONV (some
 * per-step Newton did not converge) or the first error. */
int fse_batch_residual_jacobian(fse_batch* batch, const double* const* Z0, const double* omega1,
                                double* const* R_out, int want_jacobian, int* status_out);

/* Integrate only the first n_steps (> 0) Newmark steps of the period in the
 * following evaluations; 0 restores the full period S1.  With n_steps < S1
 * the "residual" is the DFT of the truncated trajectories' end states minus
 * Z0 and the monodromy covers the truncated map: meant for sampled timing and
 * sampled parity checks of large workloads. */
int fse_set_steps(fse_ctx* ctx, int n_steps);

/* Enable (1) or disable (0) per-kernel timing: CUDA events are recorded
 * around every launch of the step loop on the context stream. */
int fse_profile(fse_ctx* ctx, int enable);

/* Device time of the last evaluation, milliseconds, up to `cap` values:
 * [0] whole evaluation; with fse_profile on: summed kernel time of
 * [1] the per-step state Newton + K_eff assembly + banded Cholesky,
 * [2] the sensitivity right-hand side, [3] the forward and [4] the backward
 * banded substitutions of the sensitivities (the latter includes the
 * Newmark update of the tangents), and [5] the mean number of in-loop
 * refactorisations of the per-step Newton per trajectory-step.  Filled by
 * fse_status() / the blocking entry points. */
int fse_timings(fse_ctx* ctx, double* ms, int cap);

/* ------------------------------------------------------------------------
 * Learned continuation predictor (not in the paper).  A 3-layer MLP
 * n_in -> n_hidden -> n_hidden -> n_out with the exact GELU
 * gelu(z) = z (1 + erf(z / sqrt 2)) / 2 between layers maps normalised point
 * parameters (w_1, w_2, F_1) to the coefficients of the torus in a POD basis of
 * converged solutions.  Kernels keep weights, inputs and activations in BF16,
 * accumulate in FP32 and keep FP32 master weights for Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  Loss: 1/(2B) sum (y - t)^2.
 * Flat parameter order W1, b1, W2, b2, W3, b3 (W row-major, out x in).
 * All data pointers are host float arrays, row-major (sample-major).
 * ------------------------------------------------------------------------ */
typedef struct fse_mlp fse_mlp;

/* Create a network with zero parameters (set them with fse_mlp_set_params),
 * batches up to max_batch samples; device < 0 uses the current device. */
int fse_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, int device, fse_mlp** out);

/* Free the network and its device memory; NULL is ignored. */
void fse_mlp_destroy(fse_mlp* mlp);

/* Number of parameters of the flat vector. */
int fse_mlp_nparams(const fse_mlp* mlp);

/* Number of outputs n_out. */
int fse_mlp_nouts(const fse_mlp* mlp);

/* Text of the last error of the network. */
const char* fse_mlp_last_error(const fse_mlp* mlp);

/* Set the FP32 master parameters (resets the Adam state). */
int fse_mlp_set_params(fse_mlp* mlp, const float* flat);

/* Copy the FP32 master parameters out. */
int fse_mlp_get_params(fse_mlp* mlp, float* flat);

/* Y (B x n_out) = network(X (B x n_in)), 1 <= B <= max_batch. */
int fse_mlp_forward(fse_mlp* mlp, const float* X, int B, float* Y);

/* Loss and gradient (flat, nullable) of the batch against the targets T. */
int fse_mlp_grad(fse_mlp* mlp, const float* X, const float* T, int B, float* loss, float* grad);

/* `steps` Adam steps of full-batch training with learning rate lr; loss (nullable)
 * receives the loss after the last step. */
int fse_mlp_train(fse_mlp* mlp, const float* X, const float* T, int B, int steps, float lr, float* loss);

/* POD basis of m snapshots (rows of `snaps`, m x nu doubles): mean (nu), the r
 * leading orthonormal modes (r x nu) of the mean-centred snapshots (method of
 * snapshots: Jacobi eigen-decomposition of the m x m Gram matrix on the GPU)
 * and their singular values (nullable).  r <= m <= 1024. */
int fse_pod_build(const double* snaps, int nu, int m, int r, double* mean, double* basis, double* sing);

/* ------------------------------------------------------------------------
 * One-parameter continuation in w_1 (App. C, natural parameter with the
 * frequency ratios fixed, Eq. Cont2).  Point j is predicted, then corrected by
 * Newton on Eq. (16) at fixed w_1 until ||R||_2 <= rel_tol ||Z(0)||_2.
 * Predictors: the secant S_j through the last two accepted points, or the
 * secant corrected by the network (from point max(4, warmup) on):
 * Z = S_j + mean + sum_k c_k mode_k, c from the MLP fed (w_1, w_2, F_1)
 * normalised to [-1, 1] over [omega_lo, omega_hi].  The network learns the
 * secant's own error: after every accepted point j >= 2 the correction
 * Z_j - S_j is stored, the POD of the corrections is rebuilt every pod_every
 * points and the network is trained on their coefficients (each mode divided
 * by its RMS over the corrections, the scale the prediction multiplies back;
 * modes below 1e-8 of the first are not learned) for train_steps
 * Adam steps after every point.  The outer linear solve is the one of
 * fse_newton_step (fse_set_linear_solver).
 * ------------------------------------------------------------------------ */
#define FSE_PRED_SECANT 0
#define FSE_PRED_MLP 1

typedef struct {
    int n_points;              /* number of w_1 values                          */
    const double* omega1;      /* host, n_points values in sweep order          */
    int predictor;             /* FSE_PRED_SECANT or FSE_PRED_MLP               */
    double rel_tol;            /* acceptance ||R|| <= rel_tol ||Z|| (1e-10)     */
    int max_newton;            /* corrector iterations per point                */
    int warmup;                /* points predicted by the secant before the MLP */
    int pod_modes;             /* POD rank r = network outputs                  */
    int pod_every;             /* POD rebuild period (points)                   */
    int train_steps;           /* Adam steps after each accepted point          */
    float lr;                  /* Adam learning rate                            */
    double omega_lo, omega_hi; /* normalisation range of w_1                    */
    int chord;                 /* 1: corrector updates reuse the Jacobian of the
                                  point's first evaluation (chord Newton; later
                                  evaluations residual only); 0: full Newton  */
} fse_cont_opts;

typedef struct {
    int newton_iters;          /* corrector updates                             */
    int evals;                 /* shooting evaluations (residual or Jacobian)   */
    double res;                /* final ||R||_2                                 */
    double znorm;              /* ||Z(0)||_2                                    */
    double pred_err;           /* ||Z_pred - Z|| / ||Z|| of the predictor       */
    double ms;                 /* device time of the point                      */
    int status;                /* FSE_OK when accepted                          */
    int predictor;             /* predictor actually used                       */
    int fallback;              /* 1: accepted by the FP64 fallback context       */
} fse_cont_point;

/* Attach (fb non-NULL) or detach (fb NULL) an FP64 context of the same problem to an
 * FSE_MIXED_FP32 context.  A point that the mixed-precision corrector of fse_continue does not
 * accept (no contraction within max_newton updates, or a non-finite trajectory: FP32 tangents
 * can be too coarse for a nearly undamped structure, whose Floquet multipliers sit close to
 * the unit circle) is corrected again from the same prediction in fb with the same options,
 * and its torus is copied back; fse_cont_point.fallback records it.  The paper has no
 * counterpart (it uses one precision).  Both contexts must be unsharded, on the same device,
 * with equal n, d, S, H, rho and S1 (checked: n, d, U~, N, S1 and rho); the caller keeps fb
 * alive while attached and sets its linear solver.  Returns FSE_EINVAL on a mismatch. */
int fse_set_fallback(fse_ctx* ctx, fse_ctx* fb);

/* Run the sweep.  Z_start: host, 2 n U~ doubles (initial guess of point 0);
 * Z_out: host, n_points x 2 n U~ (nullable); info: n_points records (nullable).
 * mlp may be NULL for the secant predictor.  Returns the worst point status. */
int fse_continue(fse_ctx* ctx, fse_mlp* mlp, const fse_cont_opts* opts, const double* Z_start,
                 double* Z_out, fse_cont_point* info);

/* ------------------------------------------------------------------------
 * Pseudo-arclength continuation in (Z(0), w_1) (App. C, Eq. C1-C3), which
 * follows the branch through folds where stepping w_1 fails.  Point 0 is
 * Z_start corrected by Newton at fixed w_1 = omega_start.  The first tangent
 * solves [J dR/dw_1; 0 1] (t_Z, t_w) = (0, 1), oriented so that t_w has the
 * sign of `direction`; later tangents are the secant through the last two
 * points.  Distances use ||dZ||^2 + (sigma dw_1)^2, sigma = omega_scale (<= 0:
 * ||Z_0|| / omega_start).  The step grows by 1.5 (up to ds_max) after a
 * correction of at most 2 Newton updates, shrinks by 0.7 after one of 5 or more,
 * and is halved (down to ds / 64) and the point predicted again when the
 * correction fails.  Point j: predictor y_pred = y_{j-1} + ds t, then
 * Newton on R(Z, w_1) = 0 and t . (y - y_pred) = 0 with the bordered matrix
 * [J dR/dw_1; t_Z^T sigma^2 t_w] (Eq. 22, Eq. 23; dense LU on the GPU, so
 * 2 n U~ <= 16383), accepted when ||R||_2 <= rel_tol ||Z||_2.  Stops after
 * n_points, at the first point that does not converge (returns FSE_ENOCONV)
 * or once w_1 leaves [omega_min, omega_max] (omega_max <= 0: no upper bound).
 * Z_out: n_points x 2 n U~ doubles (host, nullable); omega_out: n_points
 * doubles (host, nullable); info: n_points records (pred_err unused);
 * n_done: points written.
 * ------------------------------------------------------------------------ */
typedef struct {
    int n_points;
    double omega_start;        /* w_1 of Z_start                                */
    double ds;                 /* first arclength step (> 0), metric above      */
    double ds_max;             /* largest step (<= ds: fixed steps)             */
    double omega_scale;        /* sigma; <= 0 for ||Z_0|| / omega_start          */
    int direction;             /* +1: start towards larger w_1, -1: smaller     */
    double rel_tol;            /* acceptance ||R|| <= rel_tol ||Z||             */
    int max_newton;            /* corrector iterations per point (>= 1)         */
    double omega_min, omega_max;
} fse_arc_opts;

/* Run the pseudo-arclength continuation described above. */
int fse_continue_arclength(fse_ctx* ctx, const fse_arc_opts* opts, const double* Z_start, double* Z_out,
                           double* omega_out, fse_cont_point* info, int* n_done);

#ifdef __cplusplus
}
#endif

#endif /* FSE_H */
