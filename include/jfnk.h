/*
 * jfnk.h -- C ABI of a GB300 (sm_103a) implementation of the time-implicit
 * Jacobian-free Newton-Krylov solver with physics-based preconditioning of
 * Viallet et al., "A Jacobian-free Newton-Krylov method for time-implicit
 * multidimensional hydrodynamics" (A&A), for the inviscid compressible
 * equations with gravity and thermal conduction on a Cartesian grid.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.  Every array argument is a DEVICE pointer owned by the caller,
 * except where a function says "host".  The library allocates no device
 * memory: the caller queries jfnk_workspace_bytes() and hands a device buffer
 * of at least that size (256-byte aligned) to jfnk_bind(), together with the
 * CUDA stream on which all work is queued.  The handle keeps a small pinned
 * host buffer for the convergence scalars that the host reads.
 *
 * Packed vector layout (length jfnk_vector_length() = (2 + ndim) * ncell,
 * ncell = n[0] * n[1] * n[2]):  [rho | e or eps_t | u_x | u_y | (u_z)],
 * every block a C-ordered (n[2], n[1], n[0]) array with x fastest.  rho and
 * e / eps_t are cell-centred; u_d holds the velocity on the LOWER face of each
 * cell in direction d.  In a direction with reflecting walls the slot with
 * index 0 along d is the wall face: it is read as zero and written as zero;
 * the upper wall face has no slot.  Gas constant R = 1, so T = p / rho.
 *
 * Precision.  With jfnk_options.precision == JFNK_FP64 every vector is double.
 * With JFNK_MIXED the Krylov vectors passed as `void*` (Jv in/out,
 * preconditioner in/out) are float, and the Krylov basis and the
 * preconditioner solve are stored and run in float with double-accumulated
 * dot products; X, X^n, F and the Newton update stay double.
 *
 * Errors.  Negative status = error, nothing useful written, message in
 * jfnk_last_error().  Positive status = completed without meeting the
 * requested tolerance (outputs valid, see jfnk_stats).  Calls are queued
 * asynchronously on the bound stream except those that read scalars back to
 * the host and therefore return only after the stream has reached them:
 * jfnk_step, jfnk_linear_solve, jfnk_vjp and jfnk_dt_from_cfl always;
 * jfnk_jv when its host out-pointer delta_used is non-NULL; jfnk_scaling when
 * its host out-pointer xhat_norm is non-NULL.  A handle is not thread-safe.
 */
#ifndef JFNK_H
#define JFNK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JFNK_OK = 0,
    JFNK_EINVAL = -1,          /* bad argument or unsupported configuration   */
    JFNK_ECUDA = -2,           /* a CUDA call failed                          */
    JFNK_ENOMEM = -3,          /* workspace missing or too small              */
    JFNK_ENONFINITE = -4,      /* NaN / Inf met in a norm                     */
    JFNK_ENOCONV_GMRES = 1,    /* a linear solve stopped at gmres_max_it       */
    JFNK_ENOCONV_NEWTON = 2    /* the step stopped at newton_max               */
} jfnk_status;

enum { JFNK_BC_PERIODIC = 0, JFNK_BC_WALL = 1 };
enum { JFNK_ENERGY_INTERNAL = 0, JFNK_ENERGY_TOTAL = 1 };
enum { JFNK_PRECOND_NONE = 0, JFNK_PRECOND_SOUND = 1, JFNK_PRECOND_SOUND_DIFF = 2 };
enum { JFNK_PERT_OLD = 0, JFNK_PERT_NEW = 1 };
enum { JFNK_FP64 = 0, JFNK_MIXED = 1 };

/* Cartesian grid: ndim in {2, 3}; n[2] = 1 when ndim == 2; at least 4 cells
 * in every active direction; bc[d] per direction.  Preconditioned solves need
 * every n[d] to be a power of two (multigrid coarsening). */
typedef struct { int ndim; int n[3]; double lo[3], hi[3]; int bc[3]; } jfnk_grid;

/* Ideal gas: p = (gamma-1) rho e; energy_form selects e (Sect. 2, Eq. cons2)
 * or eps_t = e + |u|^2/2 (Eq. Etot) as the energy unknown. */
typedef struct { double gamma; int energy_form; } jfnk_eos;

/* Constant gravitational acceleration (Eq. cons3). */
typedef struct { double g[3]; } jfnk_gravity;

/* Conductivity chi = K0 * T^exponent (Eq. chirad with a power law); K0 = 0
 * switches conduction off. */
typedef struct { double K0; double exponent; } jfnk_conductivity;

/* Solver parameters, with the paper's values as defaults (Sects. 3.4, 4.1,
 * 4.2, 5.1.1): theta = 1/2 (Crank-Nicolson, Eq. crank_nicholson; 1 gives
 * backward Euler), lambda = 1e-7 (Eq. pert_old), alpha1 = 1e-5, alpha2 = 1
 * (Eq. jacobian_system_norm), eta = 1e-4 (Eq. forcing_term).  gmres_m is the
 * restart length, gmres_max_it the total iteration cap per linear solve,
 * newton_min = 2 forces the second iteration of Sect. 4.1.  mg_cycles V-cycles
 * (default 2) with mg_nu1 / mg_nu2 (default 2 / 2) red-black Gauss-Seidel
 * sweeps solve the semi-implicit system.  reorth = 1 adds a second classical
 * Gram-Schmidt pass to every GMRES iteration; reorth = 2 adds it only when
 * the first pass shrank the new Krylov vector below 1/sqrt(2) of its norm
 * (Daniel, Gragg, Kaufman and Stewart 1976; one extra host read per
 * iteration).
 * fixed_iterations = 1 runs exactly gmres_max_it iterations per linear solve
 * and newton_max Newton iterations (reproducible iteration counts).
 * pc_freeze = 1 takes the semi-implicit coefficients and transforms of the
 * preconditioner from X^n, the time level at which Sects. 3.3-3.4 write them,
 * for every Newton iteration of a step (only the scaling L, R follows the
 * iterate); 0 (default) rebuilds them at every Newton iterate.
 * Inner tolerance (the eta' of Sect. 3.5): inner_tol = 0 (default) runs the
 * fixed mg_cycles; inner_tol > 0 repeats V-cycles until the relative residual
 * ||b - A x|| / ||b|| of the finest-level SI system is at most inner_tol, or
 * inner_max_cycles cycles have run (the host reads the residual after every
 * cycle).  GMRES keeps the preconditioned directions, so a cycle count that
 * varies between applies leaves it valid (flexible GMRES).  inner_monitor =
 * 1 measures that relative residual after every apply inside GMRES and
 * reports it in the step statistics, at two extra reductions per apply. */
typedef struct {
    double theta, lambda, alpha1, alpha2, eta, newton_tol;
    int pert, gmres_m, gmres_max_it, newton_min, newton_max;
    int precond, mg_cycles, mg_nu1, mg_nu2, precision, reorth, fixed_iterations;
    int pc_freeze;
    double inner_tol;
    int inner_max_cycles, inner_monitor;
} jfnk_options;

#define JFNK_MAX_NEWTON 64

/* Per-step counters (the iteration statistics reported in Table 1). */
typedef struct {
    int newton_iterations;
    int gmres_iterations_total;
    int gmres_iterations[JFNK_MAX_NEWTON];
    double dx_inf[JFNK_MAX_NEWTON];         /* ||R^-1 dX||_inf per Newton iteration */
    double fhat_norm[JFNK_MAX_NEWTON];      /* ||L^-1 F||_2 at each iterate          */
    double gmres_res[JFNK_MAX_NEWTON];      /* final GMRES residual estimate / ||F^|| */
    int gmres_converged[JFNK_MAX_NEWTON];
    int converged;                          /* Newton tolerance met                  */
    int jv_evaluations;                     /* residual evaluations inside GMRES     */
    int precond_applies;
    double jv_ms;                           /* device time in the Jv residual kernels */
    double precond_ms;                      /* device time in preconditioner applies  */
    double ortho_ms;                        /* device time in Gram-Schmidt kernels    */
    double step_ms;                         /* device time of the whole step         */
    /* with profiling on: device time of each kernel of the Jv evaluation inside
     * GMRES, in the order perturb, eos, face fluxes, momentum fluxes, assemble */
    double jv_kernel_ms[5];
    long long kernel_launches;              /* kernels launched during the call      */
    /* with inner_monitor or inner_tol: the relative residual ||b - A x||/||b||
     * of the finest-level SI system after each preconditioner apply inside
     * GMRES (the inner accuracy eta' reached), mean and maximum over the
     * applies, and the V-cycles run in all applies */
    double inner_res_mean;
    double inner_res_max;
    long long inner_cycles;
    long long reorth_passes;                /* second Gram-Schmidt passes run         */
} jfnk_stats;

typedef struct jfnk_handle jfnk_handle;

/* Fill *opt with the defaults listed above (precond = SOUND, FP64). */
void jfnk_default_options(jfnk_options* opt);

/* Create a solver for one grid and physics: the grid, the equation of
 * state, gravity and conductivity of Sect. 2.  `opt` may be NULL for the
 * defaults.  Host pointers; copied.  Returns JFNK_EINVAL for unsupported
 * sizes or parameters. */
jfnk_status jfnk_create(const jfnk_grid* grid, const jfnk_eos* eos, const jfnk_gravity* gravity,
                        const jfnk_conductivity* cond, const jfnk_options* opt, jfnk_handle** out);

/* Device workspace the handle needs (bytes). */
size_t jfnk_workspace_bytes(const jfnk_handle* h);

/* Bind a caller-owned device workspace (>= jfnk_workspace_bytes, 256-byte
 * aligned) and a cudaStream_t (NULL = legacy default stream). */
jfnk_status jfnk_bind(jfnk_handle* h, void* dev_workspace, size_t bytes, void* cuda_stream);

/* Length of the packed vectors. */
long long jfnk_vector_length(const jfnk_handle* h);

/* Replace the options (same precision and restart length as at creation). */
jfnk_status jfnk_set_options(jfnk_handle* h, const jfnk_options* opt);

/* F = F_U(X) of Eq. crank_nicholson with weight theta:
 *   F = (U(X) - U(X^n))/dt - theta R_U(X) - (1-theta) R_U(X^n).
 * X, Xn, F: double, packed (Sect. 2). */
jfnk_status jfnk_residual(jfnk_handle* h, const double* X, const double* Xn, double dt, double* F);

/* Diagonal scalings of Eq. jacobian_system_norm at X: L and R (double,
 * packed; wall slots 1; either may be NULL) and, in *xhat_norm (host, may be
 * NULL), ||R^-1 X||_2.  With xhat_norm non-NULL the call synchronises the
 * bound stream to read the norm back. */
jfnk_status jfnk_scaling(jfnk_handle* h, const double* X, double* L, double* R, double* xhat_norm);

/* Scaled Jacobian-free product of Sect. 4.2 (Eqs. jacobian_free, pert_old or
 * pert_new):  Jv = L^-1 [G(X + delta R v) - G(X)] / delta,  G = U/dt - theta
 * R_U, delta from the options' perturbation rule; *delta_used (host, may be
 * NULL) receives delta.  v, Jv: precision type (see above).  With delta_used
 * non-NULL the call synchronises the bound stream to read delta back. */
jfnk_status jfnk_jv(jfnk_handle* h, const double* X, double dt, const void* v, void* Jv, double* delta_used);

/* Physics-based preconditioner of Sect. 4.3 in scaled form:
 *   w = R^-1 dX/dV J~_V^-1 dV/dU L v,
 * J~_V the semi-implicit sound-wave system (Sect. 3.3) or sound-wave +
 * conduction system (Sect. 3.4) with coefficients from X, solved by the
 * fixed multigrid V-cycles of the options.  v, w: precision type. */
jfnk_status jfnk_precond_apply(jfnk_handle* h, const double* X, double dt, const void* v, void* w);

/* One step of the semi-implicit scheme used as a time integrator (Sect.
 * 3.6): F_U(X^n) = -R_U(X^n) is transformed to the primitive variables, the
 * SI system built at X^n is solved once (the multigrid of the options), the
 * correction is transformed back and added: X^{n+1} = X^n + dX, in place in
 * X.  First order in time and stable only for advective CFL numbers well
 * below one (Sect. 3.7); theta = 1 gives the paper's scheme (backward Euler
 * in the SI terms).  Needs precond 1 or 2 (JFNK_EINVAL otherwise).
 * Asynchronous on the bound stream; non-finite values are not checked. */
jfnk_status jfnk_si_step(jfnk_handle* h, double* X, double dt);

/* One Newton linear solve (Eq. jacobian_system_norm with right
 * preconditioning, Eqs. lin_sys_rp, lin_sys_rp2, stopping rule Eq.
 * forcing_term): given the iterate X and X^n, returns the scaled correction
 * dxhat = R^-1 dX (double).  stats (host, may be NULL) gets the counters of
 * this solve in entry 0. */
jfnk_status jfnk_linear_solve(jfnk_handle* h, const double* X, const double* Xn, double dt, double* dxhat,
                              jfnk_stats* stats);

/* One implicit step (Sect. 4.1): X holds X^n on entry and X^{n+1} on exit.
 * newton_tol bounds ||R^-1 dX||_inf (Eq. nr_terminate), krylov_tol is eta
 * (Eq. forcing_term); a value <= 0 keeps the option's value. */
jfnk_status jfnk_step(jfnk_handle* h, double* X, double dt, double newton_tol, double krylov_tol,
                      jfnk_stats* stats);

/* Vector-Jacobian product of the residual (the kernel of the step adjoint;
 * the paper has no adjoint): y = (dG/dX)^T w at X with G = U/dt - theta R_U,
 * i.e. the transpose of dF_U/dX of Eq. crank_nicholson.  Double vectors,
 * packed; wall slots of y are zero.  Needs an FP64 handle (JFNK_EINVAL on a
 * mixed one, whose workspace holds no adjoint scratch).  Hand-written
 * reverse of the residual kernels; atomic accumulation makes y reproducible
 * to round-off only. */
jfnk_status jfnk_vjp_residual(jfnk_handle* h, const double* X, double dt, const double* w, double* y);

/* Adjoint of one implicit step (needs an FP64 handle).  Given the step's
 * input Xn and converged output Xnp1 and the gradient gbar of a loss with
 * respect to Xnp1, solves J^T lam = gbar (J = dG/dX at Xnp1; scaled as in Eq.
 * jacobian_system_norm, GMRES with the options' eta and restart, right-
 * preconditioned by the transpose of the physics-based preconditioner with
 * transposed multigrid cycles) and returns gXn = (db^n/dXn)^T lam and, in
 * *gK0 (host, may be NULL), theta lam.dR/dK0(Xnp1) + (1-theta) lam.dR/dK0(Xn).
 * dt is held fixed.  JFNK_ENOCONV_GMRES if the transposed solve stopped at
 * gmres_max_it (outputs from the last iterate). */
jfnk_status jfnk_vjp(jfnk_handle* h, const double* Xn, const double* Xnp1, double dt, const double* gbar, double* gXn,
                     double* gK0, jfnk_stats* stats);

/* dt = cfl * min_d dx_d / max(|u_cell| + c_s) (Sect. 1, CFL_hydro), u_cell the
 * mean of the two face velocities per direction.  *dt is host. */
jfnk_status jfnk_dt_from_cfl(jfnk_handle* h, const double* X, double cfl, double* dt);

/* Device time per kernel group of the last jfnk_step, for roofline
 * accounting: enable with on = 1 (CUDA events on the bound stream). */
jfnk_status jfnk_set_profiling(jfnk_handle* h, int on);

/* Largest grid (cells) that jfnk_residual_noalloc accepts. */
#define JFNK_NOALLOC_MAX_CELLS 65536

/* The residual of jfnk_residual, for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is an interface variant.
 * Same arguments, layout and result as jfnk_residual, but the scratch it needs
 * (b^n, p, T and the flux fields) lives in a fixed array inside the library
 * (JFNK_NOALLOC_MAX_CELLS * 23 doubles, 12.1 MB, held on every GPU that loads
 * the library until the process exits) instead of the bound workspace, so
 * the handle needs no jfnk_bind and the call allocates nothing.  Grids above
 * JFNK_NOALLOC_MAX_CELLS cells return JFNK_EINVAL with a message.  The first
 * call made with a given device current looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU race, so
 * serialise them.  Queued on the handle's stream (the legacy default stream
 * if the handle was never bound).  The device current at the call must be the
 * one the handle was bound on (JFNK_EINVAL otherwise); an unbound handle runs
 * on the current device.  The cached address does not survive a
 * cudaDeviceReset of that device: do not call this after one. */
jfnk_status jfnk_residual_noalloc(jfnk_handle* h, const double* X, const double* Xn, double dt, double* F);

/* Message of the last error on this handle (never NULL). */
const char* jfnk_last_error(const jfnk_handle* h);

void jfnk_destroy(jfnk_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* JFNK_H */
