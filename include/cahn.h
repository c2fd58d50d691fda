/*
 * cahn.h -- C ABI of the GB300 (sm_103a) solver for the per-time-step linear
 * systems of the modified Cahn-Hilliard biofilm-flow model.
 *
 * Model and method: McClanahan, Stegmeier, Sundermann, Doom, Kimn,
 * "Parallel Simulations of Biofilm Flow using the Modified Cahn-Hilliard
 * Equation".  The step advances the phase field phi (Eq. 2.4, with
 * Crank-Nicolson + extrapolation, §4), then the velocity by the projection
 * method: predictor (Eq. 4.3), pressure Poisson (Eq. 4.4), correction
 * (Eq. 4.5).  Each step solves four sparse systems (§4.1, "a sequence of
 * linear algebraic systems"):
 *
 *   CAHN_SYS_PHI  A_phi = I/dt + 1/2 G_a (kappa L_h + S I), a = M phi*
 *                 (13-point, fourth order, non-symmetric; GMRES or BiCGStab)
 *   CAHN_SYS_U/V  H = rho/dt I + eta_bar/2 L_h on interior rows, Dirichlet
 *                 wall rows (SPD; CG)
 *   CAHN_SYS_P    L_h, zero-flux walls, singular (Listing 5 null space; CG)
 *
 * and, when the nutrient is on (Eq. 2.5-2.7), a fifth one:
 *
 *   CAHN_SYS_C    K = phi_s^{n+1}/dt + A/2 phi^{n+1/2} + 1/2 G_k, the
 *                 Crank-Nicolson matrix of the nutrient equation with the
 *                 diffusion coefficient k = D_s phi_s^{n+1/2}, phi_s = 1 - phi
 *                 (5-point, variable coefficient; zero flux on both walls,
 *                 or with CAHN_NUT_BC_BULK_TOP a Dirichlet top-wall row c =
 *                 c_bulk; SPD (on the fields with a zero Dirichlet row); CG)
 *
 * all matrix-free, preconditioned by a geometric multigrid V-cycle, by
 * Jacobi (the paper's choice, Listing 4), or by one-level domain
 * decomposition (the paper's planned preconditioner, §4.1, §6).  With momentum =
 * CAHN_MOM_IMPLICIT the two predictor systems become one coupled system:
 *
 *   CAHN_SYS_UV   rho/dt I - 1/2 div(2 eta(phi) D(.)) on [u; v], the whole
 *                 variable stress of Eq. 4.1 by Crank-Nicolson (9-point
 *                 blocks coupled through the cross derivatives; Dirichlet
 *                 wall rows; SPD on the fields that vanish on the walls;
 *                 CG, Jacobi-preconditioned)
 *
 * Grid (§4): nx periodic columns (x_i = i lx/nx), ny+1 rows (y_j = j ly/ny)
 * with the walls on rows 0 and ny.  Every field is a dense row-major FP64
 * array [ny+1][nx], x fastest, no padding.  Inner products and norms are
 * trapezoid-weighted: weight 1/2 on the wall rows, 1 elsewhere.
 *
 * Conventions for every entry point:
 *   - Return 0 (CAHN_OK) or a negative CAHN_ERR_* code; cahn_last_error()
 *     gives a message for the last failure on that context.
 *   - Work is ordered on the CUDA stream given to cahn_init.  cahn_step and
 *     cahn_solve synchronise that stream once, at the end of the call, to
 *     read back the status word and statistics.
 *   - Pointers named "device" must be device memory (e.g. torch CUDA
 *     tensors) of [ny+1][nx] doubles, 16-byte aligned; "host" pointers are
 *     host memory.  The caller keeps ownership of everything it passes.
 *   - The library owns all other memory (previous-step fields, operator
 *     coefficients, Krylov bases, the multigrid hierarchy, FP32 shadows,
 *     CUDA graphs) and releases it in cahn_free.
 */
#ifndef CAHN_H
#define CAHN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CAHN_ABI_VERSION 3

/* return codes */
#define CAHN_OK                 0
#define CAHN_ERR_ARG           -1  /* invalid argument / parameter */
#define CAHN_ERR_CUDA          -2  /* a CUDA runtime call failed */
#define CAHN_ERR_NOMEM         -3  /* device allocation failed */
#define CAHN_ERR_DOMAIN        -4  /* extrapolated phi left (0,1): log energy undefined */
#define CAHN_ERR_NAN           -5  /* NaN / Inf in a residual norm */
#define CAHN_ERR_NOT_CONVERGED -6  /* a Krylov solve hit max_iters */

/* systems */
#define CAHN_SYS_PHI 0
#define CAHN_SYS_U   1
#define CAHN_SYS_V   2
#define CAHN_SYS_P   3
#define CAHN_SYS_C   4   /* nutrient (instances with nutrient = 1) */
#define CAHN_NSYS    5
#define CAHN_SYS_UV  5   /* the coupled momentum system (momentum = CAHN_MOM_IMPLICIT):
                            vectors stacked [2][ny+1][nx] (u rows, then v rows); its
                            statistics are reported in the CAHN_SYS_U slot */

/* options */
#define CAHN_FLOW_POISEUILLE 0   /* no-slip walls, constant body force 8 eta_w u_max / ly^2 */
#define CAHN_FLOW_SHEAR      1   /* u = u_max on the top wall (§5.1, Eq. 5.2) */
#define CAHN_FP64            0
#define CAHN_MIXED           1   /* FP32 inner solves, FP64 iterative refinement */
#define CAHN_GMRES           0
#define CAHN_BICGSTAB        1
#define CAHN_ENERGY_FLORY_HUGGINS 0
#define CAHN_ENERGY_DOUBLE_WELL   1   /* gamma2 phi^2 (1-phi)^2, Eq. 2.3 / 3.3 */
#define CAHN_PC_MG           0   /* geometric multigrid V-cycle */
#define CAHN_PC_JACOBI       1   /* point Jacobi (Listing 4) */
#define CAHN_PC_SCHWARZ      2   /* one-level domain decomposition (§4.1, §6): subdomains of
                                    32 x 16 nodes solved locally by 12 Chebyshev steps in shared
                                    memory; restricted additive Schwarz with overlap 2 for
                                    CAHN_SYS_PHI, non-overlapping block Jacobi (symmetric) for
                                    the CG systems; nx >= 48, ny >= 24 */
#define CAHN_NUT_BC_ZERO_FLUX 0  /* nutrient: zero total flux on both walls (§2 boundary block) */
#define CAHN_NUT_BC_BULK_TOP  1  /* nutrient: c = c_bulk on the top wall, zero flux below */
#define CAHN_MOM_SPLIT       0   /* eta_bar = max(eta) implicit, the rest of the stress explicit (Eq. 4.2) */
#define CAHN_MOM_IMPLICIT    1   /* the whole stress div(2 eta D(v)) implicit, u and v coupled */

/* One instance's grid, dimensionless parameters (§3, Eq. 3.2 / Table 1
 * style) and solver options.  Doubles are dimensionless. */
typedef struct cahn_params {
    int32_t nx, ny;          /* nx periodic columns (even, >= 4); ny intervals (even, >= 4) */
    double  lx, ly;          /* domain [0,lx) x [0,ly] */
    double  eps;             /* interface width, kappa = eps^2 */
    double  mobility;        /* M: degenerate mobility a = M phi (Eq. 2.4) */
    double  chi, n_poly;     /* Flory-Huggins chi and N */
    double  stab_s;          /* stabilisation S >= 0 (0 = plain extrapolation) */
    double  eta_water, eta_biofilm;   /* viscosities, eta(phi) = phi eta_b + (1-phi) eta_w */
    double  rho_water, rho_biofilm;   /* densities; must be equal (Table 1) */
    double  gamma_cap;       /* capillary coefficient of -Gamma div(grad phi grad phi) */
    int32_t flow_mode;       /* CAHN_FLOW_* */
    double  u_max;           /* Poiseuille peak, or top-wall speed (SHEAR) */
    double  dt;
    int32_t precision;       /* CAHN_FP64 | CAHN_MIXED */
    int32_t krylov;          /* CAHN_GMRES | CAHN_BICGSTAB for CAHN_SYS_PHI */
    int32_t restart;         /* GMRES restart length m (1..64) */
    int32_t mg_levels;       /* multigrid levels incl. the fine grid (1..16) */
    int32_t max_iters;       /* Krylov iteration cap per solve */
    double  rtol;            /* ||b - A x||_W <= rtol ||b||_W */
    int32_t energy;          /* CAHN_ENERGY_* */
    double  gamma2;          /* double-well strength */
    int32_t precond;         /* CAHN_PC_* */
    int32_t use_graph;       /* 1: replay each step as a CUDA graph with
                                device-side convergence loops; 0: host loop */
    /* Nutrient transport and network production (Eq. 2.5-2.7).  With
     * nutrient = 1 each step adds g_n = growth_eps growth_mu phi c /
     * (growth_kc + c) to the phase-field equation (extrapolated phi*, c*,
     * c* clamped at 0; the conserved mass then grows by dt <g_n, 1>_W per
     * step) and, after the phase field, solves CAHN_SYS_C for c^{n+1}:
     *   (phi_s^{n+1} c^{n+1} - phi_s^n c^n)/dt + D_c(c* phi_s* v*)
     *     + A/2 phi^{n+1/2} (c^{n+1} + c^n) + 1/2 G_k (c^{n+1} + c^n) = 0
     * with zero total nutrient flux on both walls (nutrient_bc =
     * CAHN_NUT_BC_ZERO_FLUX), or c = c_bulk on row ny instead of its
     * equation (CAHN_NUT_BC_BULK_TOP).  The caller's c array is registered
     * with cahn_attach_nutrient. */
    int32_t nutrient;        /* 0 off, 1 on */
    double  diff_s;          /* D_s >= 0 */
    double  growth_mu;       /* mu >= 0, maximum production rate */
    double  growth_kc;       /* K_c > 0, half-saturation constant */
    double  growth_eps;      /* epsilon >= 0, scaling constant of g_n */
    double  consume_a;       /* A >= 0, consumption g_c = A phi c */
    double  c_bulk;          /* c on the top wall (CAHN_NUT_BC_BULK_TOP) */
    int32_t nutrient_bc;     /* CAHN_NUT_BC_* */
    /* Velocity predictor (Eq. 4.1-4.3).  CAHN_MOM_SPLIT: Crank-Nicolson on
     * eta_bar Lap v, eta_bar = max(eta_water, eta_biofilm), the rest of the
     * viscous stress explicit; two Dirichlet Helmholtz solves (SYS_U, SYS_V).
     * CAHN_MOM_IMPLICIT: Crank-Nicolson on div(2 eta(phi^{n+1/2}) D(v)), one
     * coupled solve (CAHN_SYS_UV) per step. */
    int32_t momentum;
} cahn_params;

/* Per-instance statistics of one cahn_step / cahn_solve call. */
typedef struct cahn_stats {
    int64_t steps;           /* time steps completed by the call */
    int32_t iters[CAHN_NSYS];   /* Krylov iterations, summed over the call, per system */
    int32_t outer[CAHN_NSYS];   /* refinement sweeps (CAHN_MIXED), summed, per system */
    double  resid[CAHN_NSYS];   /* last relative residual estimate per system */
    double  mass_drift;      /* last step: (<phi,1>_W before correction - target) / target,
                                target = m0 (grown by dt <g_n, 1>_W with the nutrient on) */
    int32_t failed_system;   /* -1, or the CAHN_SYS_* that failed */
    int32_t status;          /* the call's return code */
} cahn_stats;

typedef struct cahn_ctx cahn_ctx;   /* opaque, library-owned */

/* Create a context for `batch` independent instances (1 <= batch <= 1024).
 * params[k], phi[k], u[k], v[k], p[k]: instance k's parameters and its
 * device state arrays [ny+1][nx] FP64 (phi in (0,1); u, v on the walls are
 * taken from the flow mode).  The arrays stay owned by the caller and are
 * advanced in place by cahn_step.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream).  The previous-step fields start equal to the
 * current ones (q^{-1} = q^0) and m0 = <phi,1>_W.  On failure *ctx = NULL. */
int cahn_init(cahn_ctx** ctx, int32_t batch, const cahn_params* params,
              double* const* phi, double* const* u, double* const* v,
              double* const* p, void* stream);

/* Advance every instance by `nsteps` >= 0 time steps (§4: phi solve, mass
 * correction, [nutrient solve,] velocity predictor, pressure Poisson,
 * velocity correction).  An instance with nutrient = 1 must have its c
 * registered (cahn_attach_nutrient), else CAHN_ERR_ARG.
 * stats: NULL or an array of `batch` records.  On CAHN_ERR_NOT_CONVERGED,
 * _DOMAIN or _NAN the failing instance's arrays hold the state at the start
 * of the failing step's last completed stage; the others are advanced. */
int cahn_step(cahn_ctx* ctx, int32_t nsteps, cahn_stats* stats);

/* As cahn_step, with the state in HOST arrays: copies phi/u/v/p of every
 * instance to the device, steps, and copies them back, all on the stream.
 * phi_h[k] etc. are host arrays [ny+1][nx] (pinned memory for full speed).
 * A registered nutrient c stays in its device array. */
int cahn_step_host(cahn_ctx* ctx, int32_t nsteps, double* const* phi_h,
                   double* const* u_h, double* const* v_h, double* const* p_h,
                   cahn_stats* stats);

/* One linear solve of `system` for instance `instance`, with the
 * coefficients the next step would use (a = M phi* from the current and
 * previous phi).  rhs: device [ny+1][nx] (read only).  x: device
 * [ny+1][nx], in: initial guess, out: solution.  For CAHN_SYS_P the rhs is
 * projected (rhs - <rhs,1>_W/<1,1>_W) and x returned with <x,1>_W = 0; for
 * CAHN_SYS_U/V the wall rows of x come out as rhs * dt / rho.  CAHN_SYS_C
 * (nutrient instances only) is K with phi^{n+1} = phi^n = the current phi;
 * with CAHN_NUT_BC_BULK_TOP the top row of x comes out as rhs * dt.
 * CAHN_SYS_UV (CAHN_MOM_IMPLICIT instances only): rhs and x are stacked
 * device arrays [2][ny+1][nx] (u, then v), eta at the current phi; the
 * wall rows of x come out as rhs * dt / rho; the coupled solve stops at
 * rtol / 100 (one norm covers both components, u the larger). */
int cahn_solve(cahn_ctx* ctx, int32_t instance, int32_t system,
               const double* rhs, double* x, cahn_stats* stats);

/* y = A x for `system` of instance `instance` (the matrix-free operator of
 * that system; CAHN_SYS_PHI with the coefficient a = M phi* of the state
 * as of the last cahn_init / cahn_step / cahn_solve call; CAHN_SYS_C and
 * CAHN_SYS_UV as in cahn_solve, x and y stacked for CAHN_SYS_UV).  x, y:
 * device [ny+1][nx], not aliased.  Asynchronous on the context's stream (no
 * synchronisation). */
int cahn_apply(cahn_ctx* ctx, int32_t instance, int32_t system, const double* x, double* y);

/* As cahn_apply, with the FP32 operator that the inner solves of a
 * CAHN_MIXED instance use (FP32 arithmetic, FP32 coefficient shadow).
 * x, y: device [ny+1][nx] FP32.  CAHN_ERR_ARG for an FP64 instance. */
int cahn_apply32(cahn_ctx* ctx, int32_t instance, int32_t system, const float* x, float* y);

/* One step of the FP32 smoother of a system's multigrid V-cycle on its fine
 * grid, for a CAHN_MIXED instance preconditioned by the V-cycle
 * (CAHN_PC_MG).  The V-cycle is this library's preconditioner of the
 * Krylov solves that replace the paper's GMRES + Jacobi (§4.1, Listing 4);
 * its smoother is Chebyshev-Jacobi on [lam/4, lam], lam the Gershgorin
 * bound of D^-1 A, and step k of it computes
 *   d = c1(k) d + c2(k) D^-1 (b - A x),   y = x + d,
 * with the same kernel, coefficients and D as a V-cycle's step k (d is not
 * read for k = 0; rows held at zero on the level's corrections -- the
 * predictor's wall rows -- give y = 0 there and leave d alone).  The
 * coefficient fields are those of the current state, as for cahn_apply32.
 *   k: 0 <= k < 16.
 *   x, b: device [ny+1][nx] FP32, read only; d: device FP32, read (k > 0)
 *   and written; y: device FP32, written.  y and d must not alias each
 *   other, x or b.
 * Stream-ordered on the context's stream, no synchronisation.  Errors:
 * CAHN_ERR_ARG (bad instance, system or k, NULL or aliased vectors, an FP64
 * instance, Jacobi preconditioning, CAHN_SYS_C without the nutrient),
 * CAHN_ERR_CUDA. */
int cahn_smooth32(cahn_ctx* ctx, int32_t instance, int32_t system, int32_t k, const float* x,
                  const float* b, float* d, float* y);

/* The first pass of the FP32 V-cycle of a 5-point system (CAHN_SYS_U,
 * CAHN_SYS_V, CAHN_SYS_P) on its fine grid, as the V-cycle runs it: the
 * pre-smoothing steps k = 0 .. deg-1 from x = 0 (the steps of
 * cahn_smooth32; deg = 3), then the residual b - A x restricted to the next
 * level's right-hand side, which stays in the hierarchy (the coarse-grid
 * correction of the multigrid preconditioner of §4.1's Krylov solves).
 * One launch when the hierarchy runs temporally blocked passes (the
 * default); separate launches with CAHN_MG_FUSED=0 in the environment at
 * cahn_init.  x is bit for bit the result of cahn_smooth32 for k = 0, 1, 2
 * from x = 0.
 *   b: device [ny+1][nx] FP32, read only; x: device FP32, written; x must
 *   not alias b.
 * Stream-ordered on the context's stream, no synchronisation.  Errors:
 * CAHN_ERR_ARG (bad instance or system, NULL or aliased vectors, an FP64
 * instance, a preconditioner other than CAHN_PC_MG, a one-level hierarchy),
 * CAHN_ERR_CUDA. */
int cahn_mg_down32(cahn_ctx* ctx, int32_t instance, int32_t system, const float* b, float* x);

/* The exact coarsest-level solve of the multigrid preconditioner of §4.1's
 * Krylov solves, for a 5-point level operator with constant coefficients on
 * an nx-periodic grid of ny+1 rows,
 *   (A x)_ij = c0 x_ij + cx (2 x_ij - x_i-1,j - x_i+1,j) + cy (2 x_ij - x_i,j-1 - x_i,j+1):
 * the dense matrix P that the V-cycle applies, x = P b.
 *   walls = 0: zero flux, the row beyond a wall reflected (row 1 for row 0).
 *     With c0 = 0 the operator is singular (the constants); A is then
 *     self-adjoint in the inner product weighted 1/2 on the wall rows and 1
 *     inside, and P is its pseudo-inverse there: P maps the constants to
 *     zero, and A P b = b with a zero weighted sum of P b for every b whose
 *     weighted sum is zero.  With c0 > 0, P = A^-1.
 *   walls = 1: the wall rows are held at zero (Dirichlet corrections): their
 *     rows and columns of P are zero, and P inverts A on the interior rows.
 * Host only: formed in FP64 by Gauss-Jordan elimination with partial
 * pivoting, no device work, callable without a GPU.  The V-cycle rounds P
 * to the solve's precision.
 *   P: host [n][n] FP64 with n = nx (ny + 1), row-major, written.
 * Errors (cahn_last_error(NULL) describes them): CAHN_ERR_ARG (nx < 2,
 * ny < 1, n > 4096, walls not 0 or 1, c0, cx or cy negative or not finite,
 * cx + cy = 0, NULL P, or a singular system other than walls = 0 with
 * c0 = 0). */
int cahn_lap5_coarse_inverse(int32_t nx, int32_t ny, int32_t walls, double c0, double cx,
                             double cy, double* P);

/* Discrete adjoint (vector-Jacobian product) of nsteps time steps (§4) of
 * instance `instance`, FP64 throughout its own transposed solves.
 * The forward map is the one cahn_step computes from a freshly initialised
 * state: phi^{-1} = phi^0 = phi0 (likewise u, v), p0 the first pressure, and
 * the conserved mass m0 = <phi0, 1>_W, with the instance's parameters.
 * Instances with the nutrient on, or with momentum = CAHN_MOM_IMPLICIT,
 * are rejected (CAHN_ERR_ARG): the adjoint
 * covers the phase field and the flow.
 * Given phiN_bar = dJ/dphi^N it returns
 *   phi0_bar  = dJ/dphi0 (device [ny+1][nx] FP64, written),
 *   theta_bar = {dJ/dchi, dJ/dM} (host double[2], written),
 * the exact derivatives of the discrete step (every explicit operation
 * reversed; A_phi, the predictor H and the projected pressure Poisson map
 * reversed by transposed solves to the instance's rtol), up to that
 * tolerance.  The pressure guess p0 has no influence on the result.
 *   phi0, u0, v0, p0, phiN_bar: device [ny+1][nx] FP64, read only.
 *   checkpoint: steps between stored states (>= 1; clamped to nsteps).
 *     Memory: 7 fields per checkpoint plus 3 (checkpoint + 2) fields of
 *     recomputed levels plus about 30 work fields, allocated for the call
 *     and released before it returns.  Each segment is recomputed once.
 *   stats: NULL or one record: iters/resid of the transposed solves
 *     (CAHN_SYS_PHI: A_phi^T, U/V: H, P: pressure), steps = nsteps.
 * The instance's own fields, history and captured graphs are unchanged on
 * return; the caller's phi/u/v/p buffers are not touched.  Synchronises
 * the context's stream.  Errors: CAHN_ERR_ARG, _NOMEM, _CUDA; a forward or
 * transposed solve that fails returns its code (_DOMAIN, _NAN,
 * _NOT_CONVERGED) with stats.failed_system set. */
int cahn_vjp(cahn_ctx* ctx, int32_t instance, const double* phi0, const double* u0,
             const double* v0, const double* p0, int32_t nsteps, int32_t checkpoint,
             const double* phiN_bar, double* phi0_bar, double* theta_bar, cahn_stats* stats);

/* Pressure solve that allocates no device memory (the paper has no
 * counterpart: this serves callers that cannot allocate when they need a
 * solve -- a host whose memory manager already holds the GPU's memory for
 * its own pool, a latency-critical loop where cudaMalloc / cudaFree would
 * stall on device synchronisation, a plugin limited to memory set aside
 * at load time).  It solves the CAHN_SYS_P system of cahn_solve -- L_h x =
 * rhs - <rhs,1>_W/<1,1>_W, returned with <x,1>_W = 0 -- by
 * Jacobi-preconditioned CG to ||r||_W <= rtol ||rhs||_W, with no context.
 *   rhs: device [ny+1][nx] FP64, read only.  x: device [ny+1][nx], in:
 *   initial guess, out: solution.  stream: cudaStream_t.  stats: NULL or
 *   one record (iters / resid / status of CAHN_SYS_P).
 * All intermediates live in one fixed 3.3 MB device array that every GPU
 * loading the library holds until exit; grids with nx*(ny+1) > 66,560
 * nodes (256 x 256 intervals fit) are rejected with CAHN_ERR_ARG.  The
 * first call on a device looks up the array's address and clears its
 * reduction counter (synchronising the device once), so make that first call before any
 * stream capture.  Calls share the array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Synchronises `stream` before returning.  Errors: CAHN_ERR_ARG,
 * _CUDA, _NAN, _NOT_CONVERGED; message from cahn_noalloc_last_error(). */
int cahn_solve_p_noalloc(int32_t nx, int32_t ny, double lx, double ly, double rtol,
                         int32_t max_iters, const double* rhs, double* x, void* stream,
                         cahn_stats* stats);

/* Message of the last cahn_solve_p_noalloc failure on this host thread. */
const char* cahn_noalloc_last_error(void);

/* Checkpoint / resume.  A step reads the previous levels phi^{n-1},
 * u^{n-1}, v^{n-1} (extrapolation, §4) and the conserved mass m0 besides
 * the caller's phi, u, v, p, so an exact restart needs them too.
 * cahn_get_history copies instance `instance`'s previous levels into the
 * caller's device arrays ([ny+1][nx] FP64) and its m0 into *m0;
 * cahn_set_history installs them (for a context created from the matching
 * phi, u, v, p).  Stepping after a set continues the saved run bit for bit.
 * With the nutrient on, m0 is the current mass target (m0 grown by the
 * production so far) and the nutrient's previous level travels through
 * cahn_get_nutrient_history / cahn_attach_nutrient.
 * cahn_set_history drops the context's captured step graphs (they are
 * captured again at the next step).
 * Both synchronise the context's stream.  Errors: CAHN_ERR_ARG, _CUDA. */
int cahn_get_history(cahn_ctx* ctx, int32_t instance, double* phi_prev, double* u_prev,
                     double* v_prev, double* m0);
int cahn_set_history(cahn_ctx* ctx, int32_t instance, const double* phi_prev,
                     const double* u_prev, const double* v_prev, double m0);

/* Register the caller's nutrient array of instance `instance` (created
 * with nutrient = 1): c is device [ny+1][nx] FP64, owned by the caller and
 * advanced in place by cahn_step like phi.  c_prev: device [ny+1][nx], the
 * previous level c^{n-1} for the extrapolation (NULL: c^{-1} = c, a fresh
 * start).  Both are copied at the call; c is read again at every
 * cahn_step.  Any captured graph of the context is dropped.  Synchronises
 * the context's stream.  Errors: CAHN_ERR_ARG (bad instance, NULL c, or an
 * instance without the nutrient), _CUDA. */
int cahn_attach_nutrient(cahn_ctx* ctx, int32_t instance, double* c, const double* c_prev);

/* Copy the nutrient's previous level c^{n-1} of instance `instance` into
 * the caller's device array [ny+1][nx] (for an exact restart).
 * Synchronises the context's stream.  Errors: CAHN_ERR_ARG (no nutrient
 * registered), _CUDA. */
int cahn_get_nutrient_history(cahn_ctx* ctx, int32_t instance, double* c_prev);

/* Tile height (output rows per 32-column thread block: 8, 16 or 32) that
 * the autotuner picked at cahn_init for the operator of `system` on
 * multigrid level `level` (0 = the fine grid) of `instance`: the precision
 * the system's inner solves run in (FP32 for CAHN_MIXED), the fine-grid
 * operator only (level 0) under CAHN_PC_JACOBI.  The tuner times each
 * candidate on the grid and keeps the fastest; every candidate computes the
 * same values.  Setting CAHN_TILE=8|16|32 in the environment before
 * cahn_init forces one height.  CAHN_SYS_C reports the levels of the
 * nutrient hierarchy (level 0 only under CAHN_PC_JACOBI), -1 for an
 * instance without the nutrient.  Returns -1 for a bad argument or a level
 * the hierarchy does not have. */
int cahn_tile_height(const cahn_ctx* ctx, int32_t instance, int32_t system, int32_t level);

/* Release everything the context owns; NULL is a no-op. */
int cahn_free(cahn_ctx* ctx);

/* Message of the last error on ctx (ctx may be NULL: last cahn_init error).
 * The string is owned by the library and valid until the next call. */
const char* cahn_last_error(const cahn_ctx* ctx);

/* CAHN_ABI_VERSION of the loaded library. */
int cahn_abi_version(void);

/* Kernel launches issued by the last cahn_step / cahn_solve / cahn_apply
 * call on ctx (counted on the host as they are queued). */
int64_t cahn_last_launch_count(const cahn_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* CAHN_H */
