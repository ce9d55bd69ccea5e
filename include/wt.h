/*
 * wt.h - C ABI of the GB300 (sm_103a) hybrid-spectral wave-tank library.
 *
 * The library solves, on one GPU, the hot path of the sigma-transformed
 * incompressible Navier-Stokes free-surface model of Melander, Bitsch, Chen
 * and Engsig-Karup ("A High-Order Hybrid-Spectral Incompressible Navier-Stokes
 * Model For Nonlinear Water Waves"): the mixed-stage pressure Poisson problem
 * (Sec. 3.2-3.3, Eq. poissonp with boundary rows Eq. bcpd / bcpdneu),
 * discretised with a Fourier basis in x (and y) and Chebyshev-Gauss-Lobatto
 * nodes in sigma (Sec. 3.4-3.5), solved by GMRES preconditioned with one
 * geometric p-multigrid V-cycle (Sec. 4, Algorithm 1), inside the
 * low-storage explicit Runge-Kutta stage (Eq. LSERK) together with the
 * kinematic free-surface update (Eq. kinematicFS).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: WT_OK (0) or one of the WT_E* codes below; the text of the
 *    last error of the calling thread is available from wt_last_error().
 *  - Arrays are float64 and owned by the caller; the library copies what it
 *    needs and never keeps a caller pointer after the call returns.  Each
 *    array may live in host memory or in device memory of the tank's GPU;
 *    the library inspects every pointer (cudaPointerGetAttributes) and copies
 *    host data through its own device buffers on the tank's stream.
 *  - Field layout: [Nz+1][Ny][Nx] (x fastest), sigma index 0 = free surface
 *    (sigma = 1), index Nz = bottom (sigma = 0).  Surface / bathymetry
 *    layout: [Ny][Nx].  A 2D (vertical-plane) tank has Ny = 1.
 *  - Grid: x_j = j L / Nx, y_j = j L / Ny (periodic, domain [0,L) x [0,L)),
 *    sigma_m = (cos(m pi / Nz) + 1) / 2.
 *  - Nx is a power of two in [4, 4096]; Ny is 1 or a power of two in
 *    [4, 1024]; 2 <= Nz <= 32.
 *  - Every call is stream-ordered on the tank's stream and returns after the
 *    results are complete.  By default the tank owns a non-blocking stream
 *    and orders each call after the work already queued on the legacy
 *    default stream; wt_set_stream selects a caller's stream instead.
 *  - The per-iteration kernels of the Krylov solver are captured as CUDA
 *    graphs at first use and replayed (not while kernel timing is on).
 *  - A tank handle must not be used by two threads at the same time.
 */
#ifndef WT_H
#define WT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum wt_status {
  WT_OK = 0,
  WT_EINVAL = 1,    /* invalid argument (sizes, pointers, options)            */
  WT_ENOMEM = 2,    /* device or host allocation failed                       */
  WT_ENOCONV = 3,   /* solve stopped at max_it above its tolerance;       
                       the best iterate is still written                      */
  WT_EBREAK = 4,    /* water depth d = h + eta <= 0 or a non-finite value:
                       the sigma map is invalid (e.g. a breaking wave)        */
  WT_ECUDA = 5,     /* a CUDA runtime call or kernel launch failed            */
  WT_ETIMEOUT = 6,  /* a bounded device-side wait gave up                     */
  WT_ENOTSUP = 7    /* valid request that the library does not support      */
};

enum wt_precision { WT_FP64 = 0, WT_MIXED = 1, WT_FP32 = 2, WT_REFINE = 3 };

typedef struct wt_tank wt_tank;

/* Solver and model options (wt_default_options fills the defaults shown). */
typedef struct wt_options {
  int mode;          /* WT_FP64: FP64 flexible GMRES + FP64 V-cycle.
                        WT_MIXED: FP64 flexible GMRES (FP64 residuals and
                        Krylov basis) whose preconditioner is the FP32
                        V-cycle, so every iteration refines the FP64 iterate
                        with an FP32 correction (default WT_MIXED).
                        WT_REFINE: FP64 iterative refinement - the FP64
                        residual r = b - A p, an FP32 flexible GMRES with
                        the FP32 V-cycle solving A e = r to inner_tol,
                        p += e, until tol (the FP64 operator runs once per
                        refinement step only)                               */
  double tol;        /* relative residual ||b - A p||_2 / ||b||_2 (1e-10)   */
  int restart;       /* GMRES restart length m (30)                          */
  int nu1, nu2;      /* pre- / post-smoothing sweeps (2, 2)                  */
  double omega;      /* block-Jacobi damping (0.4)                           */
  int max_it;        /* Krylov iterations per solve (200)                    */
  int filter;        /* exponential cut-off filter every stage (0)           */
  int linear;        /* linearised model, Sec. 5.3 (0)                       */
  int coarsest_max;  /* a level with at most this many unknowns is solved
                        directly by FP64 LU (64, at most 128)               */
  int bc_transfer;   /* 0: surface/bottom residual rows injected into the
                        coarse boundary rows (default); 1: whole column
                        through the Chebyshev truncation as printed          */
  int tail_max;      /* levels with at most this many unknowns run in one
                        V-cycle launch of one CTA (or of the cluster that
                        tail_cluster sets), smoothed by block-Jacobi; 0:
                        never, the default (the autotuners try it)          */
  double inner_tol;  /* WT_REFINE: relative residual of each FP32 inner
                        solve (1e-5)                                         */
  int max_ir;        /* WT_REFINE: refinement steps per solve (30)           */
  int vcycle_grid;   /* 1: the whole V-cycle of the finest-level
                        preconditioner as one cooperative launch with grid
                        barriers (bounded waits; WT_ETIMEOUT if one gives
                        up); 0: one launch per phase (default 0)            */
  int tail_cluster;  /* CTAs (2..16) of the thread-block cluster that runs
                        the levels at or below tail_max in one launch, the
                        phases separated by the cluster's hardware barrier;
                        0 or 1: one CTA (default 0)                          */
  long long barrier_cycles; /* vcycle_grid = 1: SM clock cycles a CTA waits
                        at a grid barrier before it gives up, sets the
                        abort word and the call returns WT_ETIMEOUT (the
                        barrier is then reset and the tank stays usable);
                        0: the default 2e9 (about one second)               */
  int cycle;         /* preconditioner of the Krylov solver: 0 = one V-cycle
                        (Algorithm 1, default); 1 = one full-multigrid cycle
                        (Algorithm 2: the right-hand side restricted to every
                        level, the coarsest solved, and on each finer level a
                        V-cycle from the prolongated coarse result)         */
  int smoother;      /* 0 = damped block-Jacobi over the columns (default);
                        1 = mean-depth spectral smoother: x += omega_s S
                        (f - A x), S the exact solve of the flat reference
                        problem (eta = 0, depth = min h) by horizontal
                        Fourier mode - the modes' (Nz+1)^2 inverses are
                        built once per bathymetry; 2 = a block-Jacobi sweep
                        followed by a spectral sweep.  With 1 or 2
                        vcycle_grid is not used, and the levels at or below
                        tail_max (if set) run the one-launch tail with
                        block-Jacobi sweeps, the finer levels spectral ones */
  double omega_s;    /* damping of the spectral smoother (1.0)               */
  int warp_fft;      /* 1 (default): x- and y-derivative and filter passes
                        over many lines (>= 512 x-rows, or y-lines of >= 16
                        columns; FP32 32..1024 points, FP64 with df64
                        32..256 points) run one warp per line pair with the
                        transform in registers; 0: every pass one CTA per
                        line (pair)                                          */
  int pdl;           /* 1 (default): kernels are launched with programmatic
                        dependent launch - the next kernel of the stream is
                        made resident while its predecessor runs and waits
                        (griddepcontrol.wait) for the predecessor's completion
                        before touching memory, so results are unchanged and
                        only launch latency is hidden; 0: plain stream order */
  int df64;          /* 1 (default): the FP64 spectral passes and sigma-column
                        kernels run in double-float arithmetic (each value
                        the unevaluated sum of two floats, about 48
                        significant bits, from error-free float
                        transformations) on the FP32 units, which GB300 runs
                        at 64 times its FP64 rate - the warp passes over many
                        lines (32..256 points), the column kernels over many
                        columns and the CTA-per-row passes - except that the
                        solver's true residuals (the restart residual of the
                        flexible GMRES, the refinement residual) keep the
                        CTA-per-row passes in FP64, so an FP64 solve reaches
                        FP64's attainable residual; the data stay FP64 in
                        memory (measured operator error 2e-15 .. 1e-14 of
                        max |Ap| against 1e-15 in FP64).  Double-float has
                        float's exponent range: fields whose values are all
                        below about 1e-30 or above 1e38 in magnitude need
                        df64 = 0.  2: double-float in
                        the true residuals too (attainable residual about
                        1e-11 on 1,024-point rows).  0: FP64 arithmetic      */
  int spectral_min;  /* smoother 1 or 2: levels with fewer unknowns than this
                        smooth by block-Jacobi alone (their column blocks
                        are built); 0 (default): every level spectral        */
} wt_options;

typedef struct wt_solve_info {
  int iterations;        /* Krylov iterations (= preconditioner applications) */
  double rel_residual;   /* final ||b - A p||_2 / ||b||_2, FP64 operator     */
  int status;            /* same code as the call's return value             */
  int refinements;       /* WT_REFINE: FP64 refinement steps (0 otherwise)   */
} wt_solve_info;

/* Fill *opt with the defaults listed above.  Never fails for opt != NULL. */
int wt_default_options(wt_options* opt);

/*
 * Create a tank on the current CUDA device.  Sec. 2 (geometry), Sec. 3.4
 * (grids), Sec. 4.1 (level hierarchy).  bathymetry: h(x, y) > 0, [Ny][Nx].
 * g: gravity (9.81 in the paper), nu >= 0: kinematic viscosity.  With nu > 0
 * the forcing carries nu Div_b Grad_b q for every velocity component
 * (Eq. sigmom1, forc1) with the vertical component of Grad_b q set to zero on
 * the surface nodes (a stress-free surface), and the bed is no-slip
 * (Sec. 5.4): after every stage the velocity and its stage registers are
 * zero on the bottom nodes.  The
 * adjoint calls and the batched tanks cover nu = 0 only (WT_ENOTSUP).  The
 * coarsest level must have at most 128 unknowns (WT_ENOTSUP otherwise): the
 * coarsening halves Ny only together with Nx, so 3D tanks need Ny = Nx in
 * practice (wt_levels_for shows the hierarchy without creating a tank).  On
 * success *out owns all device memory of the tank until wt_destroy.
 */
int wt_create(int Nx, int Ny, int Nz, double L, double g, double nu,
              const double* bathymetry, wt_tank** out);

/* Replace the options.  Rebuilds the level hierarchy when coarsest_max
 * changes.  WT_EINVAL for out-of-range values. */
int wt_set_options(wt_tank* t, const wt_options* opt);
int wt_get_options(const wt_tank* t, wt_options* opt);

/* Use the given cudaStream_t (passed as void*) for all later calls; NULL
 * returns to the tank's own stream.  The stream must not be the legacy
 * default stream (graph capture). */
int wt_set_stream(wt_tank* t, void* stream);

/* Grid coordinates: x [Nx], y [Ny], sigma [Nz+1] (any may be NULL). */
int wt_get_grid(const wt_tank* t, double* x, double* y, double* sigma);

/* Multigrid hierarchy: *nlevels and, if dims != NULL, dims[3*l+0..2] =
 * (Nx, Ny, Nz) of level l, finest first (capacity >= 3 * 16). */
int wt_get_levels(const wt_tank* t, int* nlevels, int* dims);

/* The hierarchy wt_create would build for an Nx x Ny x Nz grid with the
 * given coarsest_max (1..128), without a tank: host code only, no GPU or
 * CUDA call, so a caller can size a problem before creating it.  Coarsening
 * per Sec. 4.1 (Algorithm 1): halve Nx (and Ny) while Nx > Nz, halve Nz
 * (rounding up, at least 2) while Nz > Nx, both when equal; stop at a level
 * of at most coarsest_max unknowns or before Nx (Ny) < 4 or Nz < 2.  Output
 * as wt_get_levels (capacity >= 3 * 16).  WT_EINVAL for sizes wt_create
 * rejects; WT_ENOTSUP (levels still written) when the coarsest level has
 * more than 128 unknowns, as wt_create reports. */
int wt_levels_for(int Nx, int Ny, int Nz, int coarsest_max, int* nlevels, int* dims);

/* The sigma-direction matrices the library builds on the host for an
 * (Nz+1)-node CGL column and a coarser Nzc (2 <= Nzc <= Nz <= 32), without a
 * tank: host code only, no GPU or CUDA call.  Row-major host outputs (each
 * may be NULL): D [Nz+1][Nz+1] = d/dsigma (Sec. 3.5, 2 x the CGL matrix on
 * xi = 2 sigma - 1); F [Nz+1][Nz+1] = the Chebyshev exponential filter
 * (Sec. 3.6: modal transform, mode m damped by exp(-36 ((m - Nc) / (Nz + 1
 * - Nc))^2) above Nc = floor(0.9 Nz), evaluation); R [Nzc+1][Nz+1] = the
 * restriction's Chebyshev truncation (Sec. 4.2; bc_transfer 0: surface and
 * bottom rows injected, the library's default; 1: the whole column
 * truncated); P [Nz+1][Nzc+1] = the prolongation (the coarse interpolant at
 * the fine nodes).  Node m = 0 is the surface. */
int wt_sigma_matrices(int Nz, int Nzc, int bc_transfer, double* D, double* F, double* R, double* P);

/*
 * Model state: eta [Ny][Nx], u, v, w [Nz+1][Ny][Nx] (v ignored / returned as
 * zero when Ny = 1), time t.  wt_set_state also clears the 2N Runge-Kutta
 * registers K (Eq. LSERK, K^0 = 0) and the pressure warm start.
 */
int wt_set_state(wt_tank* t, const double* eta, const double* u, const double* v,
                 const double* w, double time);
int wt_get_state(const wt_tank* t, double* eta, double* u, double* v, double* w,
                 double* time);
/* Last pressure p_D [Nz+1][Ny][Nx] computed by wt_rk_stage / wt_step. */
int wt_get_pressure(const wt_tank* t, double* p);

/*
 * Ap = A_{a,b} p, the mixed-stage operator (Eq. poissonp: divergence with the
 * geometry of eta_a, gradient with that of eta_b; surface rows p, Eq. bcpd;
 * bottom rows n . Grad_b p with n = (h_x, h_y, 1), Eq. bcpdneu).
 * precision: WT_FP64 or WT_FP32 (inputs rounded to float, result widened).
 */
int wt_apply_operator(wt_tank* t, const double* eta_a, const double* eta_b,
                      const double* p, double* Ap, int precision);

/*
 * z = M^{-1} r: one p-multigrid V-cycle (Algorithm 1) from a zero initial
 * state - or one full-multigrid cycle (Algorithm 2) when the option cycle is
 * 1 - with damped block-Jacobi smoothing and spectral transfers
 * (Sec. 4.2-4.3).
 * precision: WT_FP64 or WT_FP32.  Test hook for the preconditioner.
 */
int wt_precondition(wt_tank* t, const double* eta_a, const double* eta_b,
                    const double* r, double* z, int precision);

/*
 * Solve A_{a,b} p = rhs to ||rhs - A p|| <= tol ||rhs|| (Sec. 4.4): rhs
 * carries the interior right-hand side and the surface (Dirichlet) and bottom
 * (Neumann) rows.  p is the initial guess on entry and the solution on exit.
 * tol <= 0 uses the option's tol.  info may be NULL.  WT_ENOCONV leaves the
 * best iterate in p.
 */
int wt_poisson_solve(wt_tank* t, const double* eta_a, const double* eta_b,
                     const double* rhs, double* p, double tol, wt_solve_info* info);

/*
 * One stage k = 1..5 of the five-stage fourth-order 2N-storage Runge-Kutta
 * scheme (Eq. LSERK, coefficients of Carpenter & Kennedy) with step dt:
 * free-surface update (Eq. kinematicFS), forcing (Eq. forc1), mixed-stage
 * Poisson solve and projection (Eq. rkforc1, poissonp).  Advances the time
 * by dt after stage 5.  WT_EBREAK when d <= 0 or a value is not finite.
 */
int wt_rk_stage(wt_tank* t, int k, double dt);

/* nsteps full steps of Eq. LSERK, five wt_rk_stage stages each. */
int wt_step(wt_tank* t, double dt, int nsteps);

/* Statistics of the last wt_rk_stage / wt_step: total Krylov iterations and
 * solves since the last wt_set_state. */
int wt_get_stats(const wt_tank* t, long* solves, long* iterations);

/*
 * Adjoint (reverse-mode derivative) of the 2D time step.  The paper has no
 * adjoint; these calls differentiate the discrete forward map of wt_step
 * (Sec. 3.1-3.3, Eq. kinematicFS, forc1, poissonp, bcpdneu, rkforc1, the
 * Sec. 3.6 filter when enabled) exactly, up to the solve tolerance.  2D
 * tanks only (WT_ENOTSUP for Ny > 1).  Arrays: host or device, FP64,
 * layouts as in wt_set_state.
 *
 * wt_set_bathymetry: replace h(x) ([Ny][Nx], > 0) of an existing tank (every
 *   level's truncated copy is rebuilt).
 * wt_apply_operator_transposed: out = A_{a,b}^T lam (test hook; precision
 *   WT_FP64 or WT_FP32).  A^T lam = e_surface lam_surface + Grad_b^T mu with
 *   mu = Div_a^T lam_interior plus the bottom-row terms; D_x^T = -D_x.
 * wt_adjoint_solve: A_{a,b}^T lam = rhs by the tank's solver (mode, tol,
 *   smoother, V-cycle) applied to A^T: transposed column blocks, transposed
 *   coarsest inverse, the same transfers.  lam: initial guess in, result out.
 * wt_adjoint_step: reverse one step.  (eta, u, w) is the state at the start
 *   of the step; the step is recomputed from it (the tank's state becomes
 *   the state after the step) with every stage's values kept, then the
 *   stages are reversed: on entry (lam_eta, lam_u, lam_w) hold dJ/d(state
 *   after the step), on return dJ/d(state at the start); dJ_dh (may be NULL)
 *   is incremented by this step's dJ/dh.  Every pressure solve of the
 *   recomputation and the transposed solves use the tank's options.
 *   WT_ENOCONV if any solve stopped above its tolerance (results written).
 */
int wt_set_bathymetry(wt_tank* t, const double* h);
int wt_apply_operator_transposed(wt_tank* t, const double* eta_a, const double* eta_b, const double* lam,
                                 double* out, int precision);
int wt_adjoint_solve(wt_tank* t, const double* eta_a, const double* eta_b, const double* rhs, double* lam,
                     double tol, wt_solve_info* info);
int wt_adjoint_step(wt_tank* t, double dt, const double* eta, const double* u, const double* w,
                    double* lam_eta, double* lam_u, double* lam_w, double* dJ_dh);

/*
 * Relaxation zone (Sec. 5.5: the wave generation and absorption zones of the
 * bar case, after Larsen & Dancy): for every column in the zone between x0
 * and x1 (either order; no wrap-around), with xi = (x - x0) / (x1 - x0) in
 * [0, 1], the state is blended towards the targets,
 *   q <- (1 - w) q + w q_target,  w = (exp(xi^3.5) - 1) / (e - 1),
 * so w = 0 at x0 (the zone's inner edge) and 1 at x1 (full target).  Apply
 * it between steps, with targets taken at the state's time (for instance
 * wt_stream_function_wave at that time for generation, zero for
 * absorption).  eta_target [Ny][Nx], u/v/w_target [Nz+1][Ny][Nx]: host or
 * device; a NULL target leaves that field alone (v_target is ignored in 2D).
 * Needs a state (WT_EINVAL otherwise).
 */
int wt_relax(wt_tank* t, double x0, double x1, const double* eta_target, const double* u_target,
             const double* v_target, const double* w_target);

/*
 * Steady nonlinear periodic wave by the Fourier stream-function method of
 * Rienecker & Fenton (1981), which the paper uses to initialise its
 * nonlinear accuracy study (Sec. 5.2) and its bar case (Sec. 5.5): nwaves
 * wavelengths in the periodic domain (k = 2 pi nwaves / L), height H over
 * the tank's flat bottom (h constant, else WT_EINVAL), nmodes Fourier modes
 * (2..128).  Solved on the host in FP64 (Newton's method on the surface
 * kinematic and Bernoulli conditions at nmodes + 1 points, zero mean level,
 * crest-to-trough height H, no mean Eulerian current; the height raised in
 * steps of 0.005 in steepness; the last solution is cached per tank) and
 * evaluated at the tank's nodes at time `time`: eta [Nx] and the fixed-frame
 * u, w [Nz+1][Nx] at z = sigma (h + eta) - h (each may be NULL; host or
 * device arrays), *c = phase speed (may be NULL).  H is limited to 0.85 x
 * the Battjes steepness 0.1401 tanh(0.8863 k h) (WT_EINVAL above it);
 * WT_ENOCONV if Newton's method fails.  2D tanks only.
 */
int wt_stream_function_wave(wt_tank* t, int nwaves, double H, int nmodes, double time, double* eta,
                            double* u, double* w, double* c);
/* The same stream-function solve (the Sec. 5.2 initial condition) without a
 * tank: host code only, no GPU or CUDA call.  Wavenumber k, still depth d, height H, gravity g, nmodes
 * (2..128), the same height limit and errors as wt_stream_function_wave.
 * Host outputs (each may be NULL): params[3] = (c, Q, R) - phase speed
 * (equal to the moving frame's current U), volume flux under the wave in
 * that frame, Bernoulli constant; B[nmodes] = stream-function coefficients
 * B_1..B_N of psi = -U y + sum_j B_j sinh(j k y) / cosh(j k d) cos(j k X),
 * y the height above the bed; E[nmodes + 1] = cosine coefficients E_0..E_N
 * of the surface, eta(X) = sum_j E_j cos(j k X) with X = x - c t. */
int wt_stream_function_solve(double k, double d, double H, double g, int nmodes, double* params, double* B,
                             double* E);

/*
 * Solver autotuner.  Times wt_poisson_solve on this tank's problem
 * A_{a,b} p = rhs (eta_a, eta_b [Ny][Nx], rhs [Nz+1][Ny][Nx]; host or device)
 * from a zero initial guess under a grid of settings - omega in {0.3, 0.4,
 * 0.5, 0.6}, (nu1, nu2) in {(1,1), (2,2), (3,3)}, coarsest_max in {32, 64,
 * 128}, and mode in {WT_MIXED, WT_REFINE} unless the tank is in WT_FP64 - one
 * warm-up solve plus the median of reps (1..100) timed solves each, and keeps
 * the fastest setting that reaches the tolerance; then, on that setting, the
 * WT_REFINE with inner_tol 1e-4 and 1e-3 (unless the tank is in WT_FP64),
 * the spectral smoothers (smoother 1 and 2, nu1 = nu2 in {1, 2}, on every
 * level or on the finest one, two or three levels: spectral_min; then
 * omega_s 0.8 and 1.2), the
 * full-multigrid cycle (cycle = 1) and the V-cycle's launch schedule (tail_max 2048 or 8192 with tail_cluster 0 or
 * 16, or vcycle_grid = 1).  The paper leaves these
 * choices open (Sec. 4.1).  On success the tank uses the winner, *best holds
 * it, *best_ms its median time and *entry_ms that of the options on entry
 * (best_ms <= entry_ms: the entry options are one of the candidates).  Any
 * output pointer may be NULL.  WT_ENOCONV (tank options unchanged) if no
 * candidate converged.  Allocates and frees temporary device buffers.
 */
int wt_autotune(wt_tank* t, const double* eta_a, const double* eta_b, const double* rhs, int reps,
                wt_options* best, double* best_ms, double* entry_ms);
/* The same search with one wt_step(dt) from the tank's current state as the
 * timed unit (the state, time included, is restored after every trial and on
 * return; solver statistics restart).  Needs a state (wt_set_state). */
int wt_autotune_step(wt_tank* t, double dt, int reps, wt_options* best, double* best_ms, double* entry_ms);
/* File of tuned options shared by wt_autotune and wt_autotune_step in this
 * process: path, or NULL to stop using one (the default).  JSON lines, one
 * search result per line, keyed by the kind of search ("solve" / "step"),
 * the finest grid Nx x Ny x Nz, whether the tank runs WT_FP64, filter,
 * linear and tol.  A search whose key is in the file applies the stored
 * options without measuring (*best_ms, *entry_ms: the stored times); a
 * completed search replaces its line (written to path.tmp, then renamed).
 * WT_EINVAL for an empty path.  Thread-safe. */
int wt_autotune_cache(const char* path);

/*
 * Batches of independent 2D tanks of uneven size.  The paper advances one
 * tank at a time; the batch has no counterpart there, and each of its tanks
 * takes the step of wt_step (Sec. 3.1-3.3, the solver of Sec. 4).  The tanks
 * advance together by one
 * persistent kernel launch per wt_batch_step: one CTA owns one tank and runs
 * all of its Runge-Kutta stages (free surface, metric, smoother set-up,
 * forcing, mixed-stage Poisson solve - FP64 flexible GMRES with the FP32 or
 * FP64 p-multigrid V-cycle, or FP64 refinement around an FP32 one - and the
 * projection); the largest tanks start first.
 * wt_create_batch: tank i has Nx[i], Nz[i], L[i] and bathymetry[i] ([Nx[i]],
 * host or device), Ny = 1; g and nu as in wt_create.  Each tank's coarsest
 * level must have at most 64 unknowns.  The batch owns its tanks.
 * wt_batch_set_options applies one option set to every tank: WT_MIXED (FP64
 * GMRES, FP32 V-cycle; the default), WT_FP64 (FP64 GMRES, FP64 V-cycle, the
 * plain method) or WT_REFINE (FP64 residual, FP32 GMRES + FP32 V-cycle to
 * inner_tol, at most max_ir refinements per solve); block-Jacobi V-cycles
 * only (smoother 0, cycle 0; WT_ENOTSUP otherwise).
 * wt_batch_set_state / get_state: tank i's eta [Nx], u, w [Nz+1][Nx].
 * wt_batch_step: nsteps full steps, dt[i] for tank i (host array); returns
 * after all tanks finished; WT_EBREAK / WT_ENOCONV if any tank failed.
 * wt_batch_stats: solves, Krylov iterations and the last relative residual of
 * tank i (accumulated over all wt_batch_step calls).
 */
typedef struct wt_batch wt_batch;
int wt_create_batch(int ntanks, const int* Nx, const int* Nz, const double* L, double g, double nu,
                    const double* const* bathymetry, wt_batch** out);
int wt_batch_set_options(wt_batch* b, const wt_options* opt);
int wt_batch_set_state(wt_batch* b, int i, const double* eta, const double* u, const double* w,
                       double time);
int wt_batch_get_state(const wt_batch* b, int i, double* eta, double* u, double* w, double* time);
int wt_batch_step(wt_batch* b, const double* dt, int nsteps);
int wt_batch_stats(const wt_batch* b, int i, long* solves, long* iterations, double* last_rel);
/* Launch later wt_batch_step calls on the given cudaStream_t (passed as
 * void*; NULL returns to the batch's own stream), e.g. to bracket them with
 * the caller's CUDA events.  The call still returns after the step. */
int wt_batch_set_stream(wt_batch* b, void* stream);
/* Number of tanks, tank i's sizes, and the option set the batch runs with. */
int wt_batch_size(const wt_batch* b, int* ntanks);
int wt_batch_tank_dims(const wt_batch* b, int i, int* Nx, int* Nz);
int wt_batch_get_options(const wt_batch* b, wt_options* opt);
/*
 * Batch autotuner: times one wt_batch_step(dt) of the whole batch - the
 * makespan of the persistent launch - from the tanks' current states
 * (restored before every trial and on return) for omega in {0.3, 0.4, 0.5,
 * 0.6} x (nu1, nu2) in {(1,1), (2,2)} on top of the batch's options, then,
 * unless the batch runs WT_FP64, the refinement form with inner_tol 1e-4 and
 * 1e-3 on the winner; median of reps (1..20) trials each; keeps the fastest
 * that completes.  best, best_ms, entry_ms as in wt_autotune (any may be NULL).
 * WT_ENOCONV if no candidate completes a step.
 */
int wt_batch_autotune(wt_batch* b, const double* dt, int reps, wt_options* best, double* best_ms,
                      double* entry_ms);
int wt_batch_destroy(wt_batch* b);

/*
 * Launch accounting and kernel timing (no counterpart in the paper; used to
 * measure the kernels against the GB300 roofline).  Kernel classes:
 *   WT_K_ROWPASS  spectral x-row / y-line passes (FFT derivative, resampling,
 *                 filter) with fused epilogues
 *   WT_K_OPCOLS   sigma part of the operator, WT_K_SMOOTH block-Jacobi update
 *                 (+ Nyquist coefficients), WT_K_COLMAT sigma transfers and
 *                 sigma derivatives, WT_K_BLOCKINV column-block inverses,
 *                 WT_K_COARSE coarsest LU, WT_K_KRYLOV GMRES vector kernels,
 *                 WT_K_STAGE metric and Runge-Kutta pointwise kernels,
 *                 WT_K_TAIL the single-CTA lower V-cycle.
 * wt_profile(t, mask) starts a timing window: every later launch of a class
 * whose bit is set in mask is bracketed by CUDA events on the tank's stream
 * (mask = 0 stops timing).  wt_profile_read sums the window for one class:
 * total device milliseconds, launches, and the algorithmic bytes and flops
 * of those launches.  wt_get_launches: all kernel launches of the tank since
 * wt_create (counted whether or not timing is on).
 */
enum wt_kernel_class {
  WT_K_ROWPASS = 0, WT_K_OPCOLS = 1, WT_K_SMOOTH = 2, WT_K_COLMAT = 3,
  WT_K_BLOCKINV = 4, WT_K_COARSE = 5, WT_K_KRYLOV = 6, WT_K_STAGE = 7, WT_K_TAIL = 8,
  WT_K_COUNT = 9
};
int wt_profile(wt_tank* t, unsigned mask);
int wt_profile_read(wt_tank* t, int kernel_class, double* ms, long* launches, double* bytes,
                    double* flops);
int wt_get_launches(const wt_tank* t, long* launches);

/*
 * Device time of one unit of the solve, for roofline measurements (no
 * counterpart in the paper).  With the geometry of (eta_a, eta_b) set up as
 * for a solve, reps back-to-back units on a fixed input are captured into one
 * CUDA graph, replayed once to warm up and once between two CUDA events on
 * the tank's stream: *ms_per_call = elapsed / reps, *launches_per_call (may
 * be NULL) = kernels per unit.  No per-launch events, so the figure is not
 * inflated by event overhead.  what: WT_TIME_OPERATOR (Ap = A_{a,b} p on the
 * finest level, Eq. poissonp: the unit whose algorithmic traffic is read p +
 * write Ap) or WT_TIME_VCYCLE (one V-cycle, Algorithm 1).  precision:
 * WT_FP64 or WT_FP32.  reps in [1, 10000].  WT_EINVAL while wt_profile
 * timing is on.
 */
enum wt_time_unit { WT_TIME_OPERATOR = 0, WT_TIME_VCYCLE = 1 };
int wt_time_kernel(wt_tank* t, const double* eta_a, const double* eta_b, int what, int precision, int reps,
                   double* ms_per_call, long* launches_per_call);

/*
 * Allocation-free operator apply (the paper has no counterpart; this is a
 * deployment variant of wt_apply_operator).  For callers that cannot call
 * cudaMalloc - code living inside another framework's memory pool, an
 * embedded solver that only ever receives buffers, a process whose device
 * footprint is fixed after start-up - this entry point needs no tank and
 * allocates nothing: all temporaries live in one file-scope __device__ array
 * of 2.5 MiB that every GPU loading the library holds until exit.
 * Computes Ap = A_{a,b} p of a 2D tank (Ny = 1) in FP64, the same result as
 * wt_apply_operator(..., WT_FP64), with the same kernels.
 *   Nx: power of two in [4, 2048]; Nz in [2, 32] (limit of the static array;
 *   larger sizes return WT_EINVAL).  L: domain length.
 *   h, eta_a, eta_b: device arrays [Nx]; p, Ap: device arrays [Nz+1][Nx]
 *   (host pointers return WT_EINVAL).  stream: cudaStream_t or NULL.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it.  All calls share the array and it
 * keeps the last call's contents, so calls that overlap on the GPU
 * (different streams or threads) race; serialise them.  Returns after Ap is complete; WT_EBREAK when
 * h + eta <= 0 or a value is not finite.
 */
int wt_apply_operator_static(int Nx, int Nz, double L, const double* h, const double* eta_a,
                             const double* eta_b, const double* p, double* Ap, void* stream);

/* Release every resource of the tank.  t may be NULL. */
int wt_destroy(wt_tank* t);

/* Copy the calling thread's last error text into buf (always terminated).
 * Returns the status code that produced it. */
int wt_last_error(char* buf, size_t n);

#ifdef __cplusplus
}
#endif

#endif /* WT_H */
