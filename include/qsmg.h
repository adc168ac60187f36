/*
 * qsmg.h -- C ABI of the GB300 (sm_103a) quasi-static projection library.
 *
 * The library implements the hot path of Boffi & Rycroft, "Parallel
 * three-dimensional simulations of quasi-static elastoplastic solids"
 * (arXiv 1904.03808): one quasi-static projection step (section 3.3) and the
 * geometric-multigrid solve of its velocity system (section 3.6), on one GPU.
 *
 * Grid (section 3.4, section 4): nx * ny * nz cells of spacing h, periodic in
 * x and y; velocity at cell corners (i, j, k), i < nx, j < ny, 0 <= k <= nz,
 * with the planes k = 0 and k = nz holding Dirichlet wall velocities; stress
 * and effective temperature at cell centres.
 *
 * Layouts (all FP64, C-contiguous, x fastest, DEVICE memory unless stated):
 *   velocity / corner fields   (3, nz+1, ny, nx)   components x, y, z
 *   stress                     (6, nz, ny, nx)     xx, yy, zz, yz, xz, xy
 *   effective temperature      (nz, ny, nx)
 *   stencil table              (27, 3, 3)          offset (dz+1)*9+(dy+1)*3+(dx+1)
 *
 * The linear system.  Eq. (30), dt div(C : D^{n+1}) = -div(sigma*), is
 * discretised with the collocated 3-point second derivative (Eq. 32) and the
 * 4-point mixed derivative of section 3.4, and scaled by -h^2/(mu dt):
 *     Ahat v = b,   Ahat = -(h^2/(mu dt)) A,   b = (h^2/(mu dt)) div_h sigma*.
 * Ahat is symmetric positive definite (section 3.3, condition B) and depends
 * on lambda/mu only.  Unknowns are the interior corners (0 < k < nz); wall
 * values enter through the couplings to planes 0 and nz.
 *
 * Ownership.  The caller owns every array passed in and keeps it alive for
 * the call; the library owns its level hierarchy and scratch, allocated in
 * mg_setup and released by mg_free.  All device work is issued on the stream
 * given to mg_setup; calls return after that stream has finished the work
 * they issued (the residual norms are read back to the host).
 *
 * Errors.  Every call returns an mg_status; nothing throws or traps.  A
 * failing call leaves a message for mg_last_error() (thread-local).
 */
#ifndef QSMG_H
#define QSMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MG_OK = 0,
    MG_ERR_ARG = 1,       /* null pointer, bad option value */
    MG_ERR_SHAPE = 2,     /* grid not supported (see mg_setup) */
    MG_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    MG_ERR_OOM = 4,       /* device allocation failed */
    MG_ERR_NOCONV = 5,    /* max_cycles reached above the tolerance */
    MG_ERR_NONFINITE = 6, /* residual norm became NaN or Inf */
    MG_ERR_STATE = 7      /* context unusable (earlier CUDA failure) */
} mg_status;

enum { MG_FP64 = 0, MG_MIXED = 1 };
/* mg_opts.flags */
enum {
    MG_FLAG_COLOUR_PASSES = 1, /* FP32 sweeps: one launch per colour */
    MG_FLAG_NO_GRAPH = 2,      /* FP32 inner cycles: plain launches, no CUDA graph */
    MG_FLAG_FUSED_SWEEP = 4,   /* finest FP32 sweeps: both k-parities in one launch */
    MG_FLAG_UNFUSED_TRANSFERS = 8, /* finest FP32 residual and restriction as
                                      separate passes */
    MG_FLAG_ADVECT_STRESS = 16     /* qs_step / qs_run / qs_stress_predict: add the
                                      stress advection -(v.grad) sigma to sigma* */
};
enum { MG_HIST = 128 };

/* Grid: nx, ny even and >= 4, nz even and >= 2 (cells); h spacing (m). */
typedef struct { int nx, ny, nz; double h; } mg_grid;

/* Isotropic moduli (Pa): bulk K and shear mu; lambda = K - 2 mu / 3
 * (Table 1 gives K and mu). */
typedef struct { double K, mu; } mg_moduli;

/*
 * Wall velocities (section 4, Eqs. 37-38; section 5, Eqs. 48-49).
 * kind 0 simple shear: v(k=nz) = (+U(t),0,0), v(k=0) = (-U(t),0,0),
 *   U(t) = U_B t / t_ramp for t < t_ramp, else U_B.
 * kind 1..3 spinning disc on the top wall, read as a rotation with angular
 *   velocity omega (rad/s): u = -omega y f, v = omega x f, w = 0 with
 *   f = 1 for r^2 < R^2, else exp(-lambda_w (r^2 - R^2)^2), r^2 = (x^2+y^2)/L^2,
 *   L = nx h / 2, x = -L + i h, y = -ny h / 2 + j h.  Bottom wall: kind 1
 *   fixed, kind 2 the same rotation, kind 3 the opposite rotation.
 */
typedef struct {
    int kind;
    double U_B, t_ramp, omega, R, lambda_w;
} mg_bc;

/* STZ plasticity (section 3.1, Table 1).  Energies as temperatures:
 * Delta_K = Delta/k_B, ez_K = e_z/k_B.  Omega (m^3), kB (J/K), l the chi
 * diffusion length (m), sY (Pa), tau0 (s). */
typedef struct {
    double tau0, eps0, c0, Delta_K, Omega, T, chi_inf, ez_K, sY, l, kB;
} stz_params;

/*
 * Solver options.
 *   precision     MG_FP64: FP64 V-cycles.  MG_MIXED: FP32 V-cycles inside an
 *                 FP64 iterative-refinement loop (FP64 outer residual, FP64
 *                 coarsest solve).
 *   nu1, nu2      pre/post Gauss-Seidel sweeps (section 3.6 uses 2 and 2).
 *   max_cycles    cap on V-cycles per solve (<= MG_HIST - 1).
 *   inner_cycles  MG_MIXED: FP32 V-cycles per outer refinement step (<= 10);
 *                 0 picks the count per step from the FP64 residual and the
 *                 observed V-cycle contraction.
 *   flags         0 or an OR of: MG_FLAG_COLOUR_PASSES runs FP32 sweeps as
 *                 eight colour launches instead of the two-phase kernels
 *                 (row strips, whole planes, tiles); MG_FLAG_NO_GRAPH issues the FP32 inner cycles as
 *                 plain launches instead of replaying a CUDA graph captured
 *                 at their first use; MG_FLAG_FUSED_SWEEP runs each
 *                 finest-level FP32 sweep as one cooperative launch (both
 *                 k-parities, with ready flags between neighbouring row
 *                 strips) instead of two, where the grid suits it: a third
 *                 less DRAM traffic, but slower on GB300 (same arithmetic;
 *                 kept for comparison); MG_FLAG_UNFUSED_TRANSFERS runs the
 *                 finest-level FP32 residual and its restriction as two passes
 *                 with the residual stored instead of one fused pass (kept
 *                 for comparison); MG_FLAG_ADVECT_STRESS adds to the
 *                 intermediate stress of Eq. (27) the advection term
 *                 -(v.grad) sigma of the general constitutive law (section 2),
 *                 sigma* -= dt (u.grad) sigma^n with u the mean of each cell's
 *                 8 corner velocities of v^n and ENO derivatives (Eq. 33),
 *                 cell fields extrapolated linearly two layers beyond the z
 *                 boundaries (the reverse-mode entry points reject it).
 */
typedef struct {
    int precision;
    int nu1, nu2;
    int max_cycles;
    int inner_cycles;
    int flags;
} mg_opts;

/* Per-solve statistics.  resid_hist[0] is the relative residual of the
 * initial guess, resid_hist[c] after V-cycle c (FP64 mode) or after outer
 * step c (mixed mode).  bnorm is ||b_lifted||_2. */
typedef struct {
    int cycles;       /* V-cycles run (FP64 or FP32) */
    int outer_iters;  /* refinement steps (mixed) or cycles (FP64) */
    double rel_resid; /* final ||b - Ahat v||_2 / ||b_lifted||_2 */
    double bnorm;
    double resid_hist[MG_HIST];
} mg_stats;

/* Simulation state, caller-owned device arrays (layouts above); t is the
 * time of the state, step a counter the library increments. */
typedef struct {
    double *v, *sigma, *chi;
    double t;
    long step;
} qs_state;

typedef struct mg_ctx mg_ctx;

/*
 * mg_setup -- build the multigrid hierarchy of section 3.6 for the scaled
 * operator and allocate every buffer the solve and the step need.
 *   Levels halve each dimension while all three are even and their halves are
 *   >= 4 (the paper's ceil(n/2) coarsening restricted to even sizes); coarse
 *   operators are the Galerkin products A_k = R A_{k-1} T (Eq. 36) with linear
 *   interpolation T and R = T^T; the coarsest operator is inverted densely
 *   (at most 3072 unknowns, else MG_ERR_SHAPE).
 *   stz and bc may be NULL if only mg_solve will be used.
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: MG_ERR_ARG, MG_ERR_SHAPE, MG_ERR_OOM, MG_ERR_CUDA.
 */
mg_status mg_setup(const mg_grid *grid, const mg_moduli *moduli, const mg_bc *bc,
                   const stz_params *stz, const mg_opts *opts, void *stream, mg_ctx **out);

/*
 * mg_solve -- multigrid solve of Ahat v = rhs (section 3.6) to
 *   ||rhs - Ahat v||_2 <= tol * ||b_lifted||_2, where b_lifted is rhs minus the
 *   wall columns applied to the wall values.  V-cycle: nu1 pre-sweeps of
 *   8-colour block Gauss-Seidel (colours (i&1)+2(j&1)+4(k&1) visited 0..7),
 *   residual, restriction, recursive coarse correction, prolongation, nu2
 *   post-sweeps (colours 7..0); dense solve on the coarsest level.
 *   rhs: device (3, nz+1, ny, nx); its wall planes are ignored.
 *   v: device (3, nz+1, ny, nx); in: initial guess (interior) and wall values;
 *      out: solution (walls unchanged).
 *   tol <= 0 runs exactly opts.max_cycles V-cycles (or refinement steps) and
 *   returns MG_OK.  If b_lifted = 0 the interior of v is set to 0.
 *   stats may be NULL.
 * Errors: MG_ERR_NOCONV (v holds the last iterate), MG_ERR_NONFINITE,
 *   MG_ERR_ARG, MG_ERR_CUDA.
 */
mg_status mg_solve(mg_ctx *ctx, const double *rhs, double *v, double tol, mg_stats *stats);

/*
 * qs_step -- one quasi-static projection step (section 3.3) from state->t to
 * state->t + dt, in place:
 *   sigma* and D^pl from (v^n, sigma^n, chi^n): Eq. (27) with the STZ rate of
 *     Eqs. (20)-(22) (D^pl = 0 for sbar <= s_Y) and the Eq. (31) gradient;
 *   chi^{n+1} by Eq. (26) (conservative diffusion with face-averaged D^pl;
 *     z ghost cells from linearly extrapolated sigma and chi);
 *   wall velocities at t + dt; b = (h^2/(mu dt)) div sigma* at interior
 *   corners; v^{n+1} by mg_solve warm-started from v^n;
 *   sigma^{n+1} = sigma* + dt C : D^{n+1} (Eq. 29).
 * Requires stz and bc at setup.  Errors as mg_solve; on a solver error the
 * state is still advanced with the last iterate.
 */
mg_status qs_step(mg_ctx *ctx, qs_state *state, double dt, double tol, mg_stats *stats);

/*
 * qs_run -- nsteps quasi-static projection steps (section 3.3) of size dt,
 * in place: the same arithmetic as nsteps calls of qs_step, with the stress
 * correction of each step (Eq. 29) and the predictor of the next (Eq. 27)
 * done in one pass over the cells, since both take the Eq. (31) gradient of
 * the same velocity v^{n+1}.  Between the calls' steps nothing is observable,
 * so the state is only complete on return.  qs_step is qs_run with nsteps = 1.
 *   stats: NULL, or an array of nsteps entries that receives each step's
 *          solve statistics.
 *   nsteps = 0 leaves the state untouched and returns MG_OK.
 * Errors as qs_step.  On MG_ERR_NOCONV or MG_ERR_NONFINITE the run stops
 * after the step whose solve failed, with that step completed from the last
 * iterate; state->step and state->t count the steps taken.
 */
mg_status qs_run(mg_ctx *ctx, qs_state *state, int nsteps, double dt, double tol,
                 mg_stats *stats);

/* Release every buffer of the context (NULL is a no-op). */
void mg_free(mg_ctx *ctx);

const char *mg_status_str(mg_status s);
const char *mg_last_error(void);

/* ------------------------------------------------------------------ */
/* Component entry points (the same kernels the solve and step use),   */
/* exposed for parity tests against the oracle.  Device pointers, FP64  */
/* unless stated.  Errors: MG_ERR_ARG (null array, bad level), MG_ERR_CUDA. */
/* ------------------------------------------------------------------ */

/* number of levels, and the cell dimensions of one level (dims[3]) */
int mg_num_levels(const mg_ctx *ctx);
mg_status mg_level_dims(const mg_ctx *ctx, int level, int *dims);

/* host copy of a level's stencil table (27, 3, 3), scaled operator Ahat */
mg_status mg_level_stencil(const mg_ctx *ctx, int level, double *host_S);

/* r = b - A_level x on interior nodes, zero on wall planes.  x, b, r are
 * level-sized corner arrays (3, nz_l+1, ny_l, nx_l); r must not alias x. */
mg_status mg_residual(mg_ctx *ctx, int level, const double *b, const double *x, double *r);

/* The same residual in FP32, as the mixed-precision inner V-cycles compute
 * it (section 3.6 operator, single-precision arithmetic): float arrays in
 * natural column order, r must not alias x.  On the finest level the arrays
 * pass through the solver's own FP32 buffers, so this call must not overlap
 * an mg_solve / qs_step on the same context. */
mg_status mg_residual32(mg_ctx *ctx, int level, const float *b, const float *x, float *r);

/* bc = T^T (b - A_level x) in FP32 (level -> level + 1): the residual and its
 * restriction (section 3.6), as the mixed-precision V-cycle computes them.
 * On the finest level, where its row-strip kernel takes the grid, the two
 * are fused and the residual is never stored: the kernel applies the x and y
 * parts of the full weighting to each tile's residual and a second kernel
 * the z part.  b, x: (3, nz+1, ny, nx) of the level, natural column order;
 * bc: the next level's (3, nz/2+1, ny/2, nx/2), wall planes not written.
 * Uses the solver's own FP32 buffers (must not overlap a solve on the same
 * context).  Errors: MG_ERR_ARG (null array, no coarser level), MG_ERR_CUDA. */
mg_status mg_residual_restrict32(mg_ctx *ctx, int level, const float *b, const float *x,
                                 float *bc);

/* nsweeps Gauss-Seidel sweeps on level `level`, colours 0..7 if
 * descending == 0 else 7..0; FP64 (precision 0) or FP32 arrays (precision 1). */
mg_status mg_smooth(mg_ctx *ctx, int level, const void *b, void *x, int nsweeps, int descending,
                    int precision);

/* bc = T^T r (level -> level+1) and x += T xc (level+1 -> level), FP64 */
mg_status mg_restrict(mg_ctx *ctx, int level, const double *r, double *bc);
mg_status mg_prolong_add(mg_ctx *ctx, int level, const double *xc, double *x);

/* one FP64 V-cycle on the finest level (b, x as in mg_solve) */
mg_status mg_vcycle(mg_ctx *ctx, const double *b, double *x);

/* pointwise pieces of qs_step (device arrays; sigma_star 6 per cell, dpl and
 * sbar 1 per cell, b corner-sized) */
mg_status qs_stress_predict(mg_ctx *ctx, const double *v, const double *sigma, const double *chi,
                            double dt, double *sigma_star, double *dpl, double *sbar);
mg_status qs_chi_update(mg_ctx *ctx, const double *sigma, const double *chi, const double *dpl,
                        const double *sbar, double dt, double *chi_new);
mg_status qs_rhs(mg_ctx *ctx, const double *sigma_star, double dt, double *b);
mg_status qs_stress_correct(mg_ctx *ctx, const double *v, const double *sigma_star, double dt,
                            double *sigma);
mg_status qs_wall_fill(mg_ctx *ctx, double *v, double t);

/* ------------------------------------------------------------------ */
/* Reverse mode (the paper evaluates no gradient; these entry points      */
/* differentiate the step of section 3.3 as this library computes it)    */
/* ------------------------------------------------------------------ */

/*
 * qs_step_adjoint -- the transpose of one qs_step: the adjoints of the state
 * a step starts from, given those of the state it produces.  Each equation of
 * the step is transposed in turn: the stress correction (Eq. 29), the
 * projection solve (Eq. 30; the scaled operator is symmetric, so its
 * transpose is one more mg_solve of the same operator with zero walls, to
 * `tol`), the right-hand side (the corner divergence, transposed to a cell
 * gradient), the chi update (Eq. 26, z-wall ghosts included), the STZ rate
 * (Eqs. 20-22; zero derivative at or below yield) and the predictor
 * (Eq. 27), whose velocity gradient (Eq. 31) is transposed to the corners.
 * The wall velocities are prescribed, so they carry no adjoint.
 *   state: device arrays of the state the forward step starts from (v with
 *       its wall values, sigma, chi), as passed to qs_step; not modified.
 *   dt: the forward step's dt.
 *   work_weight: weight w of this step's plastic work 2 D^pl sbar dt h^3
 *       summed over cells (the growth term of Eq. 26), added to the
 *       objective.
 *   vbar (3, nz+1, ny, nx), sigbar (6, nz, ny, nx), chibar (nz, ny, nx):
 *       device, caller-owned; on entry the adjoints of the step's output
 *       (v^{n+1}, sigma^{n+1}, chi^{n+1}), on return those of its input.
 *       Stress adjoints are per stored component (an off-diagonal entry's
 *       adjoint is the derivative with respect to the stored value, which
 *       feeds both matrix entries).  vbar's wall planes are ignored on entry
 *       and zero on return.
 *   stats: the adjoint solve's statistics (may be NULL).
 * The first call allocates the adjoint scratch (about 18 doubles a cell) on
 * the context.  Errors: MG_ERR_ARG, MG_ERR_OOM, MG_ERR_CUDA, MG_ERR_STATE,
 * and the solve's MG_ERR_NOCONV / MG_ERR_NONFINITE (the outputs are then
 * those of the last iterate).
 */
mg_status qs_step_adjoint(mg_ctx *ctx, const qs_state *state, double dt, double tol,
                          double work_weight, double *vbar, double *sigbar, double *chibar,
                          mg_stats *stats);

/*
 * qs_plastic_work -- the forward half of qs_plastic_work_grad: W = the
 * plastic work of nsteps qs_steps from `state` (sum over steps and cells of
 * 2 D^pl sbar dt h^3 -- the plastic power of Eq. 26's growth term -- with
 * D^pl and sbar of the state each step starts from); state is left at the
 * final state, as after nsteps qs_step calls.
 *   checkpoints: device, caller-owned, or NULL.  If given, it receives a copy
 *       of the state every checkpoint_every steps (steps 0, k, 2k, ...):
 *       ceil(nsteps / k) blocks of 3 (nz+1) ny nx + 7 nz ny nx doubles, each
 *       v (3, nz+1, ny, nx), then sigma (6, nz, ny, nx), then chi (nz, ny, nx).
 *       qs_plastic_work_backward takes it.
 *   work: host, receives W.
 *   stats: the last solve's statistics (may be NULL).
 * Makes no state copies of its own.  Errors: as qs_step; MG_ERR_ARG for nsteps < 1,
 * checkpoint_every < 1, or a context without stz/bc parameters.
 */
mg_status qs_plastic_work(mg_ctx *ctx, qs_state *state, int nsteps, double dt, double tol,
                          int checkpoint_every, double *checkpoints, double *work,
                          mg_stats *stats);

/*
 * qs_plastic_work_backward -- the reverse half: dW/dchi0 from the checkpoints
 * a qs_plastic_work call wrote with the same nsteps, dt, tol and
 * checkpoint_every, its state having started at time t0 and step count
 * step0.  Runs qs_step_adjoint backwards one segment at a time, recomputing
 * the segment's states from its checkpoint (the forward kernels and
 * reductions are deterministic and the times are re-accumulated from t0 as
 * the forward steps did, so the recomputed states equal the first ones bit
 * for bit).
 *   checkpoints: device, as written by qs_plastic_work; not modified.
 *   chibar: device (nz, ny, nx), receives dW/dchi0.
 *   stats: the last adjoint solve's statistics (may be NULL).
 * Device memory: checkpoint_every state copies plus two adjoint arrays,
 * allocated for the call and freed before it returns, and the context's
 * adjoint scratch (qs_step_adjoint).
 * Errors: as qs_step and qs_step_adjoint, MG_ERR_ARG as qs_plastic_work.
 */
mg_status qs_plastic_work_backward(mg_ctx *ctx, const double *checkpoints, double t0, long step0,
                                   int nsteps, double dt, double tol, int checkpoint_every,
                                   double *chibar, mg_stats *stats);

/*
 * qs_plastic_work_grad -- qs_plastic_work and qs_plastic_work_backward in one
 * call: W (host `work`) and dW/dchi0 (device `chibar`, (nz, ny, nx)), the
 * derivative of the plastic work of nsteps steps with respect to the initial
 * chi field.  state is left at the final state.  The checkpoints, every
 * checkpoint_every steps, are allocated for the call and freed before it
 * returns (ceil(nsteps / checkpoint_every) + checkpoint_every state copies,
 * 10 doubles a cell each, plus two adjoint arrays).
 * Errors: as qs_step and qs_step_adjoint, MG_ERR_ARG for nsteps < 1 or
 * checkpoint_every < 1.
 */
mg_status qs_plastic_work_grad(mg_ctx *ctx, qs_state *state, int nsteps, double dt, double tol,
                               int checkpoint_every, double *chibar, double *work,
                               mg_stats *stats);

/*
 * qs_explicit_step -- nsteps steps of the explicit method of section 3.2,
 * the forward-Euler comparison scheme of the paper (no projection; the
 * time step is limited by the elastic wave speed and by the damping,
 * dt <= h^2 / (6 kappa)).  Each step, from the state at t:
 *   stress (Eq. 25): sigma += dt (-(u.grad) sigma + L sigma + sigma L^T
 *     - tr(L) sigma + C:(D - D^pl sigma0 / sbar)), L and D from the Eq. (31)
 *     gradient of v, u the mean of a cell's 8 corner velocities;
 *   chi (Eq. 26), as in qs_step;
 *   velocity (Eq. 24) at interior corners: v += dt (-(v.grad) v
 *     + div sigma / rho + kappa lap v), the corner divergence of Eq. (31)
 *     and the Laplacian of Eq. (32);
 *   the advection terms by the ENO derivative of Eq. (33), its stencils
 *   reaching two points out; beyond the walls v is reflected through the
 *   wall value and the cell fields are extrapolated linearly;
 *   walls set at t + dt; state->t += dt, state->step += 1.
 * The printed Eq. (24) carries neither rho on the advection term nor on the
 * damping; here both are read as terms of rho dv/dt, with kappa a
 * diffusivity (m^2/s), as the paper's kappa = kappa' h and its stability
 * limit imply.
 *   rho: density (kg/m^3); kappa: damping diffusivity (m^2/s), >= 0.
 * Uses the context's moduli, STZ parameters and walls; allocates nothing.
 * Errors: MG_ERR_ARG (null arrays, dt <= 0, rho <= 0, kappa < 0,
 * nsteps < 0, context without stz/bc), MG_ERR_CUDA, MG_ERR_STATE.
 */
mg_status qs_explicit_step(mg_ctx *ctx, qs_state *state, double dt, double rho, double kappa,
                           int nsteps);

/* ------------------------------------------------------------------ */
/* Measurement hooks                                                   */
/* ------------------------------------------------------------------ */

/* Enable (1) or disable (0) timing of the finest-level smoothing calls: a
 * CUDA event pair is recorded on the context's stream around every pre- and
 * post-smoothing call on level 0; enabling resets the totals. */
mg_status mg_profile(mg_ctx *ctx, int enable);

/* Totals since mg_profile(ctx, 1): device milliseconds spent in finest-level
 * smoothing, sweeps run there, and kernel launches those sweeps made. */
mg_status mg_profile_read(mg_ctx *ctx, double *smooth_ms, long *smooth_sweeps,
                          long *smooth_launches);

/* Kernels this library has launched since it was loaded (all contexts). */
long mg_launch_count(void);

/* ------------------------------------------------------------------ */
/* Allocation-free entry point (no counterpart in the paper)           */
/* ------------------------------------------------------------------ */

/*
 * mg_residual_restrict_static -- bc = T^T (b - Ahat x) on the finest level of
 * an nx*ny*nz grid: the residual and full-weighting restriction kernels of the
 * V-cycle, for callers that cannot allocate device memory.  It needs no
 * context and calls no cudaMalloc, cudaFree or other allocating routine:
 * the intermediate fine-level residual lives in one fixed array compiled into
 * this library.  It serves callers whose device memory belongs to another
 * allocator with a fixed budget (a host framework's memory pool that must not
 * see hidden allocations), and callers on a latency-critical path where the
 * implicit device-wide synchronisation of cudaFree is not acceptable.
 *   grid, moduli: as for mg_setup (nx, ny even >= 4; nz even >= 2).
 *   b, x: device (3, nz+1, ny, nx); x carries the wall values.
 *   bc: device (3, nz/2+1, ny/2, nx/2); its interior receives T^T r, its wall
 *       planes are set to zero.
 *   stream: a cudaStream_t; the work is enqueued there and the call returns
 *       when that stream has finished it.
 * Limit: the array holds 2097152 doubles (16 MiB), so 3 (nz+1) ny nx must not
 * exceed 2097152 (e.g. 64^3 fits, 96^3 does not); larger grids return
 * MG_ERR_SHAPE with a message.  Every GPU that loads the library holds the
 * array until the process exits.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress; nothing is cached, so a cudaDeviceReset in between
 * does no harm).  The first call on a device may load the library's device
 * code there; make that first call before any stream capture.
 * All calls share the one array, which keeps the last call's residual (every
 * value a call reads was written by the same call): calls that overlap on the
 * GPU, from other streams or host threads, race on it, so serialise them.
 * Errors: MG_ERR_ARG, MG_ERR_SHAPE, MG_ERR_CUDA.
 */
mg_status mg_residual_restrict_static(const mg_grid *grid, const mg_moduli *moduli,
                                      const double *b, const double *x, double *bc,
                                      void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QSMG_H */
