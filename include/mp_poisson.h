/*
 * mp_poisson — GB300 (sm_103a) variable-density pressure-Poisson solve of the
 * projection step of an incompressible liquid–gas solver.
 *
 * The paper (arXiv 2312.11740, Section 2) fixes a staggered-grid,
 * finite-difference, fractional-step projection method: velocities on faces,
 * pressure and the level set phi at cell centres (Fig. 2 caption), phi > 0 in
 * gas and phi < 0 in liquid, variable density from phi (varDens, Section 3),
 * a multigrid Poisson solve (Grid_solvePoisson, Section 3).  The discrete
 * problem solved here is the ghost-fluid discretisation (Liu, Fedkiw & Kang
 * 2000) of  div((1/rho) grad p) = div u*  with the jump [p] = sigma*kappa:
 *
 *   (A p)_c = sum over the 6 faces f of c of beta_f (p_nb - p_c) / h^2,
 *   A p = b,  b = div_h u* + J - mean(div_h u* + J),  mean(p) = 0,
 *
 * beta_f the two-fluid face coefficient from phi, J the jump source, then
 * u = u* - beta_f (grad_h p - [p]) on every face (Delta t = 1).
 *
 * Memory layout (all arrays): C order, x fastest, idx = i + nx*(j + ny*k),
 * float64 unless stated.  Face arrays use low-face ownership: element idx of
 * an x-face array sits on the face between cells (i-1,j,k) and (i,j,k),
 * wrapped (face 0 is the face between cell nx-1 and cell 0); on a wall axis
 * face 0 is the wall, shared by the bottom and top walls.
 *
 * Pointers: "_dev" arguments are device pointers to caller-owned memory; the
 * library never frees them and keeps no pointer to them after a call
 * returns.  "_host" arguments are host memory (pageable or pinned).
 * Streams: all device work is enqueued on opts->stream; a call returns after
 * the work it enqueued is complete unless stated otherwise.
 * Errors: every call returns an mp_status and never aborts or traps; on
 * MP_ERR_CUDA the handle may be unusable and should be destroyed.
 * Threads: one handle must not be used by two host threads at once.
 */
#ifndef MP_POISSON_H
#define MP_POISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MP_OK = 0,
  MP_ERR_INVALID_ARG = 1,   /* bad size, pointer, option or boundary type */
  MP_ERR_NOT_CONVERGED = 2, /* max_iters reached; p and history hold the last iterate */
  MP_ERR_DIVERGED = 3,      /* NaN/Inf residual; p is unspecified */
  MP_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  MP_ERR_OOM = 5,           /* device or pinned allocation failed */
  MP_ERR_TIMEOUT = 6,       /* reserved: a bounded device wait gave up */
  MP_ERR_NO_NET = 7         /* learned initial guess requested without weights */
} mp_status;

/* Boundary type of an axis (per side where it differs).  The paper sets the
 * boundary types per side (xl_boundary_type / xr_boundary_type: inflow_ins,
 * outflow_ins in its runtime-parameter TOML figure, Section 4).  For the
 * pressure: a wall or an inflow side prescribes the normal velocity, so the
 * pressure correction has no normal gradient there (Neumann: the face
 * carries no pressure flux); an outflow side holds p = 0 on the boundary
 * face (Dirichlet, an antisymmetric ghost p_ghost = -p_cell whose face
 * coefficient is 1/rho of the cell's fluid).  With an outflow side the
 * operator has no null space: b keeps its mean and p is not gauged. */
typedef enum {
  MP_BC_PERIODIC = 0,          /* periodic (even number of cells) */
  MP_BC_NEUMANN = 1,           /* wall or inflow on both sides */
  MP_BC_DIRICHLET = 2,         /* outflow on both sides */
  MP_BC_NEUMANN_DIRICHLET = 3, /* wall/inflow on the low side, outflow on the high side */
  MP_BC_DIRICHLET_NEUMANN = 4  /* outflow on the low side, wall/inflow on the high side */
} mp_bc;

typedef struct {
  int nx, ny, nz;
} mp_grid;

/* Solver options.  mp_opts_default() fills the defaults given here. */
typedef struct {
  int precision;     /* 0 = FP64 throughout; 1 = mixed: FP32 smoothing/transfers and inner
                        iterations, FP64 outer residual, accumulation and coarsest solve.
                        Default 0. */
  int method;        /* 0 = conjugate gradients preconditioned by one symmetric V-cycle
                        (default); 1 = stationary V-cycle iteration. */
  int initial_guess; /* 0 = zero (default); 1 = the caller's p; 2 = learned network
                        (requires mp_poisson_set_net). */
  int max_iters;     /* outer iterations (FP64) or total inner iterations (mixed). Default 200. */
  int nu1, nu2;      /* pre/post red-black Gauss–Seidel sweeps on the finest level. Default 2, 2. */
  int nu_growth;     /* sweeps multiply by this per coarser level. Default 2. */
  int nu_max;        /* cap on sweeps per level. Default 12 (measured at 256^3 and 512^3:
                        2, 4, 8, 12, 12 ... sweeps down the levels).  The FP32 V-cycle's one-CTA tail
                        (its levels of at most 16^3 cells) uses at most 4. */
  double inner_rtol; /* mixed: the FP32 recurrence residual must fall by this factor below the
                        last true residual before the FP32 correction is folded into the FP64
                        solution and the residual replaced by the true FP64 one (reliable
                        update; the CG direction is kept).  Default 3e-3. */
  int inner_max;     /* mixed: at most this many FP32 iterations between true residuals.
                        Default 12. */
  int net_check;     /* learned guess p0 = alpha q (alpha energy-optimal) is kept when
                        0: its residual ||b - A p0|| is below ||b|| (default); with
                           deflation active, the residuals compared are those deflated CG
                           starts from, ||P (b - A p0)|| and ||P b|| (P = I - A Z E^-1 Z^T);
                        1: alpha is finite and nonzero, i.e. whenever the A-norm error of p0
                           is below that of the zero guess (always true for that alpha). */
  int deflate;       /* method 0: 1 (default) deflates CG by the indicator vectors of the
                        connected gas components (phi > 0), removing the bubbles' pressure
                        levels, which the V-cycle resolves poorly at density ratio 1000;
                        0 = plain MG-preconditioned CG.  Same converged answer.  Applies to
                        periodic and wall boundaries (off with an outflow side). */
  int smoother;      /* FP32 V-cycle levels (mixed precision) with nx a multiple of 8 and
                        no outflow side:
                        1 (default) = one fused pass per red-black sweep (both colours,
                        shared-memory halo staging, second iterate buffer); 0 = one
                        in-place launch per colour.  Bitwise the same result. */
  int label_limit;   /* bound on every find walk and union retry of the gas-component
                        labelling (default 8192; walks are a few steps long in practice).
                        A geometry whose labelling reaches it is solved without deflation
                        (mp_stats.components = 0). */
  int coarse_cluster; /* FP32 V-cycle: 1 (default) runs the level above the one-CTA tail and
                        every coarser level as one launch of an 8-CTA thread-block cluster
                        (distributed shared memory, cluster barriers between steps) where
                        the levels' z-planes split evenly; 0 = per-level launches down to
                        the one-CTA tail.  Same method, slightly different rounding. */
  void *stream;      /* cudaStream_t; NULL = legacy default stream. */
} mp_opts;

/* Statistics of the last mp_poisson_solve / mp_poisson_project_step. */
typedef struct {
  int iterations;      /* V-cycle applications (preconditioner or stationary steps) */
  int outer_steps;     /* mixed: true FP64 residuals formed after the first; FP64: = iterations */
  double relres;       /* final ||b - A p|| / ||b||, FP64, true residual */
  double r0;           /* initial ||b - A p0|| / ||b|| */
  int used_net;        /* 1 if the learned guess was kept, 0 if not requested or rejected */
  double net_relres;   /* ||b - A p_net|| / ||b|| of the learned guess, deflated as in
                          net_check 0 (0 if not requested); the guess is kept by the
                          residual check iff this is below 1 */
  int levels;          /* multigrid levels */
  int coarse_n;        /* unknowns of the coarsest (direct) level */
  int components;      /* gas components used as deflation vectors (0: deflation off) */
} mp_stats;

typedef struct mp_poisson *mp_handle;

/* Fill *opts with the defaults documented in mp_opts.
 * Defines: the options of the multigrid Poisson solve (Grid_solvePoisson,
 * Section 3); the paper gives no solver settings, each default is a stated,
 * measured choice. */
void mp_opts_default(mp_opts *opts);

/*
 * Defines: the variable-density pressure problem of the fractional-step
 * projection on the staggered grid (Section 2, Fig. 2 caption: phi > 0 in
 * air/gas), with the properties of each cell taken from phi (varDens and
 * MultiphaseMain, Section 3) through ghost-fluid face coefficients and the
 * surface-tension jump [p] = sigma*kappa (published ghost-fluid method,
 * Liu-Fedkiw-Kang 2000), and the multigrid hierarchy of Grid_solvePoisson
 * (Section 3).
 *
 * Allocate a solver for grid g (cell edge h > 0, boundary bc[axis] per axis)
 * and set its geometry from phi_dev (device, nx*ny*nz f64, phi > 0 gas),
 * liquid density rho_l > 0, gas density rho_g > 0, surface tension sigma >= 0.
 * Every axis must be >= 2 and even on periodic axes.  The hierarchy halves
 * all dims while they are all even and >= 4 and the level has more than 64
 * cells; the coarsest level must have at most 512 cells (else
 * MP_ERR_INVALID_ARG).  Allocates all device memory
 * the solver needs; no later call allocates.  opts may be NULL (defaults).
 */
mp_status mp_poisson_setup(mp_handle *out, mp_grid g, double h, const mp_bc bc[3],
                           const double *phi_dev, double rho_l, double rho_g, double sigma,
                           const mp_opts *opts);

/*
 * Defines: as mp_poisson_setup, for a level set that has moved (the level
 * set is advected every step, MultiphaseMain, Section 3).
 *
 * Recompute the geometry-dependent data (curvature, face coefficients, jump
 * source, coarse hierarchy, coarsest inverse) for a new phi on the same grid.
 * No allocation.
 */
mp_status mp_poisson_set_geometry(mp_handle hd, const double *phi_dev, double rho_l, double rho_g,
                                  double sigma);

/*
 * Defines: the phase-change variant (evaporation, the MultiphaseEvap unit
 * of Section 3, which adds interface mass transfer to the main multiphase
 * unit); the paper prints no formula, the reading is the ghost-fluid one.
 *
 * Set (mdot_dev != NULL) or clear (NULL) a phase-change mass flux: mdot_dev
 * is device memory, N f64 cell values of the mass flux per unit interface
 * area from liquid to gas (copied; the caller keeps ownership).  The normal
 * velocity then jumps by mdot [1/rho], [1/rho] = 1/rho_g - 1/rho_l, so the
 * pressure flux jumps by B = -mdot_G [1/rho] across every interface face
 * (mdot_G: the cell values interpolated to the interface point like the
 * curvature).  With p linear on each side of the interface the two jump
 * conditions give each of the face's two rows a share of B / h: the row of
 * cell c takes beta theta_nb rho_nb B / h, theta_nb the fraction of the
 * c-nb segment lying in the neighbour's fluid.  These shares join the jump
 * source J (mp_poisson_get_fields returns the sum); the velocity correction
 * (mp_poisson_project*, wall and periodic boundaries) stores the
 * liquid-side velocity on interface faces (the gas side is that plus the
 * jump).  The source sums to the created volume, which an outflow side lets
 * out; without one the operator is singular and the mean of b, the net
 * source included, is removed.  The mass flux stays set across
 * mp_poisson_set_geometry (J is recomputed with it) until cleared.  The
 * first call allocates N f64 on the device; later calls allocate nothing.
 */
mp_status mp_poisson_set_mass_flux(mp_handle hd, const double *mdot_dev);

/* Defines: no paper passage (solver configuration, see mp_opts).
 * Replace the options (stream, precision, method, ...). */
mp_status mp_poisson_set_opts(mp_handle hd, const mp_opts *opts);

/*
 * Defines: the pressure Poisson solve of the projection step
 * (Grid_solvePoisson, Section 3; fractional-step projection, Section 2).
 *
 * Solve A p = b with b = rhs + J - mean, to ||b - A p|| <= tol ||b|| (with an
 * outflow side b = rhs + J keeps its mean and p is not gauged).
 * rhs_dev: device, N f64 (e.g. div u*).  p_dev: device, N f64, in/out
 * (read only if initial_guess = 1), mean-free on exit.  iterations (may be
 * NULL) gets mp_stats.iterations.  res_hist (host, may be NULL) gets up to
 * res_hist_cap true relative residuals: [0] is the initial one, then one
 * per FP64 iteration (FP64 mode) or per reliable update (mixed mode, where
 * the FP32 iterations in between carry only a recurrence estimate);
 * res_hist_len (may be NULL) gets the count written.
 * Returns MP_OK, MP_ERR_NOT_CONVERGED (p holds the last iterate) or an error.
 */
mp_status mp_poisson_solve(mp_handle hd, const double *rhs_dev, double *p_dev, double tol,
                           int *iterations, double *res_hist, int res_hist_cap, int *res_hist_len);

/*
 * Defines: the pressure-projection part of one step of the fractional-step
 * method on the staggered grid (Section 2: velocities on faces, pressure at
 * cell centres; the predicted velocity u* comes from IncompNS_predictor in
 * the Driver_evolveAll listing, Section 3).
 *
 * One projection step on device data: rhs = div_h u*, solve as
 * mp_poisson_solve, then correct the face velocities in place,
 * u = u* - beta (grad_h p - [p]).  ux/uy/uz_dev: device, N f64 each
 * (low-face ownership), in/out.  p_dev as in mp_poisson_solve.
 * The low-face-owned layout stores one boundary face per non-periodic axis
 * (shared by both walls), so this call, mp_poisson_project_step_host,
 * mp_poisson_divergence and mp_poisson_project serve periodic and wall
 * boundaries; with an outflow side they return MP_ERR_INVALID_ARG (form
 * the divergence with your boundary velocities and call mp_poisson_solve;
 * an outflow face's velocity is corrected by -2 beta p_cell / h on a low
 * side, +2 beta p_cell / h on a high side, beta = 1/rho of the cell).
 */
mp_status mp_poisson_project_step(mp_handle hd, double *ux_dev, double *uy_dev, double *uz_dev,
                                  double *p_dev, double tol, int *iterations);

/*
 * Defines: as mp_poisson_project_step (Section 2), for callers whose fields
 * live in host memory.
 *
 * The same step on HOST buffers: copies u* (3N f64) and, for
 * initial_guess = 1, p (N f64) to the device, runs mp_poisson_project_step
 * and copies the corrected velocities and p back.  Uses device staging
 * buffers and a second (copy) stream created at setup: the copies run in
 * z-slabs (whole planes), uploads overlapping the right-hand-side assembly
 * and downloads overlapping the velocity correction; pinned buffers let the
 * copies run asynchronously.  Returns after every copy has completed (also
 * on error).  Same bits as mp_poisson_project_step.
 */
mp_status mp_poisson_project_step_host(mp_handle hd, double *ux_host, double *uy_host,
                                       double *uz_host, double *p_host, double tol,
                                       int *iterations);

/* Defines: the variable-coefficient operator div((1/rho) grad) on the
 * staggered stencil (Section 2; varDens, Section 3), ghost-fluid faces.
 * y = A x (unscaled operator, device N f64 each). */
mp_status mp_poisson_apply(mp_handle hd, const double *x_dev, double *y_dev);

/* Defines: the cell-centred divergence of face velocities on the staggered
 * grid (Section 2).
 * div_dev = div_h u (device, N f64). */
mp_status mp_poisson_divergence(mp_handle hd, const double *ux_dev, const double *uy_dev,
                                const double *uz_dev, double *div_dev);

/* Defines: the right-hand side with the surface-tension jump source
 * (reading: ghost-fluid method, Kang-Fedkiw-Liu 2000; [p] = sigma*kappa,
 * sigma the paper's mph_invWeber, runtime-parameter TOML figure,
 * Section 4), mean-projected for the singular
 * periodic/wall problem.
 * b_dev = rhs + J - mean(rhs + J), the right-hand side the solve uses. */
mp_status mp_poisson_rhs(mp_handle hd, const double *rhs_dev, double *b_dev);

/* Defines: the velocity correction of the fractional-step projection
 * (Section 2), with the pressure jump removed from the gradient on faces
 * that cross the interface (ghost-fluid reading).
 * u -= beta (grad_h p - [p]) on every face, in place. */
mp_status mp_poisson_project(mp_handle hd, const double *p_dev, double *ux_dev, double *uy_dev,
                             double *uz_dev);

/* Defines: the fields derived from phi (curvature and fluid properties,
 * MultiphaseMain and StencilsLevelSet, Section 3; jump source, ghost-fluid
 * reading).
 * Copy setup fields out (device pointers, each N f64; any may be NULL):
 * curvature kappa (evaluated in the interface band -- cells with a face
 * neighbour of the other fluid -- and 0 elsewhere), face coefficients
 * beta_x/y/z (low-face ownership, boundary faces of non-periodic axes 0;
 * an outflow face's coefficient is 1/rho of its cell's fluid), jump
 * source J (unscaled, sums to zero). */
mp_status mp_poisson_get_fields(mp_handle hd, double *kappa_dev, double *bx_dev, double *by_dev,
                                double *bz_dev, double *J_dev);

/* Defines: no paper passage (solver diagnostics).
 * Statistics of the last solve. */
mp_status mp_poisson_get_stats(mp_handle hd, mp_stats *st);

/* Defines: no paper passage; the gas regions phi > 0 (Fig. 2 caption) split
 * into connected components, the deflation vectors of the solve (reading:
 * deflated CG for bubbly flows, Tang & Vuik).
 * Connected gas components of the current geometry (face neighbours, periodic
 * axes wrapped): comp_dev (device, N int32, may be NULL) gets each cell's
 * component id (0..m-1 in the order of each component's lowest cell index,
 * -1 for liquid); m (host) gets the count.  m = 0 when deflation is off for
 * this geometry (no gas, or more than 4096 components). */
mp_status mp_poisson_get_components(mp_handle hd, int *comp_dev, int *m);

/* Per-(kernel, level) launch record, filled by mp_poisson_get_profile. */
typedef struct {
  char name[40];        /* kernel name, e.g. "rbgs_f32" */
  int level;            /* multigrid level (0 = finest) */
  long long cells;      /* cells of that level */
  long long launches;   /* launches since the last mp_poisson_set_profiling */
  double total_ms;      /* summed CUDA-event durations (0 unless profiling is on) */
  double alg_bytes;     /* summed algorithmic bytes: unique bytes each launch must move */
} mp_kernel_prof;

/*
 * Defines: no paper passage (measurement: per-kernel launch counts, event
 * times and algorithmic bytes for the roofline).
 *
 * Launch accounting.  Every kernel launch is counted per (kernel, level).
 * enable = 1 also brackets every launch with CUDA events on the handle's
 * stream (host-side cost ~1 us per launch).  Resets all counters.
 */
mp_status mp_poisson_set_profiling(mp_handle hd, int enable);

/* Defines: no paper passage (measurement, see mp_poisson_set_profiling).
 * Copy up to cap records to out (host memory); *count (may be NULL) gets
 * the number of records available. */
mp_status mp_poisson_get_profile(mp_handle hd, mp_kernel_prof *out, int cap, int *count);

/*
 * Right-hand side without allocating: b = rhs + J - mean(rhs + J), the same
 * result as mp_poisson_rhs (to rounding), for callers that cannot allocate
 * device memory.  The paper has no counterpart; this exists for library
 * users whose host application owns every device allocation (a memory pool
 * or budget they may not bypass), or whose code path must not call
 * cudaMalloc because it can block on or synchronise the device.  It needs
 * no handle: the caller passes ncells (number of cells), rhs_dev and J_dev
 * (device, ncells f64 each; J as returned by mp_poisson_get_fields) and
 * b_dev (device, ncells f64, output).  The call works on the CURRENT device
 * (its scratch and its launches): the three pointers must be memory of that
 * device.
 *
 * Scratch: a fixed array of about 512 KB in device memory that every GPU
 * loading this library holds until the process exits; it bounds ncells to
 * MP_NOALLOC_MAX_CELLS (larger sizes return MP_ERR_INVALID_ARG before any
 * device work).  Every call on a device shares that one array and it keeps
 * the last call's contents (each call writes every slot it later reads, so
 * nothing needs clearing): calls that overlap on the GPU (different
 * streams, or host threads) race and give wrong results.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream
 * capture.  The work is enqueued on `stream` (cudaStream_t, NULL = legacy
 * default stream) and the call returns without waiting for it.  Calls no
 * allocating routine.
 */
#define MP_NOALLOC_MAX_CELLS 134217728LL /* 512^3 */
mp_status mp_poisson_rhs_noalloc(long long ncells, const double *rhs_dev, const double *J_dev,
                                 double *b_dev, void *stream);

/*
 * Defines: no paper passage (the paper has no learned component); the training loss
 * of a learned initial guess for the deflated solver.
 *
 * Deflated CG corrects any start exactly along the gas components' indicator vectors
 * Z, so what it inherits from a guess is the error in the deflated energy
 * ||e||_D^2 = e^T D e with D = A - A Z E^-1 Z^T A, E = Z^T A Z (the A-energy left after
 * the best correction along Z).  For the network output q and the target t (device
 * FP32, N each; t a multiple of the solution) this returns the relative D-energy
 * error of the best multiple of q,
 *   L = 1 - (q.D t)^2 / ((q.D q)(t.D t)),
 * in loss_out (host) and, when gq_dev (device FP32, N) is not NULL, its gradient
 * dL/dq = -2 (q.Dt)/((q.Dq)(t.Dt)) D t + 2 (q.Dt)^2/((q.Dq)^2 (t.Dt)) D q.  A and Z are
 * the current geometry's (FP64).  MP_ERR_INVALID_ARG when the handle has no deflation
 * vectors (deflate off, no gas, or an outflow side); MP_ERR_DIVERGED when q or t has no
 * deflated energy.  Uses the handle's solver scratch (not during a solve).
 */
mp_status mp_poisson_deflated_energy(mp_handle hd, const float *q_dev, const float *t_dev,
                                     float *gq_dev, double *loss_out);

/* Defines: no paper passage (resource release).
 * Free everything the handle owns.  NULL is ignored. */
void mp_poisson_destroy(mp_handle hd);

/* Defines: no paper passage (error reporting).
 * Static text for a status code. */
const char *mp_status_str(mp_status s);

#ifdef __cplusplus
}
#endif

#endif /* MP_POISSON_H */
