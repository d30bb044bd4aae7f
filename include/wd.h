/*
 * wd.h -- C ABI of libwd, a GB300 (sm_103a) implementation of the high-order central
 * difference Hamilton-Jacobi wall-distance method of Kakumani, Vadlamani & Tucker,
 * "On the use of high order central difference schemes for differential equation based
 * wall distance computations" (arXiv 2111.09859).
 *
 * Conventions shared by every entry point
 *  - A grid has n[0] x n[1] x n[2] nodes.  Node (i, j, k) of every caller array sits at
 *    i + n[0] * (j + n[1] * k) (dense, i fastest).  In 2-D, n[2] > 1 stacks n[2]
 *    independent grids of n[0] x n[1] nodes (grid k holds the nodes with that k; same
 *    boundary kinds, own coordinates, masks and convergence norms); they are solved
 *    together by the same launches, and stats report the worst of them.
 *  - "phi" arrays hold the grid's state precision: double for WD_FP64, float for
 *    WD_FP32_METRIC64 and WD_FP32.  Metric exports are always double.
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; *_host are host
 *    pointers read during the call only.  The library owns every internal buffer.
 *  - Each grid owns a non-blocking CUDA stream on which all of its device work runs
 *    (captured into CUDA graphs during solves).  Every call first waits for the work
 *    already queued on the caller's stream (given to wd_create_grid or wd_set_stream) and
 *    makes that stream wait for the call's own work, so the caller's stream stays ordered.
 *    wd_solve, wd_steps, wd_step_unsteady and wd_solve_batch return after the work has
 *    finished; the operator entry points (wd_derivative ... wd_apply_bc) only enqueue.
 *  - Every function returns a wd_status and never aborts.  After WD_ERR_CUDA the CUDA
 *    context may be unusable; after any other error the grid stays valid.
 *    wd_last_error() gives a one-line description of the most recent failure on the
 *    calling thread.
 *  - Calls on one grid must not overlap; distinct grids may be used from distinct threads.
 */
#ifndef WD_H
#define WD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_grid_s* wd_grid;

typedef enum {
    WD_OK = 0,
    WD_ERR_INVALID_ARG = 1,
    WD_ERR_OOM = 2,
    WD_ERR_CUDA = 3,
    WD_ERR_NOT_CONVERGED = 4,
    WD_ERR_DIVERGED = 5,
    WD_ERR_TIMEOUT = 6
} wd_status;

/* boundary kind of each face (Sec. 3.5) */
enum { WD_BC_WALL = 0,      /* Dirichlet phi = 0 on the face (Eq. 22) */
       WD_BC_FARFIELD = 1,  /* linear extrapolation along the grid line, scaled by the
                               local spacing ratio (reading of Eq. 23) */
       WD_BC_NEUMANN = 2,   /* phi copied from the neighbour: d(phi)/dn = 0 (Eq. 23) */
       WD_BC_PERIODIC = 3 };/* both faces of the direction */

/* state / metric precision */
enum { WD_FP64 = 0,          /* everything double */
       WD_FP32_METRIC64 = 1, /* float state, stencils, LAD and line solves; the metric
                                Jacobians (coordinate derivatives and their inverse) are
                                computed in double at creation and rounded to float for the
                                loop; change norms accumulate in double */
       WD_FP32 = 2 };        /* as WD_FP32_METRIC64, but the coordinates are rounded to float
                                and differentiated in float before the (double) inversion */

/* equation (Sec. 2.3) */
enum { WD_HJ_STD = 0,        /* Gamma = eps * phi (Eq. 6) */
       WD_HJ_LAD = 1,        /* Gamma = MIN(eps*phi, LAD term) (Eq. 7) */
       WD_EIKONAL = 2 };     /* Gamma = 0 (Eq. 17) */

/* spatial scheme (Sec. 3.2.2, Eq. 16) */
enum { WD_E2 = 0, WD_E4 = 1, WD_E6 = 2, WD_C4 = 3, WD_C6 = 4,
       WD_UW = 5 };          /* the paper's baseline (Sec. 3.2.1): the advection term U.grad(phi)
                                of the HJ / Eikonal equations by first-order upwinding with the
                                sign-selected slopes of Eqs. UW1-UW5; the metrics, the Laplacian
                                and the Poisson guess by E2.  Runs on the generic per-operator
                                path, so on single grids only (a stack of 2-D grids with WD_UW
                                is WD_ERR_INVALID_ARG); wd_default_params turns the filter off
                                for it. */

/* initial guess */
enum { WD_INIT_ZERO = 0,     /* phi = 0 (Sec. 3.5) */
       WD_INIT_POISSON = 1,  /* Poisson pseudo steps + Spalding equation (Eqs. 3-4, 19) */
       WD_INIT_GIVEN = 2 };  /* the caller's phi_dev contents (warm start) */

typedef struct {
    int ndim;              /* 2 or 3 */
    int n[3];              /* nodes per direction, each >= 8 for d < ndim; in 2-D n[2] is the
                              number of stacked grids (1 for a single grid; > 1 needs
                              periodic or wall faces in direction 0) */
    int bc_lo[3];          /* WD_BC_* of the face at index 0 of each direction */
    int bc_hi[3];          /* WD_BC_* of the face at index n-1 of each direction */
    double period[3][3];   /* periodic direction d: x(i + n[d]) = x(i) + period[d] */
    int precision;         /* WD_FP64 / WD_FP32_METRIC64 / WD_FP32 */
    int scheme;            /* WD_E2 .. WD_C6: every derivative and the metrics (Sec. 3.2.2);
                              WD_UW: the baseline upwind scheme */
    double L_ref;          /* reference length of the convergence norms (Eq. 20) */
} wd_grid_desc;

typedef struct {
    int equation;          /* WD_HJ_STD / WD_HJ_LAD / WD_EIKONAL */
    int curvature;         /* 1: Nakanishi correction, Sec. 5.4 / Eq. 25 */
    double eps;            /* epsilon of Eqs. 6, 7, 25 */
    double C_lad;          /* C of Eq. 7 */
    double lad_exp;        /* exponent of Delta x_l in Eq. 7 (the paper prints 3) */
    double alpha_f;        /* filter coefficient of Eq. 21, |alpha_f| < 0.5 */
    int filter;            /* 1: filter along every direction after each pseudo step */
    double cfl;            /* local pseudo time step factor */
    double eps0;           /* epsilon_0 of the unit normal in Eq. 25 */
    double tol_l2;         /* stop when RMS(phi_new - phi_old)/L_ref <= tol_l2 (<= 0: off) */
    double tol_linf;       /* stop when max|phi_new - phi_old|/L_ref <= tol_linf, Eq. 20 */
    int max_iters;         /* HJ pseudo steps at most */
    int check_every;       /* pseudo steps between convergence checks (host reads) */
    int init;              /* WD_INIT_* */
    double poisson_tol;    /* Poisson stop on RMS(dphi')/L_ref^2 (<= 0: run poisson_max_iters) */
    int poisson_max_iters; /* Poisson pseudo steps at most */
} wd_solve_params;

typedef struct {
    int iters;             /* HJ pseudo steps taken */
    int poisson_iters;     /* Poisson pseudo steps taken */
    double res_l2;         /* RMS change of the last step / L_ref */
    double res_linf;       /* max change of the last step / L_ref */
    int converged;         /* tolerance met */
    int diverged;          /* NaN / Inf met */
    int stalled;           /* FP32 state only: stopped because the change norm stopped
                              decreasing (rounding floor) before reaching the tolerance;
                              converged is set too */
    double seconds;        /* wall time of the call */
    size_t device_bytes;   /* library-owned device memory of the grid */
} wd_stats;

/* Fills *p with the defaults used by the tests and the benchmark: LAD HJ, eps 0.2,
 * C 0.1, exponent 3, alpha_f 0.49, filter on, cfl 0.8 (explicit) / 0.6 (compact) for the
 * given scheme, eps0 1e-8, tol_l2 1e-10, 100 Poisson steps. */
void wd_default_params(int scheme, wd_solve_params* p);

/* Creates a grid (Sec. 3.1): uploads the node coordinates xyz_host (ndim x N doubles:
 * all x, then all y, then all z), computes the metrics on the GPU with the grid's scheme,
 * marks wall faces and the optional Dirichlet nodes (mask_host[p] != 0, values
 * dval_host[p], NULL -> 0) and precomputes the line-solve tables.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).
 * Errors: WD_ERR_INVALID_ARG (bad sizes or boundary kinds, non-positive L_ref),
 * WD_ERR_OOM, WD_ERR_CUDA. */
wd_status wd_create_grid(const wd_grid_desc* desc, const double* xyz_host,
                         const uint8_t* mask_host, const double* dval_host,
                         void* cuda_stream, wd_grid* out);

/* Frees every device buffer of the grid (NULL is ignored); no counterpart in the paper. */
void wd_destroy_grid(wd_grid g);

/* Changes the stream used by later calls on g. */
wd_status wd_set_stream(wd_grid g, void* cuda_stream);

/* Steady solve (Sec. 3.3): initial guess, then HJ pseudo-time marching (RK4 with local
 * time steps, boundary conditions after every stage, filter after every step) until the
 * tolerances hold, max_iters is reached, or a NaN appears.  With a float state the march
 * also stops once the RMS change has not fallen below 0.95 x its best value for 200
 * pseudo steps (the float rounding floor; stats->stalled = 1).  phi_dev (N values of the
 * state precision, dense layout) is read when init == WD_INIT_GIVEN and always receives
 * the result.  Returns WD_OK when converged or when no tolerance was set,
 * WD_ERR_NOT_CONVERGED after max_iters with a tolerance set, WD_ERR_DIVERGED on NaN/Inf. */
wd_status wd_solve(wd_grid g, const wd_solve_params* p, void* phi_dev, wd_stats* stats);

/* Unsteady re-solve (Sec. 3.3, last paragraph; Sec. 5.5): replaces the Dirichlet set by
 * mask_dev / dval_dev (device arrays of N uint8 and N state-precision values; wall faces
 * stay Dirichlet 0; NULL keeps the current set) and marches from the previous solution in
 * phi_dev (warm start, init ignored).  Same return values as wd_solve. */
wd_status wd_step_unsteady(wd_grid g, const uint8_t* mask_dev, const void* dval_dev,
                           const wd_solve_params* p, void* phi_dev, wd_stats* stats);

/* Steady solves of Sec. 3.3 (as wd_solve) of n independent grids of any shapes with the same
 * parameters; phi_dev[i] and stats[i] belong to grids[i].  The solves run as interleaved
 * resumable tasks on the grids' own streams: each round queues one slice of check_every
 * pseudo steps of every unfinished solve before waiting for any, so the slices of all grids
 * run side by side on the GPU.  Each grid gets bit for bit what wd_solve gives it alone.
 * stats[i].seconds is the wall time of the whole batch.  Returns the first non-OK status in
 * grid order (every grid is still solved).  Errors: WD_ERR_INVALID_ARG for n < 0, NULL
 * arrays, a NULL grid or phi, or a grid listed twice. */
wd_status wd_solve_batch(wd_grid* grids, int n, const wd_solve_params* p, void** phi_dev,
                         wd_stats* stats);

/* Device bytes wd_create_grid would allocate for desc (0 if desc is invalid): the node
 * coordinates and the metric arrays of Sec. 3.1, the RK4 and pseudo-time work fields of
 * Sec. 3.3, the line-solve tables of Eqs. 16 and 21 (the allocation itself has no
 * counterpart in the paper).  The request loop admits requests by this footprint. */
size_t wd_query_footprint(const wd_grid_desc* desc, const wd_solve_params* p);

/* Name of a status code, and a one-line description of the calling thread's most recent
 * failure (no counterpart in the paper). */
const char* wd_status_string(wd_status s);
const char* wd_last_error(void);

/* ---- operator entry points: one step of the method each, for parity testing ---------- */

/* Metrics of Sec. 3.1 (a1): xi_dev[(l*3+m)*N + p] = d(xi_l)/d(x_m), J_dev[p] = det of
 * dx_m/dxi_l, dx_dev[l*N + p] = |dx/dxi_l| (double, dense; unused entries are 0). */
wd_status wd_get_metrics(wd_grid g, double* xi_dev, double* J_dev, double* dx_dev);

/* First derivative along direction dir with unit computational spacing (Eq. 16 and its
 * boundary rows), in the grid's scheme and state precision (a4). */
wd_status wd_derivative(wd_grid g, int dir, const void* in_dev, void* out_dev);

/* One implicit filter pass along dir (Eq. 21), order reduced to 2 near non-periodic ends,
 * end nodes unfiltered (a10).  in_dev may equal out_dev. */
wd_status wd_filter(wd_grid g, double alpha_f, int dir, const void* in_dev, void* out_dev);

/* Right-hand side R with d(phi)/dt* = R and the local pseudo time step (a5-a9):
 * kind 0 = HJ (Eqs. 5-7, 9, 25), kind 1 = Poisson (Eq. 19). */
wd_status wd_rhs(wd_grid g, const wd_solve_params* p, int kind, const void* phi_dev,
                 void* R_dev, void* dt_dev);

/* Spalding auxiliary equation (Eq. 4, minus root): phi' -> phi (a3). */
wd_status wd_spalding(wd_grid g, const void* phip_dev, void* phi_dev);

/* HJ boundary conditions in place: far-field / Neumann faces direction by direction,
 * then every Dirichlet node (a2). */
wd_status wd_apply_bc(wd_grid g, void* phi_dev);

/* Exactly nsteps pseudo steps (RK4 + BCs + filter + change norms) from phi_dev in place:
 * kind 0 = HJ, kind 1 = Poisson (a9-a11).  stats gets the last step's norms. */
wd_status wd_steps(wd_grid g, const wd_solve_params* p, int kind, void* phi_dev, int nsteps,
                   wd_stats* stats);

/* ---- instrumentation (no counterpart in the paper) ---------------------------------- */

/* kernel classes timed by wd_profile */
enum { WD_K_DERIV = 0,   /* first derivatives of phi along one direction */
       WD_K_DIV = 1,     /* metric-weighted divergence pass (Laplacian / curvature) */
       WD_K_FILTER = 2,  /* implicit filter pass */
       WD_K_GAUSS = 3,   /* Gaussian smoothing pass of the LAD diffusivity */
       WD_K_POINT = 4,   /* pointwise kernels: chain rule, LAD term, RK stage, Spalding */
       WD_K_BC = 5,      /* boundary conditions */
       WD_K_NORM = 6,    /* change norms + commit */
       WD_K_LINE0 = 7,   /* line-resident 2-D step: direction-0 pass of an RK stage */
       WD_K_LINE1 = 8,   /* line-resident 2-D step: direction-1 pass of an RK stage (with the
                            stage update) */
       WD_K_NCLASS = 9 };

/* enable != 0 clears the counters and brackets every later kernel launch on g with CUDA
 * events on g's stream (this adds a small gap between launches); enable == 0 stops. */
wd_status wd_profile(wd_grid g, int enable);

/* Total device time (ms, from the events) and launch count of kernel class cls since
 * profiling was enabled; synchronises the stream. */
wd_status wd_profile_read(wd_grid g, int cls, double* ms_total, long long* launches);

/* ---- allocation-free variant (no counterpart in the paper) ---------------------------- */

/* Change norms of two state arrays with no device allocation at all.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device memory,
 * e.g. an application whose own memory pool has already taken the device memory (a
 * cudaMalloc would fail or evict its pool), or a real-time loop that must not call the
 * allocator (cudaMalloc / cudaFree can synchronise the device and stall every stream).
 * It computes what the solver's convergence check computes: over the n entries whose
 * mask_dev byte is 0 (mask_dev NULL: all entries), norms_dev[0] = RMS(new - old) / scale
 * and norms_dev[1] = max|new - old| / scale, accumulated in double in a fixed order.
 *   new_dev, old_dev  device arrays of n values: double for WD_FP64, float otherwise
 *   mask_dev          device array of n bytes, or NULL
 *   norms_dev         caller-owned device array of 2 doubles (written)
 *   cuda_stream       cudaStream_t the work is enqueued on (the call does not wait)
 * All arrays must be on the current device.  Scratch: one library-owned file-scope device
 * array of about 25 KB per GPU that loads the library, held until the process exits; no
 * cudaMalloc / cudaFree ever runs.  The first call on a device looks up that array's
 * device address and keeps it for the process, so do not call this entry point on a device
 * after cudaDeviceReset.  Every call shares the array and clears its arrival counter
 * first: calls whose kernels overlap on the GPU (different streams without ordering) race
 * and give wrong norms.
 * Errors: WD_ERR_INVALID_ARG for NULL arrays, n outside [1, 2^30] (the maximum size),
 * a bad precision or scale <= 0; WD_ERR_CUDA if the launch fails. */
wd_status wd_change_norms_noalloc(const void* new_dev, const void* old_dev,
                                  const uint8_t* mask_dev, long long n, int precision,
                                  double scale, double* norms_dev, void* cuda_stream);

/* Launch shapes chosen by the autotuner for this grid (0: not tuned, the default shape):
 * the block size of the pointwise stage kernel of the fused 2-D path, the block rows of the
 * Cartesian stencil kernels, and the number of parts (1, 2 or 4) a stack of 2-D grids on the
 * line-resident path is split into, each part's launches running on its own stream so that
 * they fill each other's last waves.  Before a grid's first pseudo step the library times the
 * candidates (128 / 256 / 512 threads; 4 / 8 / 16 rows of 32; 1 / 2 / 4 parts) on the grid's
 * own arrays and keeps the fastest, cached per grid shape for the process; none of them
 * changes any result.  The environment variable WD_AUTOTUNE=0 disables it.  Any pointer may
 * be NULL.  Errors: WD_ERR_INVALID_ARG for a NULL grid. */
wd_status wd_get_tuning(wd_grid g, int* stage_threads, int* stencil_rows, int* batch_parts);

/* ---- geometry reuse ---------------------------------------------------------------- */

/* Replaces the coordinates and the caller Dirichlet set of an existing grid without any
 * device allocation: same descriptor, new xyz_host / mask_host / dval_host (as for
 * wd_create_grid).  Recomputes the metrics (Sec. 3.1), the LAD scales and the far-field
 * spacing ratios on the grid's stream.  Temporary device memory comes from the CUDA
 * stream-ordered allocator, so the call never waits for work on other streams.
 * Errors: WD_ERR_INVALID_ARG for a NULL grid or xyz_host; WD_ERR_OOM; WD_ERR_CUDA. */
wd_status wd_reset_geometry(wd_grid g, const double* xyz_host, const uint8_t* mask_host,
                            const double* dval_host);

/* ---- receding surface (Sec. 5.5) ------------------------------------------------------ */

/* Surface receding by s (the unsteady re-solve, Sec. 5.5).  For every node q of the dense
 * field phi_dev (n[0]*n[1]*n[2] values of the grid's state precision, updated in place):
 * phi_dev[q] -= s (the distance to the receded surface where phi was the distance to the
 * old one, and the warm start of the next solve); mask_dev[q] = 1 where the new
 * phi_dev[q] <= 0 (burned; nodes already solid hold phi <= 0 and stay solid), else 0; and
 * dval_dev[q] = max(phi_dev[q], floor) where the mask is set, else 0.  Pass mask, dval and
 * phi to wd_step_unsteady (or wd_server_submit_grid with warm = 1).  All arrays are
 * caller-owned device memory; the work is enqueued on the grid's stream.
 * Errors: WD_ERR_INVALID_ARG for NULL arrays, s < 0 or floor > 0. */
wd_status wd_recede(wd_grid g, void* phi_dev, double s, double floor, uint8_t* mask_dev,
                    void* dval_dev);

/* Grain regression (Sec. 5.5, Eq. levelset with right-hand side 0): nsteps steps of
 * d(phi)/dt + F |grad phi| = 0 by classical RK4 with the global time step dt, on the dense
 * field phi_dev (n[0]*n[1]*n[2] values of the grid's state precision, updated in place; 2-D,
 * stacked 2-D or 3-D).  |grad phi| = |sum_l grad(xi_l) s_l| with s_l the upwind slopes of
 * Eqs. UW3-UW5 (of -phi when F < 0, so that the front always takes its upwind side); the
 * front {phi = 0} moves along grad(phi) at speed F.  Every non-periodic face holds a zero
 * normal gradient (the face node copies its neighbour after every stage); Dirichlet nodes
 * and the grid's wall faces are not held.  Stable for dt * |F| * sum_l |grad xi_l| below about
 * 1.4 (RK4 on first-order upwinding); the caller picks dt.  Synchronous.
 * Errors: WD_ERR_INVALID_ARG for NULL phi_dev, nsteps < 0, dt <= 0 or non-finite F / dt. */
wd_status wd_levelset(wd_grid g, void* phi_dev, double F, double dt, int nsteps);

/* Length of the level set {phi = level} of a single 2-D grid (the burning perimeter when
 * phi is the wall distance and level = 0 or the burned depth): marching squares over every
 * cell, with the crossings interpolated linearly along the cell edges in physical
 * coordinates, ambiguous cells resolved by the mean of the four corners, lengths summed in
 * double in a fixed order.  phi_dev: dense device field of the grid's precision.
 * Synchronous; *length receives the sum.  Errors: WD_ERR_INVALID_ARG for a 3-D or stacked
 * grid or NULL pointers. */
wd_status wd_level_length(wd_grid g, const void* phi_dev, double level, double* length);

/* ---- request loop (continuous batching of independent solves) ---------------------- */

/* A server owns one scheduler thread on the current device.  Submitted requests wait in
 * a FIFO queue and are admitted while the sum of the device footprints of the admitted
 * requests (wd_query_footprint) stays within max_device_bytes and at most max_active run
 * at once.  Every admitted request runs the solve of wd_solve as a resumable task on its
 * grid's own stream, one slice of check_every pseudo steps (a CUDA graph) at a time, so
 * the slices of all admitted requests overlap on the GPU; a request that arrives while
 * others run is admitted as soon as memory and a slot are free, and finished requests
 * free theirs at once.  Each request gives the same result as wd_solve alone (the same
 * kernels, the same slicing and the same convergence checks).  Grids the server creates
 * are kept per shape for reuse (wd_reset_geometry), within the same memory cap. */
typedef struct wd_server_s* wd_server;

typedef struct {
    size_t max_device_bytes;   /* admission cap; 0 = 80% of the free device memory at creation */
    int max_active;            /* requests running at once; 0 = 32 */
    int pool_per_shape;        /* idle grids kept per shape; 0 = 2, < 0 = none */
} wd_server_config;

/* Errors: WD_ERR_INVALID_ARG for NULL out or negative limits; WD_ERR_CUDA. */
wd_status wd_server_create(const wd_server_config* cfg, wd_server* out);

/* New request on a grid the server creates from desc, xyz_host, mask_host, dval_host (the
 * arguments of wd_create_grid; copied before the call returns).  phi receives the
 * wall distance: n[0]*n[1]*n[2] values of the grid's state precision, in device memory or
 * page-locked host memory, owned by the caller and left untouched until the request is
 * done; with p->init == WD_INIT_GIVEN it also holds the initial state.  *ticket
 * identifies the request.
 * Errors: WD_ERR_INVALID_ARG (bad descriptor or parameters, NULL pointers);
 * WD_ERR_OOM when the request alone is larger than max_device_bytes. */
wd_status wd_server_submit(wd_server s, const wd_grid_desc* desc, const double* xyz_host,
                           const uint8_t* mask_host, const double* dval_host,
                           const wd_solve_params* p, void* phi, long long* ticket);

/* New request on a grid the caller owns (a session that keeps its state on the device
 * across requests, e.g. the receding-surface re-solves of wd_step_unsteady).  mask_dev /
 * dval_dev (or NULL) update the Dirichlet set first as in wd_step_unsteady; warm != 0
 * starts from phi.  The request is ordered after the work queued on the grid's stream
 * (wd_set_stream) at the time of the call; the grid must not be used by the caller until
 * the request is done.  Its footprint counts against the cap while it runs. */
wd_status wd_server_submit_grid(wd_server s, wd_grid g, const uint8_t* mask_dev,
                                const void* dval_dev, int warm, const wd_solve_params* p,
                                void* phi, long long* ticket);

/* Waits up to timeout_s seconds (< 0: no limit) for the request.  On completion fills
 * *stats, *latency_s (submission to completion, host clock) and returns the request's
 * own status (WD_OK, WD_ERR_NOT_CONVERGED, ...), and the ticket is released.
 * Returns WD_ERR_TIMEOUT if the request is still queued or running (the ticket stays
 * valid), WD_ERR_INVALID_ARG for an unknown ticket. */
wd_status wd_server_wait(wd_server s, long long ticket, double timeout_s, wd_stats* stats,
                         double* latency_s);

/* Counters since creation: requests queued, running, done; device bytes admitted now;
 * peak number of requests running at once. */
wd_status wd_server_info(wd_server s, long long* queued, long long* running, long long* done,
                         size_t* admitted_bytes, long long* peak_running);

/* Finishes every submitted request, stops the thread and frees every server-owned grid. */
void wd_server_destroy(wd_server s);

#ifdef __cplusplus
}
#endif
#endif
