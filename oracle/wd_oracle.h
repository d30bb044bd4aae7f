/*
 * wd_oracle.h -- plain, slow, FP64 CPU oracle for the Hamilton-Jacobi wall-distance
 * method of Kakumani, Vadlamani & Tucker, "On the use of high order central difference
 * schemes for differential equation based wall distance computations" (arXiv 2111.09859).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library.  It shares no source, header,
 * table or helper with the CUDA path; the two meet only through seeded inputs.
 *
 * Everything is double precision, single threaded, written as plain loops in the order
 * of the paper: grid metrics (Sec. 3.1), central derivatives E2/E4/E6/C4/C6 (Sec. 3.2.2,
 * Eq. 16), HJ residual with standard / LAD Gamma (Eqs. 5-7, 9) and the Nakanishi
 * curvature correction (Sec. 5.4, Eq. 25), pseudo-time RK4 with local time stepping
 * (Sec. 3.3, Eqs. 18-19), the implicit filter (Sec. 3.4, Eq. 21), boundary conditions
 * (Sec. 3.5, Eqs. 22-23) and the convergence norms (Sec. 3.3, Eq. 20).
 *
 * Node (i,j,k) of a grid with n[0] x n[1] x n[2] nodes sits at i + n[0]*(j + n[1]*k).
 */
#ifndef WD_ORACLE_H
#define WD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* boundary kinds per face */
#define OR_BC_WALL      0  /* Dirichlet phi = 0 (Eq. 22) */
#define OR_BC_FARFIELD  1  /* linear extrapolation along the grid line (reading of Eq. 23) */
#define OR_BC_NEUMANN   2  /* d(phi)/dn = 0 by copying the neighbour (Eq. 23 literally) */
#define OR_BC_PERIODIC  3  /* both faces of a direction must be periodic */

/* spatial schemes (Sec. 3.2.2) */
#define OR_E2 0
#define OR_E4 1
#define OR_E6 2
#define OR_C4 3
#define OR_C6 4
#define OR_UW 5   /* baseline: upwind advection term (Eqs. UW1-UW5), E2 for the metrics
                     and the Laplacian (Sec. 3.2.1) */

/* equations */
#define OR_HJ_STD  0   /* Gamma = eps*phi, Eq. 6 */
#define OR_HJ_LAD  1   /* Gamma = MIN(eps*phi, LAD), Eq. 7 */
#define OR_EIKONAL 2   /* Gamma = 0, Eq. 17 */

/* initial guess */
#define OR_INIT_ZERO    0  /* phi = 0 (Sec. 3.5) */
#define OR_INIT_POISSON 1  /* Poisson + Spalding auxiliary equation (Eqs. 3-4, 10, 19) */
#define OR_INIT_GIVEN   2  /* caller's phi (warm start, Sec. 3.3 unsteady procedure) */

typedef struct {
    int ndim;          /* 2 or 3 */
    int n[3];          /* nodes per direction; n[2] = 1 when ndim = 2 */
    int bc_lo[3];      /* OR_BC_* for the face at index 0 of each direction */
    int bc_hi[3];      /* OR_BC_* for the face at index n-1 of each direction */
    double period[3][3]; /* periodic direction d: x(i + n) = x(i) + period[d] */
    double L_ref;      /* reference length used by the convergence norms (Eq. 20) */
} or_grid_desc;

typedef struct {
    int equation;      /* OR_HJ_STD / OR_HJ_LAD / OR_EIKONAL */
    int scheme;        /* OR_E2 .. OR_C6, used for every derivative and the metrics */
    int curvature;     /* 1: Nakanishi correction, Eq. 25 */
    double eps;        /* epsilon of Eqs. 6-7 and 25 */
    double C_lad;      /* C of Eq. 7 */
    double lad_exp;    /* exponent of Delta x_l in Eq. 7 (printed as 3) */
    double alpha_f;    /* filter coefficient, Eq. 21 */
    int filter;        /* 1: filter after every pseudo step */
    double cfl;        /* local pseudo time step factor */
    double eps0;       /* epsilon_0 of the unit normal in Eq. 25 */
    double tol_l2;     /* stop when RMS(dphi)/L_ref <= tol_l2 (<=0: unused) */
    double tol_linf;   /* stop when max|dphi|/L_ref <= tol_linf, Eq. 20 (<=0: unused) */
    int max_iters;
    int check_every;
    int init;          /* OR_INIT_* */
    double poisson_tol;   /* RMS(dphi')/L_ref^2 stop for the Poisson guess (<=0: unused) */
    int poisson_max_iters;
} or_params;

typedef struct {
    int iters;              /* HJ pseudo steps taken */
    int poisson_iters;      /* Poisson pseudo steps taken */
    double res_l2;          /* RMS of the last step's change / L_ref */
    double res_linf;        /* max of the last step's change / L_ref */
    int converged;          /* 1 if the tolerance was met */
    int diverged;           /* 1 if a NaN / Inf appeared */
} or_stats;

typedef struct or_ctx_s or_ctx;

/* Builds the context: copies coordinates (3 x N, x then y then z; z ignored in 2D),
 * computes the metrics with `scheme` (Sec. 3.2.2: metrics use the same schemes),
 * marks wall faces and `mask` nodes as Dirichlet with values `dval` (NULL -> 0).
 * Returns NULL on invalid input. */
or_ctx* or_create(const or_grid_desc* desc, const double* xyz, int scheme,
                  const unsigned char* mask, const double* dval);
void or_destroy(or_ctx* c);

/* Replaces the Dirichlet set (immersed / receding walls); wall faces stay Dirichlet 0. */
void or_set_dirichlet(or_ctx* c, const unsigned char* mask, const double* dval);

/* Metric export: xi[(l*3+m)*N + p] = d(xi_l)/d(x_m) at node p; J[p]; dx[l*N+p] = |dx/dxi_l|. */
void or_get_metrics(const or_ctx* c, double* xi, double* J, double* dx);

/* One directional first derivative with unit computational spacing (Eq. 16). */
void or_deriv(const or_ctx* c, int scheme, int dir, const double* in, double* out);

/* One directional implicit filter pass (Eq. 21), boundary order reduced to 2 (Sec. 3.4). */
void or_filter(const or_ctx* c, double alpha_f, int dir, const double* in, double* out);

/* HJ right-hand side R (so that d(phi)/dt* = R) and the local pseudo time step. */
void or_rhs_hj(const or_ctx* c, const or_params* p, const double* phi, double* R, double* dt);

/* Poisson right-hand side R = 1 + lap(phi') and its local pseudo time step (Eq. 19). */
void or_rhs_poisson(const or_ctx* c, const or_params* p, const double* phi, double* R, double* dt);

/* Spalding auxiliary equation, Eq. 4 with the minus root: phi' -> phi. */
void or_spalding(const or_ctx* c, const or_params* p, const double* phip, double* phi);

/* Applies the HJ boundary conditions in place (far field faces, then Dirichlet nodes). */
void or_apply_bc(const or_ctx* c, double* phi);

/* Runs exactly n HJ pseudo steps (RK4 + BCs + filter) from phi in place. */
void or_hj_steps(const or_ctx* c, const or_params* p, double* phi, int n, or_stats* st);

/* Runs exactly n Poisson pseudo steps from phi' in place. */
void or_poisson_steps(const or_ctx* c, const or_params* p, double* phip, int n, or_stats* st);

/* Full solve: initial guess, HJ pseudo-time marching to the tolerance. Returns 0 when
 * converged, 1 when max_iters was reached, 2 on divergence. */
int or_solve(const or_ctx* c, const or_params* p, double* phi, or_stats* st);

/* Advection term of the baseline upwind scheme (Sec. 3.2.1, Eqs. UW1-UW5):
 * adv = sum_l [0.5 (Uh_l + |Uh_l|) B_l + 0.5 (Uh_l - |Uh_l|) F_l] with Uh_l the contravariant
 * component of grad(phi) built from the upwind slopes. */
void or_upwind_advection(const or_ctx* c, const double* phi, double* adv);

/* Upwind slope of Eqs. UW3-UW5 from the backward and forward differences B and F. */
double or_upwind_slope(double B, double F);

/* |grad phi| of the level-set equation (Eq. levelset) from the upwind slopes, for a front
 * moving at normal speed F (the selection is mirrored for F < 0). */
void or_levelset_gradmag(const or_ctx* c, double F, const double* phi, double* gm);

/* n steps of the level-set equation d(phi)/dt + F |grad phi| = 0 (Sec. 5.5) by classical RK4
 * with the global time step dt; zero normal gradient on every non-periodic face after each
 * stage.  Dirichlet nodes are not held. */
void or_levelset_steps(const or_ctx* c, double F, double dt, double* phi, int n);

/* Dense-free tridiagonal helpers exported for pinning: rows a_i x_{i-1} + b_i x_i +
 * c_i x_{i+1} = d_i.  cyclic != 0 couples a_0 to x_{n-1} and c_{n-1} to x_0. */
void or_tridiag(int n, int cyclic, const double* a, const double* b, const double* c,
                const double* d, double* x);

/* Filter coefficients a_0..a_hw of the centred filter of order 2*hw (Sec. 3.4). */
void or_filter_coeffs(int hw, double alpha_f, double* a);

#ifdef __cplusplus
}
#endif
#endif
