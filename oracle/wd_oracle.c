/*
 * wd_oracle.c -- plain FP64 CPU oracle of the HJ / LAD pseudo-HJ wall-distance method
 * (Kakumani, Vadlamani & Tucker, arXiv 2111.09859).  TEST INFRASTRUCTURE ONLY: it is
 * loaded by tests/, __graft_entry__.smoke() and bench.py's CPU baseline, never by the
 * product path.  Slow on purpose: every directional operator gathers one grid line,
 * applies a 1D formula written out term by term, and scatters it back; every
 * tridiagonal system is solved by the Thomas algorithm (cyclic systems by the
 * Sherman-Morrison identity).  No blocking, fusion or reordering beyond the paper's
 * sequence.
 *
 * Parity pins (tests/test_oracle_*.py): polynomial exactness and modified wavenumbers of
 * the derivatives, the filter transfer function, dense solves of the tridiagonal systems,
 * analytic metrics of polar grids, the 1D Spalding identity, the exact linear fixed point,
 * closed-form distances and brute force; for the baseline upwind scheme and the level-set
 * march, Godunov's numerical Hamiltonian, linear fields on sheared grids, the exact channel
 * distance, first-order convergence rates and the exact front speed.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "wd_oracle.h"

struct or_ctx_s {
    or_grid_desc g;
    int N;                 /* total nodes */
    int scheme;            /* scheme the metrics were computed with */
    double* xyz;           /* 3N coordinates */
    double* xi;            /* 9N: xi[(l*3+m)*N+p] = d(xi_l)/d(x_m) */
    double* J;             /* N: det(dx_m/dxi_l) */
    double* dx;            /* 3N: |dx/dxi_l| */
    double* ff_ratio;      /* 6N: far-field spacing ratio, face (d,side) at [(2d+side)N + p] */
    unsigned char* dmask;  /* N: 1 = Dirichlet node */
    double* dval;          /* N: Dirichlet value */
};

/* ------------------------------------------------------------------------------------ */
/* indexing                                                                             */
/* ------------------------------------------------------------------------------------ */

static int node_index(const or_grid_desc* g, const int c[3])
{
    return c[0] + g->n[0] * (c[1] + g->n[1] * c[2]);
}

static int line_count(const or_ctx* C, int dir) { return C->N / C->g.n[dir]; }

/* Node indices of line q along direction dir (q enumerates the other two coordinates). */
static void line_nodes(const or_grid_desc* g, int dir, int q, int* ids)
{
    int o1 = (dir + 1) % 3, o2 = (dir + 2) % 3;
    int c[3];
    c[o1] = q % g->n[o1];
    c[o2] = q / g->n[o1];
    for (int t = 0; t < g->n[dir]; t++) {
        c[dir] = t;
        ids[t] = node_index(g, c);
    }
}

static int is_periodic(const or_grid_desc* g, int dir)
{
    return g->bc_lo[dir] == OR_BC_PERIODIC;
}

/* wrap index t into [0, n) for periodic lines */
static int wrap(int t, int n)
{
    int r = t % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------------------------ */
/* tridiagonal solvers                                                                  */
/* ------------------------------------------------------------------------------------ */

/* Thomas algorithm for a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i (a_0, c_{n-1} ignored). */
static void thomas(int n, const double* a, const double* b, const double* c,
                   const double* d, double* x)
{
    double* cp = (double*)malloc(sizeof(double) * n);
    double* dp = (double*)malloc(sizeof(double) * n);
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int i = 1; i < n; i++) {
        double m = b[i] - a[i] * cp[i - 1];
        cp[i] = (i < n - 1) ? c[i] / m : 0.0;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
}

/* Cyclic tridiagonal system: row 0 carries a_0 on x_{n-1}, row n-1 carries c_{n-1} on x_0.
 * Sherman-Morrison: A = B + u v^T with u = (g,0,..,0,c_{n-1}), v = (1,0,..,0,a_0/g),
 * so B differs from A only in its two corner diagonal entries. */
static void cyclic_solve(int n, const double* a, const double* b, const double* c,
                         const double* d, double* x)
{
    double g = -b[0];
    double* bb = (double*)malloc(sizeof(double) * n);
    double* u = (double*)calloc(n, sizeof(double));
    double* z = (double*)malloc(sizeof(double) * n);
    memcpy(bb, b, sizeof(double) * n);
    bb[0] = b[0] - g;
    bb[n - 1] = b[n - 1] - a[0] * c[n - 1] / g;
    thomas(n, a, bb, c, d, x);
    u[0] = g;
    u[n - 1] = c[n - 1];
    thomas(n, a, bb, c, u, z);
    double vy = x[0] + a[0] * x[n - 1] / g;
    double vz = z[0] + a[0] * z[n - 1] / g;
    double f = vy / (1.0 + vz);
    for (int i = 0; i < n; i++) x[i] -= f * z[i];
    free(bb);
    free(u);
    free(z);
}

void or_tridiag(int n, int cyclic, const double* a, const double* b, const double* c,
                const double* d, double* x)
{
    if (cyclic) cyclic_solve(n, a, b, c, d, x);
    else thomas(n, a, b, c, d, x);
}

/* ------------------------------------------------------------------------------------ */
/* 1D first derivatives, unit computational spacing (Sec. 3.2.2, Eq. 16)                */
/*   alpha f'_{i-1} + f'_i + alpha f'_{i+1} = b (f_{i+2}-f_{i-2})/4 + a (f_{i+1}-f_{i-1})/2 */
/*   E2: a=1.  E4: a=4/3, b=-1/3.  E6: the 7-point textbook stencil (45,-9,1)/60.        */
/*   C4: alpha=1/4, a=3/2.  C6: alpha=1/3, a=14/9, b=1/9.                                 */
/* Boundary rows (the paper defers them to its Ref. [visbal]; reading used here):        */
/*   node 0:  explicit one-sided (-25,48,-36,16,-3)/12 (4th order);                      */
/*   node 1:  explicit centred (f_2 - f_0)/2 (2nd order);                                 */
/*   node >= 2: the scheme's centred row, except that E6 uses E4 at node 2.              */
/*   The right end mirrors the left with a sign change.  A biased 4th-order row at node 1 */
/*   (or a compact row coupled to a one-sided node-0 row) gives the linearised pseudo-   */
/*   step eigenvalues with positive real part at concave wall corners; the centred      */
/*   node-1 row does not.                                                                */
/* ------------------------------------------------------------------------------------ */

/* f at index t of a line of length n; periodic lines wrap */
#define F(t) (f[periodic ? wrap((t), n) : (t)])

static double e2_int(const double* f, int i, int n, int periodic)
{
    return 0.5 * (F(i + 1) - F(i - 1));
}
static double e4_int(const double* f, int i, int n, int periodic)
{
    return (2.0 / 3.0) * (F(i + 1) - F(i - 1)) - (1.0 / 12.0) * (F(i + 2) - F(i - 2));
}
static double e6_int(const double* f, int i, int n, int periodic)
{
    return 0.75 * (F(i + 1) - F(i - 1)) - 0.15 * (F(i + 2) - F(i - 2))
         + (1.0 / 60.0) * (F(i + 3) - F(i - 3));
}
#undef F

/* one-sided 4th-order row at the left end; the right end uses reversed f and a minus */
static double clos0_4(double f0, double f1, double f2, double f3, double f4)
{
    return (-25.0 * f0 + 48.0 * f1 - 36.0 * f2 + 16.0 * f3 - 3.0 * f4) / 12.0;
}

/* explicit boundary row value at distance `edge` (0 or 1) from the nearer end */
static double boundary_row(const double* f, int i, int n)
{
    if (i == 0) return clos0_4(f[0], f[1], f[2], f[3], f[4]);
    if (i == n - 1) return -clos0_4(f[n - 1], f[n - 2], f[n - 3], f[n - 4], f[n - 5]);
    return 0.5 * (f[i + 1] - f[i - 1]);   /* node 1 or n-2 */
}

static void deriv_explicit_1d(int scheme, int n, int periodic, const double* f, double* df)
{
    for (int i = 0; i < n; i++) {
        int edge = i < n - 1 - i ? i : n - 1 - i;
        if (!periodic && edge < 2) df[i] = boundary_row(f, i, n);
        else if (scheme == OR_E2) df[i] = e2_int(f, i, n, periodic);
        else if (scheme == OR_E4 || (!periodic && edge == 2)) df[i] = e4_int(f, i, n, periodic);
        else df[i] = e6_int(f, i, n, periodic);
    }
}

static void deriv_compact_1d(int scheme, int n, int periodic, const double* f, double* df)
{
    double* a = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    double* c = (double*)malloc(sizeof(double) * n);
    double* d = (double*)malloc(sizeof(double) * n);
    for (int i = 0; i < n; i++) {
        int edge = i < n - 1 - i ? i : n - 1 - i;
        int ip = periodic ? wrap(i + 1, n) : i + 1;
        int im = periodic ? wrap(i - 1, n) : i - 1;
        b[i] = 1.0;
        if (!periodic && edge < 2) {
            /* explicit boundary rows: no coupling to the neighbours' derivatives */
            a[i] = 0.0;
            c[i] = 0.0;
            d[i] = boundary_row(f, i, n);
        } else if (scheme == OR_C4) {
            /* C4: 1/4 f'_{i-1} + f'_i + 1/4 f'_{i+1} = 3/2 (f_{i+1} - f_{i-1}) / 2 */
            a[i] = 0.25;
            c[i] = 0.25;
            d[i] = 1.5 * (f[ip] - f[im]) / 2.0;
        } else {
            /* C6: 1/3 f'_{i-1} + f'_i + 1/3 f'_{i+1}
             *     = 14/9 (f_{i+1} - f_{i-1}) / 2 + 1/9 (f_{i+2} - f_{i-2}) / 4 */
            int ip2 = periodic ? wrap(i + 2, n) : i + 2;
            int im2 = periodic ? wrap(i - 2, n) : i - 2;
            a[i] = 1.0 / 3.0;
            c[i] = 1.0 / 3.0;
            d[i] = (14.0 / 9.0) * (f[ip] - f[im]) / 2.0 + (1.0 / 9.0) * (f[ip2] - f[im2]) / 4.0;
        }
    }
    if (periodic) cyclic_solve(n, a, b, c, d, df);
    else thomas(n, a, b, c, d, df);
    free(a);
    free(b);
    free(c);
    free(d);
}

static void deriv_1d(int scheme, int n, int periodic, const double* f, double* df)
{
    if (scheme == OR_UW) scheme = OR_E2;   /* the baseline's central terms (Sec. 3.2.1) */
    if (scheme == OR_C4 || scheme == OR_C6) deriv_compact_1d(scheme, n, periodic, f, df);
    else deriv_explicit_1d(scheme, n, periodic, f, df);
}

/* ------------------------------------------------------------------------------------ */
/* implicit filter (Sec. 3.4, Eq. 21)                                                   */
/*   alpha_f fh_{i-1} + fh_i + alpha_f fh_{i+1} = sum_{n=0}^{N} a_n/2 (f_{i+n} + f_{i-n}) */
/* The a_n of the order-2N member are fixed by T(pi) = 0 and T(w) = 1 + O(w^{2N}) with   */
/* T(w) = sum a_n cos(n w) / (1 + 2 alpha_f cos w).  Near a non-periodic end the order  */
/* drops to 2 N' with N' = distance to the end (Sec. 3.4); the end node is unfiltered.  */
/* ------------------------------------------------------------------------------------ */

void or_filter_coeffs(int hw, double al, double* a)
{
    switch (hw) {
    case 1:
        a[0] = 0.5 + al;
        a[1] = 0.5 + al;
        break;
    case 2:
        a[0] = 5.0 / 8.0 + 3.0 * al / 4.0;
        a[1] = 0.5 + al;
        a[2] = -1.0 / 8.0 + al / 4.0;
        break;
    case 3:
        a[0] = 11.0 / 16.0 + 5.0 * al / 8.0;
        a[1] = 15.0 / 32.0 + 17.0 * al / 16.0;
        a[2] = -3.0 / 16.0 + 3.0 * al / 8.0;
        a[3] = 1.0 / 32.0 - al / 16.0;
        break;
    case 4:
        a[0] = (93.0 + 70.0 * al) / 128.0;
        a[1] = (7.0 + 18.0 * al) / 16.0;
        a[2] = (-7.0 + 14.0 * al) / 32.0;
        a[3] = (1.0 - 2.0 * al) / 16.0;
        a[4] = (-1.0 + 2.0 * al) / 128.0;
        break;
    case 5:
        a[0] = (193.0 + 126.0 * al) / 256.0;
        a[1] = (105.0 + 302.0 * al) / 256.0;
        a[2] = 15.0 * (-1.0 + 2.0 * al) / 64.0;
        a[3] = 45.0 * (1.0 - 2.0 * al) / 512.0;
        a[4] = 5.0 * (-1.0 + 2.0 * al) / 256.0;
        a[5] = (1.0 - 2.0 * al) / 512.0;
        break;
    default:
        a[0] = 1.0;
        break;
    }
}

static void filter_1d(int n, int periodic, double al, const double* f, double* out)
{
    double* a = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    double* c = (double*)malloc(sizeof(double) * n);
    double* d = (double*)malloc(sizeof(double) * n);
    double co[6];
    for (int i = 0; i < n; i++) {
        int hw = 5;
        if (!periodic) {
            int e = i < n - 1 - i ? i : n - 1 - i;
            if (e < hw) hw = e;
        }
        b[i] = 1.0;
        if (hw == 0) {
            a[i] = 0.0;
            c[i] = 0.0;
            d[i] = f[i];
            continue;
        }
        a[i] = al;
        c[i] = al;
        or_filter_coeffs(hw, al, co);
        double s = co[0] * f[i];
        for (int m = 1; m <= hw; m++) {
            int ip = periodic ? wrap(i + m, n) : i + m;
            int im = periodic ? wrap(i - m, n) : i - m;
            s += 0.5 * co[m] * (f[ip] + f[im]);
        }
        d[i] = s;
    }
    if (periodic) cyclic_solve(n, a, b, c, d, out);
    else thomas(n, a, b, c, d, out);
    free(a);
    free(b);
    free(c);
    free(d);
}

/* 5-point fourth difference (1,-4,6,-4,1) at unit spacing (d^4/dxi^4 of Eq. 7).  Within
 * two nodes of a non-periodic end the nearest complete stencil (centred on node 2 or
 * n-3) is used, so that a kink that reaches a wall corner still sees diffusion. */
static void d4_1d(int n, int periodic, const double* f, double* out)
{
    for (int i = 0; i < n; i++) {
        int c = i;
        if (!periodic) {
            if (c < 2) c = 2;
            if (c > n - 3) c = n - 3;
        }
        int m2 = periodic ? wrap(c - 2, n) : c - 2, m1 = periodic ? wrap(c - 1, n) : c - 1;
        int p1 = periodic ? wrap(c + 1, n) : c + 1, p2 = periodic ? wrap(c + 2, n) : c + 2;
        out[i] = f[m2] - 4.0 * f[m1] + 6.0 * f[c] - 4.0 * f[p1] + f[p2];
    }
}

/* Truncated 9-point Gaussian smoothing of the artificial diffusivity, as in the LAD
 * method of Kawai & Lele that Sec. 2.3.2 follows: out_i = sum_{l=-4..4} g_|l| f_{i+l}.
 * Non-periodic ends reflect about the end node (f_{-l} = f_l). */
static void gauss_1d(int n, int periodic, const double* f, double* out)
{
    static const double gw[5] = {3565.0 / 10368.0, 3091.0 / 12960.0, 1997.0 / 25920.0,
                                 149.0 / 12960.0, 107.0 / 103680.0};
    for (int i = 0; i < n; i++) {
        double s = gw[0] * f[i];
        for (int l = 1; l <= 4; l++) {
            int ip = i + l, im = i - l;
            if (periodic) {
                ip = wrap(ip, n);
                im = wrap(im, n);
            } else {
                if (ip > n - 1) ip = 2 * (n - 1) - ip;
                if (im < 0) im = -im;
            }
            s += gw[l] * (f[ip] + f[im]);
        }
        out[i] = s;
    }
}

/* ------------------------------------------------------------------------------------ */
/* directional operators on the grid: gather a line, apply, scatter                     */
/* ------------------------------------------------------------------------------------ */

enum { OP_DERIV, OP_FILTER, OP_D4, OP_GAUSS };

static void apply_dir(const or_ctx* C, int op, int scheme, double al, int dir,
                      const double* in, double* out)
{
    const or_grid_desc* g = &C->g;
    int n = g->n[dir];
    int per = is_periodic(g, dir);
    int* ids = (int*)malloc(sizeof(int) * n);
    double* f = (double*)malloc(sizeof(double) * n);
    double* r = (double*)malloc(sizeof(double) * n);
    int L = line_count(C, dir);
    for (int q = 0; q < L; q++) {
        line_nodes(g, dir, q, ids);
        for (int t = 0; t < n; t++) f[t] = in[ids[t]];
        if (op == OP_DERIV) deriv_1d(scheme, n, per, f, r);
        else if (op == OP_FILTER) filter_1d(n, per, al, f, r);
        else if (op == OP_D4) d4_1d(n, per, f, r);
        else gauss_1d(n, per, f, r);
        for (int t = 0; t < n; t++) out[ids[t]] = r[t];
    }
    free(ids);
    free(f);
    free(r);
}

void or_deriv(const or_ctx* C, int scheme, int dir, const double* in, double* out)
{
    apply_dir(C, OP_DERIV, scheme, 0.0, dir, in, out);
}

void or_filter(const or_ctx* C, double alpha_f, int dir, const double* in, double* out)
{
    apply_dir(C, OP_FILTER, 0, alpha_f, dir, in, out);
}

/* ------------------------------------------------------------------------------------ */
/* grid metrics (Sec. 3.1): A[m][l] = dx_m/dxi_l by the solve's scheme (Sec. 3.2.2),    */
/* d(xi_l)/d(x_m) = (A^-1)[l][m], J = det A, Delta x_l = |column l of A|.                */
/* ------------------------------------------------------------------------------------ */

static double det3(const double A[3][3])
{
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
         - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
         + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* inverse by cofactors: inv[l][m] = cof(A)[m][l] / det */
static void inv3(const double A[3][3], double inv[3][3], double* detA)
{
    double d = det3(A);
    inv[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / d;
    inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / d;
    inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / d;
    inv[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / d;
    inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / d;
    inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / d;
    inv[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / d;
    inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / d;
    inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / d;
    *detA = d;
}

static void compute_metrics(or_ctx* C)
{
    const or_grid_desc* g = &C->g;
    int N = C->N, nd = g->ndim;
    double* A = (double*)calloc((size_t)9 * N, sizeof(double)); /* A[(m*3+l)*N+p] */
    double* tmp = (double*)malloc(sizeof(double) * N);
    double* dtmp = (double*)malloc(sizeof(double) * N);
    for (int l = 0; l < nd; l++) {
        int per = is_periodic(g, l);
        int n = g->n[l];
        for (int m = 0; m < nd; m++) {
            /* periodic direction: differentiate x_m - period*t/n (a periodic function)
             * and add back the exact derivative period/n of the linear part */
            double shift = per ? g->period[l][m] : 0.0;
            for (int p = 0; p < N; p++) {
                int c[3];
                c[0] = p % g->n[0];
                c[1] = (p / g->n[0]) % g->n[1];
                c[2] = p / (g->n[0] * g->n[1]);
                tmp[p] = C->xyz[m * N + p] - shift * (double)c[l] / (double)n;
            }
            or_deriv(C, C->scheme, l, tmp, dtmp);
            for (int p = 0; p < N; p++) A[(m * 3 + l) * N + p] = dtmp[p] + shift / (double)n;
        }
    }
    for (int p = 0; p < N; p++) {
        double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Mi[3][3], det;
        for (int m = 0; m < 3; m++)
            for (int l = 0; l < 3; l++) M[m][l] = (m < nd && l < nd) ? A[(m * 3 + l) * N + p] : (m == l ? 1.0 : 0.0);
        inv3(M, Mi, &det);
        C->J[p] = det;
        for (int l = 0; l < 3; l++)
            for (int m = 0; m < 3; m++)
                C->xi[(l * 3 + m) * N + p] = (l < nd && m < nd) ? Mi[l][m] : 0.0;
        for (int l = 0; l < 3; l++) {
            double s = 0.0;
            for (int m = 0; m < nd; m++) s += M[m][l] * M[m][l];
            C->dx[l * N + p] = l < nd ? sqrt(s) : 0.0;
        }
    }
    free(A);
    free(tmp);
    free(dtmp);
}

static double dist_nodes(const or_ctx* C, int p, int q)
{
    double s = 0.0;
    for (int m = 0; m < 3; m++) {
        double d = C->xyz[m * C->N + p] - C->xyz[m * C->N + q];
        s += d * d;
    }
    return sqrt(s);
}

/* spacing ratio |x_b - x_{b+-1}| / |x_{b+-1} - x_{b+-2}| on every face node */
static void compute_ff_ratio(or_ctx* C)
{
    const or_grid_desc* g = &C->g;
    int n0 = g->n[0], n1 = g->n[1];
    for (int d = 0; d < g->ndim; d++) {
        int n = g->n[d];
        for (int side = 0; side < 2; side++) {
            double* r = C->ff_ratio + (size_t)(2 * d + side) * C->N;
            for (int p = 0; p < C->N; p++) {
                int c[3] = {p % n0, (p / n0) % n1, p / (n0 * n1)};
                int b = side ? n - 1 : 0, s = side ? -1 : 1;
                if (c[d] != b) {
                    r[p] = 0.0;
                    continue;
                }
                int c1[3] = {c[0], c[1], c[2]}, c2[3] = {c[0], c[1], c[2]};
                c1[d] = b + s;
                c2[d] = b + 2 * s;
                int p1 = node_index(g, c1), p2 = node_index(g, c2);
                r[p] = dist_nodes(C, p, p1) / dist_nodes(C, p1, p2);
            }
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* context                                                                              */
/* ------------------------------------------------------------------------------------ */

static int on_face(const or_grid_desc* g, int p, int d, int side)
{
    int c[3] = {p % g->n[0], (p / g->n[0]) % g->n[1], p / (g->n[0] * g->n[1])};
    return c[d] == (side ? g->n[d] - 1 : 0);
}

void or_set_dirichlet(or_ctx* C, const unsigned char* mask, const double* dval)
{
    const or_grid_desc* g = &C->g;
    for (int p = 0; p < C->N; p++) {
        C->dmask[p] = mask ? (mask[p] != 0) : 0;
        C->dval[p] = (mask && mask[p] && dval) ? dval[p] : 0.0;
    }
    /* wall faces: phi = 0 (Eq. 22) */
    for (int d = 0; d < g->ndim; d++)
        for (int side = 0; side < 2; side++) {
            int bc = side ? g->bc_hi[d] : g->bc_lo[d];
            if (bc != OR_BC_WALL) continue;
            for (int p = 0; p < C->N; p++)
                if (on_face(g, p, d, side)) {
                    C->dmask[p] = 1;
                    C->dval[p] = 0.0;
                }
        }
}

or_ctx* or_create(const or_grid_desc* desc, const double* xyz, int scheme,
                  const unsigned char* mask, const double* dval)
{
    if (!desc || !xyz) return NULL;
    if (desc->ndim != 2 && desc->ndim != 3) return NULL;
    if (desc->ndim == 2 && desc->n[2] != 1) return NULL;
    for (int d = 0; d < desc->ndim; d++) {
        if (desc->n[d] < 8) return NULL;
        int plo = desc->bc_lo[d] == OR_BC_PERIODIC, phi = desc->bc_hi[d] == OR_BC_PERIODIC;
        if (plo != phi) return NULL;
    }
    if (scheme < OR_E2 || scheme > OR_UW) return NULL;
    or_ctx* C = (or_ctx*)calloc(1, sizeof(or_ctx));
    C->g = *desc;
    C->N = desc->n[0] * desc->n[1] * desc->n[2];
    C->scheme = scheme;
    int N = C->N;
    C->xyz = (double*)calloc((size_t)3 * N, sizeof(double));
    memcpy(C->xyz, xyz, sizeof(double) * (size_t)desc->ndim * N);
    C->xi = (double*)calloc((size_t)9 * N, sizeof(double));
    C->J = (double*)calloc(N, sizeof(double));
    C->dx = (double*)calloc((size_t)3 * N, sizeof(double));
    C->ff_ratio = (double*)calloc((size_t)6 * N, sizeof(double));
    C->dmask = (unsigned char*)calloc(N, 1);
    C->dval = (double*)calloc(N, sizeof(double));
    compute_metrics(C);
    compute_ff_ratio(C);
    or_set_dirichlet(C, mask, dval);
    return C;
}

void or_destroy(or_ctx* C)
{
    if (!C) return;
    free(C->xyz);
    free(C->xi);
    free(C->J);
    free(C->dx);
    free(C->ff_ratio);
    free(C->dmask);
    free(C->dval);
    free(C);
}

void or_get_metrics(const or_ctx* C, double* xi, double* J, double* dx)
{
    if (xi) memcpy(xi, C->xi, sizeof(double) * 9 * (size_t)C->N);
    if (J) memcpy(J, C->J, sizeof(double) * (size_t)C->N);
    if (dx) memcpy(dx, C->dx, sizeof(double) * 3 * (size_t)C->N);
}

/* ------------------------------------------------------------------------------------ */
/* boundary conditions (Sec. 3.5)                                                       */
/* ------------------------------------------------------------------------------------ */

/* Far-field / Neumann faces direction by direction (0, 1, 2), then Dirichlet nodes.
 * poisson != 0: every non-wall, non-periodic face is Neumann and Dirichlet values are 0. */
static void apply_bc(const or_ctx* C, double* phi, int poisson)
{
    const or_grid_desc* g = &C->g;
    for (int d = 0; d < g->ndim; d++) {
        for (int side = 0; side < 2; side++) {
            int bc = side ? g->bc_hi[d] : g->bc_lo[d];
            if (bc == OR_BC_WALL || bc == OR_BC_PERIODIC) continue;
            if (poisson) bc = OR_BC_NEUMANN;
            const double* rat = C->ff_ratio + (size_t)(2 * d + side) * C->N;
            int stride = d == 0 ? 1 : (d == 1 ? g->n[0] : g->n[0] * g->n[1]);
            int s = side ? -stride : stride;
            for (int p = 0; p < C->N; p++) {
                if (!on_face(g, p, d, side)) continue;
                if (bc == OR_BC_NEUMANN) phi[p] = phi[p + s];
                else phi[p] = phi[p + s] + rat[p] * (phi[p + s] - phi[p + 2 * s]);
            }
        }
    }
    for (int p = 0; p < C->N; p++)
        if (C->dmask[p]) phi[p] = poisson ? 0.0 : C->dval[p];
}

void or_apply_bc(const or_ctx* C, double* phi) { apply_bc(C, phi, 0); }

/* ------------------------------------------------------------------------------------ */
/* baseline upwind scheme (Sec. 3.2.1, Eqs. UW1-UW5) and the level-set equation (Sec. 5.5) */
/* ------------------------------------------------------------------------------------ */

/* Backward and forward differences B_l, F_l along direction dir at unit computational
 * spacing (Eq. UW2).  Periodic lines wrap; the end node of an open line has one of the two
 * and uses it for both (such nodes are wall, far-field or Neumann nodes, whose values the
 * boundary conditions set). */
static void one_sided_diffs(const or_ctx* C, int dir, const double* phi, double* B, double* F)
{
    const or_grid_desc* g = &C->g;
    int n = g->n[dir];
    int per = is_periodic(g, dir);
    int* ids = (int*)malloc(sizeof(int) * n);
    int L = line_count(C, dir);
    for (int q = 0; q < L; q++) {
        line_nodes(g, dir, q, ids);
        for (int t = 0; t < n; t++) {
            double b = 0.0, f = 0.0;
            int have_b = per || t > 0, have_f = per || t < n - 1;
            if (have_b) b = phi[ids[t]] - phi[ids[per ? wrap(t - 1, n) : t - 1]];
            if (have_f) f = phi[ids[per ? wrap(t + 1, n) : t + 1]] - phi[ids[t]];
            if (!have_b) b = f;
            if (!have_f) f = b;
            B[ids[t]] = b;
            F[ids[t]] = f;
        }
    }
    free(ids);
}

/* SIGN(1, x) of Eqs. UW4-UW5: +1 for x >= 0, -1 for x < 0 */
static double sign1(double x) { return x >= 0.0 ? 1.0 : -1.0; }

/* Eqs. UW3-UW5.  The weight n_{i-1} is 1 where B >= 0 and B + F >= 0: phi grows from node
 * i-1 and that side is upwind, so the slope is the difference that reaches node i-1, B.
 * The weight n_{i+1} is 1 where F < 0 and B + F < 0, and takes F.  Both weights vanish at a
 * local minimum of phi (B < 0 < F), where the slope is 0.  (The printed Eq. UW3 pairs
 * n_{i-1} with F; that pairing takes the downwind difference, so the weights are read as
 * naming the side their difference reaches.) */
double or_upwind_slope(double B, double F)
{
    double s = sign1(F + B);
    double n_im1 = 0.25 * (1.0 + s) * (1.0 + sign1(B));
    double n_ip1 = 0.25 * (1.0 - s) * (1.0 - sign1(F));
    return n_im1 * B + n_ip1 * F;
}

/* Eq. UW1 summed over the directions: sum_l Uh_l d(phi)/d(xi_l) with
 * Uh_l = sum_m d(xi_l)/d(x_m) U_m, U_m = sum_k d(xi_k)/d(x_m) s_k and s_k the upwind slope
 * along k (Eqs. UW3-UW5); each direction's product takes B where Uh_l >= 0, F where < 0. */
void or_upwind_advection(const or_ctx* C, const double* phi, double* adv)
{
    int N = C->N, nd = C->g.ndim;
    double* B = (double*)malloc(sizeof(double) * (size_t)3 * N);
    double* F = (double*)malloc(sizeof(double) * (size_t)3 * N);
    for (int l = 0; l < nd; l++) one_sided_diffs(C, l, phi, B + (size_t)l * N, F + (size_t)l * N);
    for (int p = 0; p < N; p++) {
        double sl[3] = {0.0, 0.0, 0.0}, Um[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < nd; k++) sl[k] = or_upwind_slope(B[(size_t)k * N + p], F[(size_t)k * N + p]);
        for (int m = 0; m < nd; m++)
            for (int k = 0; k < nd; k++) Um[m] += C->xi[(k * 3 + m) * N + p] * sl[k];
        double a = 0.0;
        for (int l = 0; l < nd; l++) {
            double uh = 0.0;
            for (int m = 0; m < nd; m++) uh += C->xi[(l * 3 + m) * N + p] * Um[m];
            a += 0.5 * (uh + fabs(uh)) * B[(size_t)l * N + p] + 0.5 * (uh - fabs(uh)) * F[(size_t)l * N + p];
        }
        adv[p] = a;
    }
    free(B);
    free(F);
}

/* |grad phi| = (sum_m U_m^2)^(1/2) with U_m from the upwind slopes.  For F < 0 the front
 * moves towards decreasing phi: the slopes are those of -phi (differences -B, -F), whose
 * magnitude is what enters |grad phi|. */
void or_levelset_gradmag(const or_ctx* C, double Fs, const double* phi, double* gm)
{
    int N = C->N, nd = C->g.ndim;
    double sg = Fs < 0.0 ? -1.0 : 1.0;
    double* B = (double*)malloc(sizeof(double) * (size_t)3 * N);
    double* F = (double*)malloc(sizeof(double) * (size_t)3 * N);
    for (int l = 0; l < nd; l++) one_sided_diffs(C, l, phi, B + (size_t)l * N, F + (size_t)l * N);
    for (int p = 0; p < N; p++) {
        double sl[3] = {0.0, 0.0, 0.0}, g2 = 0.0;
        for (int k = 0; k < nd; k++)
            sl[k] = or_upwind_slope(sg * B[(size_t)k * N + p], sg * F[(size_t)k * N + p]);
        for (int m = 0; m < nd; m++) {
            double u = 0.0;
            for (int k = 0; k < nd; k++) u += C->xi[(k * 3 + m) * N + p] * sl[k];
            g2 += u * u;
        }
        gm[p] = sqrt(g2);
    }
    free(B);
    free(F);
}

/* zero normal gradient on every non-periodic face (Sec. 5.5), direction by direction */
static void levelset_bc(const or_ctx* C, double* phi)
{
    const or_grid_desc* g = &C->g;
    for (int d = 0; d < g->ndim; d++) {
        if (is_periodic(g, d)) continue;
        int stride = d == 0 ? 1 : (d == 1 ? g->n[0] : g->n[0] * g->n[1]);
        for (int side = 0; side < 2; side++) {
            int s = side ? -stride : stride;
            for (int p = 0; p < C->N; p++)
                if (on_face(g, p, d, side)) phi[p] = phi[p + s];
        }
    }
}

void or_levelset_steps(const or_ctx* C, double Fs, double dt, double* phi, int n)
{
    int N = C->N;
    double* p0 = (double*)malloc(sizeof(double) * N);
    double* s = (double*)malloc(sizeof(double) * N);
    double* gm = (double*)malloc(sizeof(double) * N);
    double* K[4];
    for (int k = 0; k < 4; k++) K[k] = (double*)malloc(sizeof(double) * N);
    static const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    for (int it = 0; it < n; it++) {
        memcpy(p0, phi, sizeof(double) * N);
        for (int k = 0; k < 4; k++) {
            if (k == 0) memcpy(s, p0, sizeof(double) * N);
            else {
                for (int p = 0; p < N; p++) s[p] = p0[p] + cst[k] * dt * K[k - 1][p];
                levelset_bc(C, s);
            }
            or_levelset_gradmag(C, Fs, s, gm);
            for (int p = 0; p < N; p++) K[k][p] = -Fs * gm[p];       /* Eq. levelset, RHS 0 */
        }
        for (int p = 0; p < N; p++)
            phi[p] = p0[p] + dt / 6.0 * (K[0][p] + 2.0 * K[1][p] + 2.0 * K[2][p] + K[3][p]);
        levelset_bc(C, phi);
    }
    free(p0);
    free(s);
    free(gm);
    for (int k = 0; k < 4; k++) free(K[k]);
}

/* ------------------------------------------------------------------------------------ */
/* right-hand sides                                                                     */
/* ------------------------------------------------------------------------------------ */

/* U_m = sum_l d(xi_l)/d(x_m) * d(phi)/d(xi_l)  (Sec. 3.1) */
static void grad_phys(const or_ctx* C, int scheme, const double* phi, double* U /* 3N */)
{
    int N = C->N, nd = C->g.ndim;
    double* D = (double*)malloc(sizeof(double) * (size_t)3 * N);
    for (int l = 0; l < nd; l++) or_deriv(C, scheme, l, phi, D + (size_t)l * N);
    for (int m = 0; m < 3; m++)
        for (int p = 0; p < N; p++) {
            double s = 0.0;
            for (int l = 0; l < nd; l++) s += C->xi[(l * 3 + m) * N + p] * D[(size_t)l * N + p];
            U[(size_t)m * N + p] = m < nd ? s : 0.0;
        }
    free(D);
}

/* divergence written as in Eq. 9: sum_m sum_l d(xi_l)/d(x_m) * d(V_m)/d(xi_l) */
static void div_phys(const or_ctx* C, int scheme, const double* V /* 3N */, double* out)
{
    int N = C->N, nd = C->g.ndim;
    double* D = (double*)malloc(sizeof(double) * N);
    for (int p = 0; p < N; p++) out[p] = 0.0;
    for (int m = 0; m < nd; m++)
        for (int l = 0; l < nd; l++) {
            or_deriv(C, scheme, l, V + (size_t)m * N, D);
            for (int p = 0; p < N; p++) out[p] += C->xi[(l * 3 + m) * N + p] * D[p];
        }
    free(D);
}

static double metric_sum1(const or_ctx* C, int p)   /* sum_l |grad xi_l| */
{
    double s = 0.0;
    for (int l = 0; l < C->g.ndim; l++) {
        double q = 0.0;
        for (int m = 0; m < C->g.ndim; m++) {
            double x = C->xi[(l * 3 + m) * C->N + p];
            q += x * x;
        }
        s += sqrt(q);
    }
    return s;
}

/* sum_l sum_k |grad xi_l . grad xi_k|: the Gershgorin bound of the metric tensor of the
 * second-order term (equal to sum_l |grad xi_l|^2 on orthogonal grids); the local pseudo
 * time step uses it so that the cross terms of skewed grids are covered */
static double metric_sum2(const or_ctx* C, int p)
{
    double s = 0.0;
    for (int l = 0; l < C->g.ndim; l++)
        for (int k = 0; k < C->g.ndim; k++) {
            double q = 0.0;
            for (int m = 0; m < C->g.ndim; m++)
                q += C->xi[(l * 3 + m) * C->N + p] * C->xi[(k * 3 + m) * C->N + p];
            s += fabs(q);
        }
    return s;
}

void or_rhs_hj(const or_ctx* C, const or_params* P, const double* phi, double* R, double* dt)
{
    int N = C->N, nd = C->g.ndim;
    double* U = (double*)malloc(sizeof(double) * (size_t)3 * N);
    double* lap = (double*)malloc(sizeof(double) * N);
    double* kap = (double*)calloc(N, sizeof(double));
    double* lad = (double*)calloc(N, sizeof(double));
    double* d4 = (double*)malloc(sizeof(double) * N);

    /* U = grad(phi) through the chain rule, then the Laplacian as div(U) (Eq. 9) */
    grad_phys(C, P->scheme, phi, U);
    div_phys(C, P->scheme, U, lap);

    /* baseline scheme: the advection term U.grad(phi) by upwinding (Eqs. UW1-UW5) */
    double* adv = NULL;
    if (P->scheme == OR_UW) {
        adv = (double*)malloc(sizeof(double) * N);
        or_upwind_advection(C, phi, adv);
    }

    /* Nakanishi curvature (Eq. 25): kappa = div(n), n = grad(phi) / (|grad(phi)| + eps0) */
    if (P->curvature) {
        double* nv = (double*)calloc((size_t)3 * N, sizeof(double));
        for (int p = 0; p < N; p++) {
            double g2 = 0.0;
            for (int m = 0; m < nd; m++) g2 += U[(size_t)m * N + p] * U[(size_t)m * N + p];
            for (int m = 0; m < nd; m++) nv[(size_t)m * N + p] = U[(size_t)m * N + p] / (sqrt(g2) + P->eps0);
        }
        div_phys(C, P->scheme, nv, kap);
        free(nv);
    }

    /* LAD term of Eq. 7: C | sum_l (sum_m xi_{l,x_m}^2)^2 d4_l(phi) Delta x_l^exp |, then
     * smoothed by the truncated Gaussian along every direction (Kawai & Lele's LAD). */
    if (P->equation == OR_HJ_LAD) {
        for (int l = 0; l < nd; l++) {
            apply_dir(C, OP_D4, 0, 0.0, l, phi, d4);
            for (int p = 0; p < N; p++) {
                double q = 0.0;
                for (int m = 0; m < nd; m++) {
                    double x = C->xi[(l * 3 + m) * N + p];
                    q += x * x;
                }
                lad[p] += q * q * d4[p] * pow(C->dx[(size_t)l * N + p], P->lad_exp);
            }
        }
        for (int p = 0; p < N; p++) lad[p] = P->C_lad * fabs(lad[p]);
        for (int l = 0; l < nd; l++) {
            apply_dir(C, OP_GAUSS, 0, 0.0, l, lad, d4);
            memcpy(lad, d4, sizeof(double) * N);
        }
    }

    for (int p = 0; p < N; p++) {
        double g2 = 0.0;
        for (int m = 0; m < nd; m++) g2 += U[(size_t)m * N + p] * U[(size_t)m * N + p];
        double gm = sqrt(g2);
        double gam;
        double phip = phi[p] > 0.0 ? phi[p] : 0.0;
        if (P->equation == OR_HJ_STD) gam = P->eps * phip;                 /* Eq. 6 */
        else if (P->equation == OR_HJ_LAD) {                               /* Eq. 7 */
            double a = P->eps * phip, b = lad[p];
            gam = a < b ? a : b;
        } else gam = 0.0;                                                  /* Eq. 17 */
        double v = 0.0, r;
        double a2 = adv ? adv[p] : g2;                                     /* U.grad(phi) */
        if (P->curvature) {
            v = 0.001 * (1.0 - gm) * (1.0 - gm);
            double corr = gm * kap[p] > 0.0 ? gm * kap[p] : 0.0;
            r = 1.0 + (gam + v) * (lap[p] - corr) - a2;                    /* Eq. 25 */
        } else {
            r = 1.0 + gam * lap[p] - a2;                                   /* Eqs. 5, 18 */
        }
        R[p] = r;
        if (dt) {
            double a = gm > 1.0 ? gm : 1.0;
            dt[p] = P->cfl / (metric_sum1(C, p) * a + (gam + v) * metric_sum2(C, p));
        }
    }
    free(U);
    free(lap);
    free(kap);
    free(lad);
    free(d4);
    free(adv);
}

void or_rhs_poisson(const or_ctx* C, const or_params* P, const double* phi, double* R, double* dt)
{
    int N = C->N;
    double* U = (double*)malloc(sizeof(double) * (size_t)3 * N);
    double* lap = (double*)malloc(sizeof(double) * N);
    grad_phys(C, P->scheme, phi, U);
    div_phys(C, P->scheme, U, lap);
    for (int p = 0; p < N; p++) {
        R[p] = 1.0 + lap[p];                                   /* Eq. 19 read as phi'_t = lap + 1 */
        if (dt) dt[p] = P->cfl / metric_sum2(C, p);
    }
    free(U);
    free(lap);
}

void or_spalding(const or_ctx* C, const or_params* P, const double* phip, double* phi)
{
    int N = C->N, nd = C->g.ndim;
    double* U = (double*)malloc(sizeof(double) * (size_t)3 * N);
    grad_phys(C, P->scheme, phip, U);
    for (int p = 0; p < N; p++) {
        double g2 = 0.0;
        for (int m = 0; m < nd; m++) g2 += U[(size_t)m * N + p] * U[(size_t)m * N + p];
        double arg = g2 + 2.0 * phip[p];
        phi[p] = -sqrt(g2) + sqrt(arg > 0.0 ? arg : 0.0);       /* Eq. 4, minus root */
    }
    free(U);
}

/* ------------------------------------------------------------------------------------ */
/* pseudo-time stepping (Sec. 3.3): classical RK4, local step frozen over the stages,   */
/* BCs after every stage, filter along every direction after the step (Sec. 3.4).       */
/* ------------------------------------------------------------------------------------ */

static void one_step(const or_ctx* C, const or_params* P, int poisson, double* phi,
                     double* l2, double* linf)
{
    int N = C->N;
    double* p0 = (double*)malloc(sizeof(double) * N);
    double* s = (double*)malloc(sizeof(double) * N);
    double* dt = (double*)malloc(sizeof(double) * N);
    double* K[4];
    for (int k = 0; k < 4; k++) K[k] = (double*)malloc(sizeof(double) * N);
    memcpy(p0, phi, sizeof(double) * N);

    static const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    for (int k = 0; k < 4; k++) {
        if (k == 0) memcpy(s, p0, sizeof(double) * N);
        else {
            for (int p = 0; p < N; p++) s[p] = p0[p] + cst[k] * dt[p] * K[k - 1][p];
            apply_bc(C, s, poisson);
        }
        if (poisson) or_rhs_poisson(C, P, s, K[k], k == 0 ? dt : NULL);
        else or_rhs_hj(C, P, s, K[k], k == 0 ? dt : NULL);
    }
    for (int p = 0; p < N; p++)
        phi[p] = p0[p] + dt[p] / 6.0 * (K[0][p] + 2.0 * K[1][p] + 2.0 * K[2][p] + K[3][p]);
    apply_bc(C, phi, poisson);
    if (P->filter) {
        for (int d = 0; d < C->g.ndim; d++) {
            or_filter(C, P->alpha_f, d, phi, s);
            memcpy(phi, s, sizeof(double) * N);
        }
        apply_bc(C, phi, poisson);
    }
    /* change over the non-Dirichlet nodes */
    double ss = 0.0, mx = 0.0;
    int cnt = 0;
    for (int p = 0; p < N; p++) {
        if (C->dmask[p]) continue;
        double d = phi[p] - p0[p];
        ss += d * d;
        if (!(fabs(d) <= mx)) mx = fabs(d);   /* keeps NaN */
        cnt++;
    }
    *l2 = cnt ? sqrt(ss / cnt) : 0.0;
    *linf = mx;
    free(p0);
    free(s);
    free(dt);
    for (int k = 0; k < 4; k++) free(K[k]);
}

void or_hj_steps(const or_ctx* C, const or_params* P, double* phi, int n, or_stats* st)
{
    double l2 = 0.0, li = 0.0;
    for (int i = 0; i < n; i++) one_step(C, P, 0, phi, &l2, &li);
    if (st) {
        st->iters = n;
        st->res_l2 = l2 / C->g.L_ref;
        st->res_linf = li / C->g.L_ref;
        st->converged = 0;
        st->diverged = !(isfinite(l2) && isfinite(li));
    }
}

void or_poisson_steps(const or_ctx* C, const or_params* P, double* phip, int n, or_stats* st)
{
    double l2 = 0.0, li = 0.0;
    for (int i = 0; i < n; i++) one_step(C, P, 1, phip, &l2, &li);
    if (st) {
        st->poisson_iters = n;
        st->res_l2 = l2 / (C->g.L_ref * C->g.L_ref);
        st->res_linf = li / (C->g.L_ref * C->g.L_ref);
        st->diverged = !(isfinite(l2) && isfinite(li));
    }
}

static int met(double v, double tol) { return tol <= 0.0 || v <= tol; }

int or_solve(const or_ctx* C, const or_params* P, double* phi, or_stats* st)
{
    int N = C->N;
    double L = C->g.L_ref;
    or_stats s;
    memset(&s, 0, sizeof(s));
    int every = P->check_every > 0 ? P->check_every : 1;

    if (P->init == OR_INIT_POISSON) {
        double* pp = (double*)calloc(N, sizeof(double));
        apply_bc(C, pp, 1);
        double l2 = 0.0, li = 0.0;
        int it = 0;
        while (it < P->poisson_max_iters) {
            one_step(C, P, 1, pp, &l2, &li);
            it++;
            if (!(isfinite(l2) && isfinite(li))) break;
            if (P->poisson_tol > 0.0 && it % every == 0 && l2 / (L * L) <= P->poisson_tol) break;
        }
        s.poisson_iters = it;
        or_spalding(C, P, pp, phi);
        free(pp);
    } else if (P->init == OR_INIT_ZERO) {
        for (int p = 0; p < N; p++) phi[p] = 0.0;
    }
    apply_bc(C, phi, 0);

    int rc = 1;
    int have_tol = P->tol_l2 > 0.0 || P->tol_linf > 0.0;
    double l2 = 0.0, li = 0.0;
    int it = 0;
    while (it < P->max_iters) {
        one_step(C, P, 0, phi, &l2, &li);
        it++;
        if (!(isfinite(l2) && isfinite(li))) {
            rc = 2;
            s.diverged = 1;
            break;
        }
        if (have_tol && (it % every == 0 || it == P->max_iters) &&
            met(l2 / L, P->tol_l2) && met(li / L, P->tol_linf)) {
            rc = 0;
            s.converged = 1;
            break;
        }
    }
    s.iters = it;
    s.res_l2 = l2 / L;
    s.res_linf = li / L;
    if (st) *st = s;
    return rc;
}
