// wd_linesys.cu -- host-side precomputation of the constant-coefficient tridiagonal
// systems solved along grid lines: compact first derivatives (Sec. 3.2.2, Eq. 16) and the
// implicit filter (Sec. 3.4, Eq. 21).
//
// Every system has unit diagonal and constant off-diagonals except in its boundary rows,
// and is the same for every line of a direction, so its elimination can be prepared once
// per (direction, scheme or alpha_f).  The GPU solves each line by parallel cyclic
// reduction (one thread per row, log2 N levels): the multipliers of every level and the
// final pivots depend only on the matrix and are computed here in double.  Periodic lines
// use the Sherman-Morrison identity on top of the corner-free matrix.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "wd_api_internal.h"

namespace wd {

// Solves the small dense system M x = r in place (Gaussian elimination, partial pivoting).
// Returns false when singular.
bool dense_solve(int n, std::vector<double>& M, std::vector<double>& r)
{
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int i = col + 1; i < n; i++)
            if (std::fabs(M[i * n + col]) > std::fabs(M[piv * n + col])) piv = i;
        if (M[piv * n + col] == 0.0) return false;
        if (piv != col) {
            for (int k = 0; k < n; k++) std::swap(M[col * n + k], M[piv * n + k]);
            std::swap(r[col], r[piv]);
        }
        for (int i = col + 1; i < n; i++) {
            double f = M[i * n + col] / M[col * n + col];
            if (f == 0.0) continue;
            for (int k = col; k < n; k++) M[i * n + k] -= f * M[col * n + k];
            r[i] -= f * r[col];
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = r[i];
        for (int k = i + 1; k < n; k++) s -= M[i * n + k] * r[k];
        r[i] = s / M[i * n + i];
    }
    return true;
}

// Right-hand-side coefficients a_0..a_hw of the centred filter of order 2 hw, from the
// conditions that define it: transfer function T(w) = sum a_n cos(n w) / (1 + 2 al cos w)
// with T(0) = 1, T(pi) = 0 and T(w) - 1 = O(w^(2 hw)), i.e.
//   sum a_n = 1 + 2 al,   sum (-1)^n a_n = 0,   sum n^(2k) a_n = 2 al  (k = 1 .. hw-1).
bool filter_coefficients(int hw, double al, double* a)
{
    int n = hw + 1;
    std::vector<double> M((size_t)n * n, 0.0), r(n, 0.0);
    for (int m = 0; m < n; m++) {
        M[0 * n + m] = 1.0;
        M[1 * n + m] = (m % 2 == 0) ? 1.0 : -1.0;
    }
    r[0] = 1.0 + 2.0 * al;
    r[1] = 0.0;
    for (int k = 1; k < hw; k++) {
        for (int m = 0; m < n; m++) M[(size_t)(k + 1) * n + m] = std::pow((double)m, 2.0 * k);
        r[k + 1] = 2.0 * al;
    }
    if (!dense_solve(n, M, r)) return false;
    for (int m = 0; m < n; m++) a[m] = r[m];
    return true;
}

// Off-diagonals of the derivative system (unit diagonal).  Boundary rows 0, 1, N-2, N-1
// of a non-periodic line are explicit (no coupling); the interior rows of C4 / C6 couple
// with alpha = 1/4 / 1/3.
void derivative_rows(int scheme, int N, int periodic, std::vector<double>& a,
                     std::vector<double>& c, int& implicit)
{
    a.assign(N, 0.0);
    c.assign(N, 0.0);
    implicit = (scheme == WD_C4 || scheme == WD_C6);
    if (!implicit) return;
    double al = scheme == WD_C4 ? 0.25 : 1.0 / 3.0;
    for (int t = 0; t < N; t++) {
        int edge = t < N - 1 - t ? t : N - 1 - t;
        if (!periodic && edge < 2) continue;
        a[t] = al;
        c[t] = al;
    }
}

// Off-diagonals of the filter system: alpha_f everywhere except the unfiltered end rows.
void filter_rows(double al, int N, int periodic, std::vector<double>& a,
                 std::vector<double>& c, int& implicit)
{
    a.assign(N, 0.0);
    c.assign(N, 0.0);
    implicit = al != 0.0;
    for (int t = 0; t < N; t++) {
        if (!periodic && (t == 0 || t == N - 1)) continue;
        a[t] = al;
        c[t] = al;
    }
}

// Thomas solve of a corner-free tridiagonal system (host, double)
static void thomas_host(int n, const std::vector<double>& a, const std::vector<double>& b,
                        const std::vector<double>& c, const std::vector<double>& d,
                        std::vector<double>& x)
{
    std::vector<double> cp(n), dp(n);
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int i = 1; i < n; i++) {
        double m = b[i] - a[i] * cp[i - 1];
        cp[i] = c[i] / m;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
    }
    x.assign(n, 0.0);
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
}

static void build_part_table(int N, int periodic, const std::vector<double>& a0v,
                             const std::vector<double>& c0v, int implicit, HostLineTab& tab);

// Builds the PCR tables of the system a_t x_{t-1} + x_t + c_t x_{t+1} = d_t
// (periodic: a_0 couples x_{N-1} and c_{N-1} couples x_0).
wd_status build_line_table(int N, int periodic, const std::vector<double>& a0v,
                           const std::vector<double>& c0v, int implicit, HostLineTab& tab)
{
    free_line_table(tab);
    tab.N = N;
    tab.implicit = implicit;
    tab.periodic = periodic;
    std::vector<double> a = a0v, b(N, 1.0), c = c0v;
    if (periodic) {
        // B = A - u v^T with u = (-1, 0, .., 0, c_{N-1}), v = (1, 0, .., 0, -a_0): corner-free,
        // diagonal changed in its first and last entries
        b[0] = 2.0;
        b[N - 1] = 1.0 + a[0] * c[N - 1];
        tab.a0 = a[0];
    }
    a[0] = 0.0;
    c[N - 1] = 0.0;
    std::vector<double> z(N, 0.0);
    if (periodic && implicit) {
        std::vector<double> u(N, 0.0);
        u[0] = -1.0;
        u[N - 1] = c0v[N - 1];
        thomas_host(N, a, b, c, u, z);
        tab.inv_den = 1.0 / (1.0 + z[0] - tab.a0 * z[N - 1]);
    }
    int L = 0;
    while ((1 << L) < N) L++;
    tab.L = implicit ? L : 0;
    std::vector<double> h((size_t)(2 * L + 3) * N, 0.0);
    double* alpha = h.data();
    double* gamma = alpha + (size_t)L * N;
    double* ib = gamma + (size_t)L * N;
    double* ib32 = ib + N;
    double* zt = ib32 + N;
    // Early stop: once every row's remaining off-diagonal weight (|a| + |c|) / |b| is below
    // the rounding of the working precision, further levels change nothing representable;
    // C6 (alpha = 1/3) gets there in about 6 (float) / 7 (double) levels, the filter with
    // alpha_f -> 1/2 needs nearly all log2 N levels.
    auto coupling = [&](void) {
        double w = 0.0;
        for (int i = 0; i < N; i++) w = std::max(w, (std::fabs(a[i]) + std::fabs(c[i])) / std::fabs(b[i]));
        return w;
    };
    tab.L64 = tab.L;
    tab.L32 = tab.L;
    bool have32 = false;
    if (implicit) {
        if (coupling() < 1e-9) {
            tab.L32 = 0;
            have32 = true;
            for (int i = 0; i < N; i++) ib32[i] = 1.0 / b[i];
        }
        for (int lev = 0; lev < L; lev++) {
            int hh = 1 << lev;
            std::vector<double> na(N, 0.0), nb = b, nc(N, 0.0);
            for (int i = 0; i < N; i++) {
                double al = 0.0, ga = 0.0;
                if (i - hh >= 0) {
                    al = -a[i] / b[i - hh];
                    na[i] = al * a[i - hh];
                    nb[i] += al * c[i - hh];
                }
                if (i + hh < N) {
                    ga = -c[i] / b[i + hh];
                    nc[i] = ga * c[i + hh];
                    nb[i] += ga * a[i + hh];
                }
                alpha[(size_t)lev * N + i] = al;
                gamma[(size_t)lev * N + i] = ga;
            }
            a = na;
            b = nb;
            c = nc;
            const double w = coupling();
            if (!have32 && w < 1e-9) {
                tab.L32 = lev + 1;
                have32 = true;
                for (int i = 0; i < N; i++) ib32[i] = 1.0 / b[i];
            }
            if (w < 1e-18) {
                tab.L64 = lev + 1;
                break;
            }
        }
    }
    for (int i = 0; i < N; i++) {
        ib[i] = implicit ? 1.0 / b[i] : 1.0;
        if (!have32) ib32[i] = ib[i];
        zt[i] = z[i];
    }
    size_t nd = h.size();
    std::vector<float> hf(nd);
    for (size_t i = 0; i < nd; i++) hf[i] = (float)h[i];
    tab.bytes = nd * (sizeof(double) + sizeof(float));
    if (cudaMalloc(&tab.dtab, nd * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&tab.ftab, nd * sizeof(float)) != cudaSuccess) {
        free_line_table(tab);
        cudaGetLastError();
        return set_error(WD_ERR_OOM, "cudaMalloc of a line-solve table failed");
    }
    if (cudaMemcpy(tab.dtab, h.data(), nd * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(tab.ftab, hf.data(), nd * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_line_table(tab);
        return set_error(WD_ERR_CUDA, "upload of a line-solve table failed");
    }
    tab.valid = 1;
    build_part_table(N, periodic, a0v, c0v, implicit, tab);
    return WD_OK;
}

void free_line_table(HostLineTab& tab)
{
    if (tab.dtab) cudaFree(tab.dtab);
    if (tab.ftab) cudaFree(tab.ftab);
    if (tab.pdtab) cudaFree(tab.pdtab);
    if (tab.pftab) cudaFree(tab.pftab);
    tab.dtab = nullptr;
    tab.ftab = nullptr;
    tab.pdtab = nullptr;
    tab.pftab = nullptr;
    tab.valid = 0;
    tab.pok = 0;
    tab.bytes = 0;
}

// rows per lane of the partition solve for a line of N rows (0: not supported)
int part_rows(int N, int periodic)
{
    static const int Rs[] = {3, 4, 5, 8, 9, 16, 17, 32, 33, 64};
    for (int R : Rs) {
        if (periodic ? N == 32 * R : N <= 32 * R) return R;
    }
    return 0;
}

// Partition tables of the system a_t x_{t-1} + x_t + c_t x_{t+1} = d_t (periodic: a_0
// couples x_{N-1}, c_{N-1} couples x_0), checked against a direct solve by emulating the
// device algorithm on the host; on any mismatch the line falls back to the PCR passes.
static void build_part_table(int N, int periodic, const std::vector<double>& a0v,
                             const std::vector<double>& c0v, int implicit, HostLineTab& tab)
{
    tab.pok = 0;
    const int R = part_rows(N, periodic);
    if (R < 2) return;
    tab.pR = R;
    const int NP = 32 * R, m = R - 1;
    // full rows, identity padding
    std::vector<double> A(NP, 0.0), B(NP, 1.0), Cc(NP, 0.0);
    for (int i = 0; i < N; i++) {
        A[i] = implicit ? a0v[i] : 0.0;
        Cc[i] = implicit ? c0v[i] : 0.0;
    }
    if (!periodic) {
        A[0] = 0.0;
        Cc[N - 1] = 0.0;
    }
    std::vector<double> loc((size_t)5 * m * 32, 0.0), sep((size_t)13 * 32, 0.0);
    auto L = [&](int c, int k, int lane) -> double& { return loc[((size_t)c * m + k) * 32 + lane]; };
    auto S = [&](int c, int lane) -> double& { return sep[(size_t)c * 32 + lane]; };
    std::vector<double> Pf(32), Pl(32), Qf(32), Ql(32);   // P, Q at the first / last interior row
    for (int l = 0; l < 32; l++) {
        const int r0 = l * R;
        std::vector<double> w(m), g(m), P(m), Q(m);
        for (int k = 0; k < m; k++) {
            const int i = r0 + k;
            const double ak = k > 0 ? A[i] : 0.0;
            w[k] = B[i] - (k > 0 ? ak * g[k - 1] : 0.0);
            g[k] = (k < m - 1 ? Cc[i] : 0.0) / w[k];
            L(0, k, l) = ak;
            L(1, k, l) = 1.0 / w[k];
            L(2, k, l) = g[k];
        }
        // P = T^-1 (-a_{r0} e_0), Q = T^-1 (-c_{r0+m-1} e_{m-1}) by the same factors
        auto tsolve = [&](std::vector<double> r, std::vector<double>& x) {
            std::vector<double> z(m);
            for (int k = 0; k < m; k++) z[k] = (r[k] - (k > 0 ? L(0, k, l) * z[k - 1] : 0.0)) / w[k];
            x.assign(m, 0.0);
            x[m - 1] = z[m - 1];
            for (int k = m - 2; k >= 0; k--) x[k] = z[k] - g[k] * x[k + 1];
        };
        std::vector<double> e(m, 0.0);
        e[0] = -A[r0];
        tsolve(e, P);
        std::fill(e.begin(), e.end(), 0.0);
        e[m - 1] = -Cc[r0 + m - 1];
        tsolve(e, Q);
        for (int k = 0; k < m; k++) {
            L(3, k, l) = P[k];
            L(4, k, l) = Q[k];
        }
        Pf[l] = P[0];
        Pl[l] = P[m - 1];
        Qf[l] = Q[0];
        Ql[l] = Q[m - 1];
    }
    // reduced system of the separators s_l = x_{lR + R - 1}
    std::vector<double> M(32 * 32, 0.0);
    for (int l = 0; l < 32; l++) {
        const int sg = l * R + R - 1, ln = (l + 1) & 31;
        const double as = A[sg], cs = Cc[sg];
        S(0, l) = as;
        S(1, l) = cs;
        M[l * 32 + ((l + 31) & 31)] += as * Pl[l];
        M[l * 32 + l] += B[sg] + as * Ql[l] + cs * Pf[ln];
        M[l * 32 + ln] += cs * Qf[ln];
    }
    for (int lev = 0; lev < 5; lev++) {
        const int h = 1 << lev;
        std::vector<double> Mn(M);
        for (int l = 0; l < 32; l++) {
            const int lm = (l - h) & 31, lp = (l + h) & 31;
            const double al = -M[l * 32 + lm] / M[lm * 32 + lm];
            const double ga = lm == lp ? 0.0 : -M[l * 32 + lp] / M[lp * 32 + lp];
            S(2 + lev, l) = al;
            S(7 + lev, l) = ga;
            for (int c = 0; c < 32; c++) Mn[l * 32 + c] = M[l * 32 + c] + al * M[lm * 32 + c] + ga * M[lp * 32 + c];
        }
        M = Mn;
    }
    for (int l = 0; l < 32; l++) {
        for (int c = 0; c < 32; c++)
            if (c != l && std::fabs(M[l * 32 + c]) > 1e-13 * std::fabs(M[l * 32 + l])) return;
        S(12, l) = 1.0 / M[l * 32 + l];
    }
    // emulate the device solve on a deterministic right-hand side and compare
    std::vector<double> r(NP, 0.0), x(NP, 0.0);
    for (int i = 0; i < N; i++) r[i] = std::sin(0.37 * i + 0.1) + 0.25 * std::cos(1.91 * i);
    {
        std::vector<double> y(NP), D(32), s(32);
        for (int l = 0; l < 32; l++) {
            const int r0 = l * R;
            for (int k = 0; k < m; k++) y[r0 + k] = (r[r0 + k] - L(0, k, l) * (k ? y[r0 + k - 1] : 0.0)) * L(1, k, l);
            for (int k = m - 2; k >= 0; k--) y[r0 + k] -= L(2, k, l) * y[r0 + k + 1];
        }
        for (int l = 0; l < 32; l++) {
            const int ln = (l + 1) & 31;
            D[l] = r[l * R + R - 1] - S(0, l) * y[l * R + m - 1] - S(1, l) * y[ln * R];
        }
        for (int lev = 0; lev < 5; lev++) {
            const int h = 1 << lev;
            std::vector<double> Dn(32);
            for (int l = 0; l < 32; l++)
                Dn[l] = D[l] + S(2 + lev, l) * D[(l - h) & 31] + S(7 + lev, l) * D[(l + h) & 31];
            D = Dn;
        }
        for (int l = 0; l < 32; l++) s[l] = D[l] * S(12, l);
        for (int l = 0; l < 32; l++) {
            const double sp = s[(l + 31) & 31];
            for (int k = 0; k < m; k++) x[l * R + k] = y[l * R + k] + L(3, k, l) * sp + L(4, k, l) * s[l];
            x[l * R + R - 1] = s[l];
        }
    }
    // residual of the full system
    double res = 0.0, sc = 0.0;
    for (int i = 0; i < NP; i++) {
        const double xm = i > 0 ? x[i - 1] : (periodic ? x[NP - 1] : 0.0);
        const double xp = i < NP - 1 ? x[i + 1] : (periodic ? x[0] : 0.0);
        res = std::max(res, std::fabs(A[i] * xm + B[i] * x[i] + Cc[i] * xp - r[i]));
        sc = std::max(sc, std::fabs(r[i]));
    }
    for (int i = N; i < NP; i++) res = std::max(res, std::fabs(x[i]));
    if (!(res <= 1e-12 * (sc > 0 ? sc : 1.0))) return;
    const size_t nd = loc.size() + sep.size();
    std::vector<double> h(nd);
    std::copy(loc.begin(), loc.end(), h.begin());
    std::copy(sep.begin(), sep.end(), h.begin() + loc.size());
    std::vector<float> hf(nd);
    for (size_t i = 0; i < nd; i++) hf[i] = (float)h[i];
    if (cudaMalloc(&tab.pdtab, nd * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&tab.pftab, nd * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaMemcpy(tab.pdtab, h.data(), nd * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(tab.pftab, hf.data(), nd * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    tab.bytes += nd * (sizeof(double) + sizeof(float));
    tab.pok = 1;
}

template <typename T>
static LineTab<T> make_view(const HostLineTab& h, const T* base)
{
    LineTab<T> t;
    int N = h.N, L = h.L;
    t.N = N;
    t.L = L;
    t.implicit = h.implicit;
    t.periodic = h.periodic && h.implicit;
    t.alpha = base;
    t.gamma = base + (size_t)L * N;
    t.ib = base + (size_t)2 * L * N + (sizeof(T) == 4 ? N : 0);
    t.z = base + (size_t)(2 * L + 2) * N;
    t.L = sizeof(T) == 4 ? h.L32 : h.L64;
    t.a0 = T(h.a0);
    t.inv_den = T(h.inv_den);
    return t;
}

template <>
LineTab<double> HostLineTab::view<double>() const { return make_view<double>(*this, dtab); }
template <>
LineTab<float> HostLineTab::view<float>() const { return make_view<float>(*this, ftab); }

}  // namespace wd
