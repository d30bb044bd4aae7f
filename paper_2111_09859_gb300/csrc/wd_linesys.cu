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
    return WD_OK;
}

void free_line_table(HostLineTab& tab)
{
    if (tab.dtab) cudaFree(tab.dtab);
    if (tab.ftab) cudaFree(tab.ftab);
    tab.dtab = nullptr;
    tab.ftab = nullptr;
    tab.valid = 0;
    tab.bytes = 0;
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
