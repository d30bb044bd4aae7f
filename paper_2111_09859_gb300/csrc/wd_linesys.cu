// wd_linesys.cu -- host-side precomputation of the constant-coefficient tridiagonal
// systems solved along grid lines: compact first derivatives (Sec. 3.2.2, Eq. 16) and the
// implicit filter (Sec. 3.4, Eq. 21).
//
// Every system has unit diagonal and constant off-diagonals except in its boundary rows,
// and is the same for every line of a direction, so the whole solve can be factorised
// once per (direction, scheme or alpha_f).  The GPU solves each line with the partition
// (divide-and-conquer) method: the line is cut into P chunks, each thread runs a local
// Thomas sweep on its chunk, and the 2P unknown chunk-end values are obtained from a
// precomputed dense inverse of the reduced system; each chunk then adds the responses to
// its two neighbours' end values.  All factors below are computed in double.
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

// Inverse of an n x n matrix (row-major) by Gauss-Jordan with partial pivoting.
static bool dense_inverse(int n, std::vector<double> A, std::vector<double>& inv)
{
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) inv[(size_t)i * n + i] = 1.0;
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int i = col + 1; i < n; i++)
            if (std::fabs(A[(size_t)i * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = i;
        double p = A[(size_t)piv * n + col];
        if (p == 0.0) return false;
        if (piv != col)
            for (int k = 0; k < n; k++) {
                std::swap(A[(size_t)col * n + k], A[(size_t)piv * n + k]);
                std::swap(inv[(size_t)col * n + k], inv[(size_t)piv * n + k]);
            }
        double ip = 1.0 / A[(size_t)col * n + col];
        for (int k = 0; k < n; k++) {
            A[(size_t)col * n + k] *= ip;
            inv[(size_t)col * n + k] *= ip;
        }
        for (int i = 0; i < n; i++) {
            if (i == col) continue;
            double f = A[(size_t)i * n + col];
            if (f == 0.0) continue;
            for (int k = 0; k < n; k++) {
                A[(size_t)i * n + k] -= f * A[(size_t)col * n + k];
                inv[(size_t)i * n + k] -= f * inv[(size_t)col * n + k];
            }
        }
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

// chunks per line: at most 16 nodes per chunk (the GPU keeps a chunk in registers), at
// least 4 nodes per chunk
int choose_chunks(int N)
{
    int P = (N + 15) / 16;
    if (P < 1) P = 1;
    while (P > 1 && N / P < 4) P--;
    return P;
}

// Builds the partition tables of the system with rows a_t x_{t-1} + x_t + c_t x_{t+1}
// (periodic: a_0 couples x_{N-1} and c_{N-1} couples x_0).
wd_status build_line_table(int N, int periodic, const std::vector<double>& a,
                           const std::vector<double>& c, int implicit, HostLineTab& tab)
{
    free_line_table(tab);
    int P = choose_chunks(N);
    tab.N = N;
    tab.P = P;
    tab.implicit = implicit;
    tab.periodic = periodic;
    std::vector<int> bnd(P + 1);
    for (int ch = 0; ch <= P; ch++) bnd[ch] = (int)((long long)ch * N / P);
    tab.maxm = 0;
    for (int ch = 0; ch < P; ch++) tab.maxm = std::max(tab.maxm, bnd[ch + 1] - bnd[ch]);
    if (tab.maxm > 16) return set_error(WD_ERR_INVALID_ARG, "line chunk longer than 16 nodes");
    size_t nd = (size_t)5 * N + 2 * P + (size_t)4 * P * P;
    std::vector<double> h(nd, 0.0);
    double *la = h.data(), *lib = la + N, *lcp = lib + N, *v = lcp + N, *w = v + N;
    double *acoup = w + N, *ccoup = acoup + P, *Sinv = ccoup + P;
    if (implicit) {
        for (int ch = 0; ch < P; ch++) {
            int s = bnd[ch], e = bnd[ch + 1];
            for (int t = s; t < e; t++) {
                la[t] = (t == s) ? 0.0 : a[t];
                double den = 1.0 - ((t == s) ? 0.0 : a[t] * lcp[t - 1]);
                lib[t] = 1.0 / den;
                lcp[t] = (t < e - 1) ? c[t] * lib[t] : 0.0;
            }
            // responses to unit values in the first and the last row of the chunk
            for (int which = 0; which < 2; which++) {
                double* out = which == 0 ? v : w;
                double prev = 0.0;
                for (int t = s; t < e; t++) {
                    double d = (which == 0 ? (t == s) : (t == e - 1)) ? 1.0 : 0.0;
                    prev = (d - la[t] * prev) * lib[t];
                    out[t] = prev;
                }
                double next = out[e - 1];
                for (int t = e - 2; t >= s; t--) {
                    next = out[t] - lcp[t] * next;
                    out[t] = next;
                }
            }
            acoup[ch] = a[s];
            ccoup[ch] = c[e - 1];
        }
        int n2 = 2 * P;
        std::vector<double> S((size_t)n2 * n2, 0.0), Si;
        for (int i = 0; i < n2; i++) S[(size_t)i * n2 + i] = 1.0;
        for (int ch = 0; ch < P; ch++) {
            int s = bnd[ch], e = bnd[ch + 1];
            int prev = (ch - 1 + P) % P, next = (ch + 1) % P;
            S[(size_t)(2 * ch) * n2 + 2 * prev + 1] += acoup[ch] * v[s];
            S[(size_t)(2 * ch) * n2 + 2 * next] += ccoup[ch] * w[s];
            S[(size_t)(2 * ch + 1) * n2 + 2 * prev + 1] += acoup[ch] * v[e - 1];
            S[(size_t)(2 * ch + 1) * n2 + 2 * next] += ccoup[ch] * w[e - 1];
        }
        if (!dense_inverse(n2, S, Si)) return set_error(WD_ERR_INVALID_ARG, "singular line system");
        std::memcpy(Sinv, Si.data(), sizeof(double) * n2 * n2);
    }
    std::vector<float> hf(nd);
    for (size_t i = 0; i < nd; i++) hf[i] = (float)h[i];
    tab.bytes = nd * (sizeof(double) + sizeof(float)) + (P + 1) * sizeof(int);
    if (cudaMalloc(&tab.bnd, (P + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&tab.dtab, nd * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&tab.ftab, nd * sizeof(float)) != cudaSuccess) {
        free_line_table(tab);
        cudaGetLastError();
        return set_error(WD_ERR_OOM, "cudaMalloc of a line-solve table failed");
    }
    if (cudaMemcpy(tab.bnd, bnd.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(tab.dtab, h.data(), nd * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(tab.ftab, hf.data(), nd * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_line_table(tab);
        return set_error(WD_ERR_CUDA, "upload of a line-solve table failed");
    }
    tab.valid = 1;
    return WD_OK;
}

void free_line_table(HostLineTab& tab)
{
    if (tab.bnd) cudaFree(tab.bnd);
    if (tab.dtab) cudaFree(tab.dtab);
    if (tab.ftab) cudaFree(tab.ftab);
    tab.bnd = nullptr;
    tab.dtab = nullptr;
    tab.ftab = nullptr;
    tab.valid = 0;
    tab.bytes = 0;
}

template <typename T>
static LineTab<T> make_view(const HostLineTab& h, const T* base)
{
    LineTab<T> t;
    int N = h.N, P = h.P;
    t.N = N;
    t.P = P;
    t.implicit = h.implicit;
    t.periodic = h.periodic;
    t.bnd = h.bnd;
    t.la = base;
    t.lib = base + N;
    t.lcp = base + 2 * N;
    t.v = base + 3 * N;
    t.w = base + 4 * N;
    t.acoup = base + 5 * N;
    t.ccoup = base + 5 * N + P;
    t.Sinv = base + 5 * N + 2 * P;
    return t;
}

template <>
LineTab<double> HostLineTab::view<double>() const { return make_view<double>(*this, dtab); }
template <>
LineTab<float> HostLineTab::view<float>() const { return make_view<float>(*this, ftab); }

}  // namespace wd
