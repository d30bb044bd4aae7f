// wd_cart3d.cu -- pseudo-step kernels for uniform Cartesian 3-D grids with explicit schemes
// (E2 / E4 / E6).  The metrics are then the constants d(xi_l)/d(x_m) = delta_lm / h_l, so
//     U_l = D_l(phi) / h_l,   lap(phi) = sum_l D_l(U_l) / h_l   (Eq. 9 with diagonal metrics),
//     LAD term (Eq. 7) = C | sum_l d4_l(phi) / h_l |   (s_l = (1/h_l^2)^2 h_l^3),
// and every pass is a stencil along grid lines read straight from global memory (L1/L2 serve
// the neighbours), with no shared-memory staging or barriers.  One RK stage = four launches:
//   U   U_0, U_1, U_2 and the raw LAD term,
//   GX  Gaussian of the LAD term along direction 0,
//   GY  Gaussian along direction 1,
//   S   Gaussian along direction 2, Laplacian, Gamma, right-hand side, local time step, RK4
//       stage and the Dirichlet reset.
// The formulas, boundary rows and the order of operations are those of the generic path.
#include "wd_api_internal.h"
#include "wd_cart3d.h"

namespace wd {

// node coordinates of padded element e
__device__ __forceinline__ void coords(const Dims& D, long long e, int& i, int& j, int& k)
{
    i = (int)(e % D.pitch);
    const long long r = e / D.pitch;
    j = (int)(r % D.n[1]);
    k = (int)(r / D.n[1]);
}

// value at line offset o from node e along direction d (t = e's index on that line)
template <typename T>
__device__ __forceinline__ T ln(const T* __restrict__ f, long long e, long long st, int t, int o,
                                int N, int per)
{
    int u = t + o;
    if (per) u = u < 0 ? u + N : (u >= N ? u - N : u);
    return __ldg(f + e + (long long)(u - t) * st);
}

// explicit first derivative at line index t (Eq. 16 rows; same boundary rows as the line
// passes: one-sided at the end node, centred 2nd order at the next, E4 at the third for E6)
template <typename T>
__device__ __forceinline__ T d1(const T* __restrict__ f, long long e, long long st, int t, int N,
                                int per, int sch)
{
#define LV(o) ln(f, e, st, t, (o), N, per)
    if (!per) {
        if (t == 0) return (T(-25.0) * LV(0) + T(48.0) * LV(1) - T(36.0) * LV(2) + T(16.0) * LV(3) - T(3.0) * LV(4)) * T(1.0 / 12.0);
        if (t == N - 1) return -(T(-25.0) * LV(0) + T(48.0) * LV(-1) - T(36.0) * LV(-2) + T(16.0) * LV(-3) - T(3.0) * LV(-4)) * T(1.0 / 12.0);
        if (t == 1 || t == N - 2) return T(0.5) * (LV(1) - LV(-1));
    }
    const T a1 = LV(1) - LV(-1);
    if (sch == WD_E2) return T(0.5) * a1;
    const T a2 = LV(2) - LV(-2);
    if (sch == WD_E4 || (!per && (t == 2 || t == N - 3))) return T(2.0 / 3.0) * a1 - T(1.0 / 12.0) * a2;
    const T a3 = LV(3) - LV(-3);
    return T(0.75) * a1 - T(0.15) * a2 + T(1.0 / 60.0) * a3;
#undef LV
}

// 5-point fourth difference (nearest complete stencil near non-periodic ends)
template <typename T>
__device__ __forceinline__ T d4(const T* __restrict__ f, long long e, long long st, int t, int N, int per)
{
    int c = t;
    if (!per) c = c < 2 ? 2 : (c > N - 3 ? N - 3 : c);
    const long long ec = e + (long long)(c - t) * st;
    return ln(f, ec, st, c, -2, N, per) - T(4) * ln(f, ec, st, c, -1, N, per) + T(6) * __ldg(f + ec)
         - T(4) * ln(f, ec, st, c, 1, N, per) + ln(f, ec, st, c, 2, N, per);
}

// truncated 9-point Gaussian (Kawai & Lele), even reflection at non-periodic ends
template <typename T>
__device__ __forceinline__ T gauss(const T* __restrict__ f, long long e, long long st, int t, int N, int per)
{
    const T w[5] = {T(3565.0 / 10368.0), T(3091.0 / 12960.0), T(1997.0 / 25920.0), T(149.0 / 12960.0),
                    T(107.0 / 103680.0)};
    T s = w[0] * __ldg(f + e);
#pragma unroll
    for (int m = 1; m <= 4; m++) {
        int up = t + m, um = t - m;
        if (per) {
            up = up >= N ? up - N : up;
            um = um < 0 ? um + N : um;
        } else {
            up = up > N - 1 ? 2 * (N - 1) - up : up;
            um = um < 0 ? -um : um;
        }
        s += w[m] * (__ldg(f + e + (long long)(up - t) * st) + __ldg(f + e + (long long)(um - t) * st));
    }
    return s;
}

#define C3_LOOP(D)                                                                           \
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (D).total;      \
         e += (long long)gridDim.x * blockDim.x)

template <typename T>
__global__ void __launch_bounds__(256) k_c3_u(C3Args<T> a)
{
    const Dims& D = a.D;
    const long long st[3] = {1, D.stride(1), D.stride(2)};
    C3_LOOP(D)
    {
        int c[3];
        coords(D, e, c[0], c[1], c[2]);
        if (c[0] >= D.n[0]) continue;
        T lad = T(0);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            const T u = d1(a.src, e, st[l], c[l], D.n[l], D.per[l], a.scheme) * T(a.ih[l]);
            (l == 0 ? a.U0 : (l == 1 ? a.U1 : a.U2))[e] = u;
            if (a.lad) lad += d4(a.src, e, st[l], c[l], D.n[l], D.per[l]) * T(a.slad[l]);
        }
        if (a.lad) a.L[e] = T(a.C_lad) * (lad < T(0) ? -lad : lad);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_c3_gauss(C3Args<T> a, int d, const T* __restrict__ in, T* out)
{
    const Dims& D = a.D;
    const long long st = D.stride(d);
    C3_LOOP(D)
    {
        int c[3];
        coords(D, e, c[0], c[1], c[2]);
        if (c[0] >= D.n[0]) continue;
        out[e] = gauss(in, e, st, c[d], D.n[d], D.per[d]);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_c3_stage(C3Args<T> a)
{
    const Dims& D = a.D;
    const long long st[3] = {1, D.stride(1), D.stride(2)};
    C3_LOOP(D)
    {
        int c[3];
        coords(D, e, c[0], c[1], c[2]);
        if (c[0] >= D.n[0]) continue;
        T lap = T(0);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            const T* U = l == 0 ? a.U0 : (l == 1 ? a.U1 : a.U2);
            lap += d1(U, e, st[l], c[l], D.n[l], D.per[l], a.scheme) * T(a.ih[l]);
        }
        T R, gam = T(0), gm = T(0);
        if (a.poisson) {
            R = T(1) + lap;                                                  // Eq. 19
        } else {
            const T ux = a.U0[e], uy = a.U1[e], uz = a.U2[e];
            const T g2 = ux * ux + uy * uy + uz * uz;
            gm = sqrt(g2);
            const T ph = a.src[e];
            const T php = ph > T(0) ? ph : T(0);
            if (a.equation == WD_HJ_STD) gam = T(a.eps) * php;               // Eq. 6
            else if (a.equation == WD_HJ_LAD) {                              // Eq. 7
                const T g1 = T(a.eps) * php, gl = gauss(a.G2, e, st[2], c[2], D.n[2], D.per[2]);
                gam = g1 < gl ? g1 : gl;
            }
            R = T(1) + gam * lap - g2;                                       // Eqs. 5, 18
        }
        T dtv;
        if (a.stage == 0) {
            if (a.poisson) dtv = T(a.cfl) / T(a.sig2);
            else {
                const T am = gm > T(1) ? gm : T(1);
                dtv = T(a.cfl) / (T(a.sig1) * am + gam * T(a.sig2));
            }
            a.dtv[e] = dtv;
        } else {
            dtv = a.dtv[e];
        }
        const T n = a.phin[e];
        T out;
        if (a.stage == 0) {
            a.acc[e] = R * T(1.0 / 6.0);
            out = n + T(0.5) * dtv * R;
        } else if (a.stage == 1) {
            a.acc[e] += R * T(1.0 / 3.0);
            out = n + T(0.5) * dtv * R;
        } else if (a.stage == 2) {
            a.acc[e] += R * T(1.0 / 3.0);
            out = n + dtv * R;
        } else {
            out = n + dtv * (a.acc[e] + R * T(1.0 / 6.0));
        }
        if (a.mask[e]) out = a.poisson ? T(0) : a.dval[e];
        a.dst[e] = out;
    }
}

static int c3_grid(long long total)
{
    long long b = (total + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t c3_launch(const C3Args<T>& a, int which, cudaStream_t st)
{
    const int gb = c3_grid(a.D.total);
    switch (which) {
    case C3_U: k_c3_u<T><<<gb, 256, 0, st>>>(a); break;
    case C3_GX: k_c3_gauss<T><<<gb, 256, 0, st>>>(a, 0, a.L, a.G1); break;
    case C3_GY: k_c3_gauss<T><<<gb, 256, 0, st>>>(a, 1, a.G1, a.G2); break;
    default: k_c3_stage<T><<<gb, 256, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

template cudaError_t c3_launch<double>(const C3Args<double>&, int, cudaStream_t);
template cudaError_t c3_launch<float>(const C3Args<float>&, int, cudaStream_t);

}  // namespace wd
