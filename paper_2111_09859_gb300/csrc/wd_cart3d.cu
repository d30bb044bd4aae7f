// wd_cart3d.cu -- pseudo-step kernels for uniform Cartesian 3-D grids with explicit schemes
// (E2 / E4 / E6).  The metrics are then the constants d(xi_l)/d(x_m) = delta_lm / h_l, so
//     U_l = D_l(phi) / h_l,   lap(phi) = sum_l D_l(U_l) / h_l   (Eq. 9 with diagonal metrics),
//     LAD term (Eq. 7) = C | sum_l d4_l(phi) s_l |   (s_l = h_l^(exponent - 4)),
// and every pass is a stencil along grid lines read straight from global memory (L1/L2 serve
// the neighbours).  One RK stage = four launches:
//   U   U_0, U_1, U_2 and the raw LAD term,
//   GX  Gaussian of the LAD term along direction 0,
//   GY  Gaussian along direction 1,
//   S   Gaussian along direction 2, Laplacian, Gamma, right-hand side, local time step, RK4
//       stage and the Dirichlet reset.
// Threads are laid out as the grid (x fastest, 32 x 8 per block, one z plane per block row
// of the launch), offsets are 32-bit, and a node whose stencil stays clear of the faces
// takes a branch-free path; the boundary rows are those of the line passes.  The formulas
// and the order of operations are those of the generic path.
#include "wd_api_internal.h"
#include "wd_cart3d.h"

namespace wd {

// Values f[t + o], o = -4 .. 4, of one grid line around node t (index e, stride st): the
// offsets a formula may use are loaded, wrapped on periodic lines; on other lines offsets
// outside the line are left 0 (no formula reads them).
template <typename T>
struct Win {
    T v[9];
    __device__ __forceinline__ T operator()(int o) const { return v[o + 4]; }
};

template <int HW, typename T>
__device__ __forceinline__ void load_win(Win<T>& w, const T* __restrict__ f, int e, int st, int t, int N,
                                         int per)
{
    const bool inner = per ? (t >= HW && t < N - HW) : (t >= 4 && t < N - 4);
    if (inner) {
        const T* p = f + e;
#pragma unroll
        for (int o = -4; o <= 4; o++) w.v[o + 4] = (o >= -HW && o <= HW) ? __ldg(p + o * st) : T(0);
        return;
    }
#pragma unroll
    for (int o = -4; o <= 4; o++) {
        int u = t + o;
        if (per) u = u < 0 ? u + N : (u >= N ? u - N : u);
        const bool ok = per ? (o >= -HW && o <= HW) : (u >= 0 && u < N);
        w.v[o + 4] = ok ? __ldg(f + e + (u - t) * st) : T(0);
    }
}

// explicit first derivative at line index t (Eq. 16 rows; the boundary rows of the line
// passes: one-sided at the end node, centred 2nd order at the next, E4 at the third for E6)
template <int SCH, typename T>
__device__ __forceinline__ T d1w(const Win<T>& w, int t, int N, int per)
{
    constexpr int sch = SCH;
    if (!per) {
        if (t == 0) return (T(-25.0) * w(0) + T(48.0) * w(1) - T(36.0) * w(2) + T(16.0) * w(3) - T(3.0) * w(4)) * T(1.0 / 12.0);
        if (t == N - 1) return -(T(-25.0) * w(0) + T(48.0) * w(-1) - T(36.0) * w(-2) + T(16.0) * w(-3) - T(3.0) * w(-4)) * T(1.0 / 12.0);
        if (t == 1 || t == N - 2) return T(0.5) * (w(1) - w(-1));
    }
    const T a1 = w(1) - w(-1);
    if (sch == WD_E2) return T(0.5) * a1;
    const T a2 = w(2) - w(-2);
    if (sch == WD_E4 || (!per && (t == 2 || t == N - 3))) return T(2.0 / 3.0) * a1 - T(1.0 / 12.0) * a2;
    const T a3 = w(3) - w(-3);
    return T(0.75) * a1 - T(0.15) * a2 + T(1.0 / 60.0) * a3;
}

// 5-point fourth difference (nearest complete stencil near non-periodic ends)
template <typename T>
__device__ __forceinline__ T d4w(const Win<T>& w, int t, int N, int per)
{
    int c = 0;
    if (!per) c = (t < 2 ? 2 : (t > N - 3 ? N - 3 : t)) - t;
    return w(c - 2) - T(4) * w(c - 1) + T(6) * w(c) - T(4) * w(c + 1) + w(c + 2);
}

// truncated 9-point Gaussian (Kawai & Lele), even reflection at non-periodic ends
template <typename T>
__device__ __forceinline__ T gaussw(const Win<T>& w, int t, int N, int per)
{
    const T c[5] = {T(3565.0 / 10368.0), T(3091.0 / 12960.0), T(1997.0 / 25920.0), T(149.0 / 12960.0),
                    T(107.0 / 103680.0)};
    T s = c[0] * w(0);
#pragma unroll
    for (int m = 1; m <= 4; m++) {
        int up = m, um = -m;
        if (!per) {
            if (t + m > N - 1) up = 2 * (N - 1) - t - m - t;
            if (t - m < 0) um = m - 2 * t;
        }
        s += c[m] * (w(up) + w(um));
    }
    return s;
}

struct C3Node {
    int c[3];      // i, j, k
    int e;         // padded index
    int st[3];     // strides
};

template <typename T>
__device__ __forceinline__ bool c3_node(const C3Args<T>& a, C3Node& q)
{
    const Dims& D = a.D;
    q.c[0] = blockIdx.x * 32 + threadIdx.x;
    q.c[1] = blockIdx.y * 8 + threadIdx.y;
    q.c[2] = blockIdx.z;
    if (q.c[0] >= D.n[0] || q.c[1] >= D.n[1]) return false;
    q.st[0] = 1;
    q.st[1] = D.pitch;
    q.st[2] = D.pitch * D.n[1];
    q.e = q.c[0] + q.st[1] * q.c[1] + q.st[2] * q.c[2];
    return true;
}

template <int SCH>
struct C3Half {
    static constexpr int HD = SCH == WD_E6 ? 3 : (SCH == WD_E4 ? 2 : 1);   // derivative
};

template <typename T, int SCH, int LAD>
__global__ void __launch_bounds__(256) k_c3_u(C3Args<T> a)
{
    C3Node q;
    if (!c3_node(a, q)) return;
    const Dims& D = a.D;
    constexpr int HD = C3Half<SCH>::HD;
    constexpr int HW = LAD && HD < 2 ? 2 : HD;
    T lad = T(0);
#pragma unroll
    for (int l = 0; l < 3; l++) {
        Win<T> w;
        load_win<HW>(w, a.src, q.e, q.st[l], q.c[l], D.n[l], D.per[l]);
        (l == 0 ? a.U0 : (l == 1 ? a.U1 : a.U2))[q.e] = d1w<SCH>(w, q.c[l], D.n[l], D.per[l]) * a.ih[l];
        if (LAD) lad += d4w(w, q.c[l], D.n[l], D.per[l]) * a.slad[l];
    }
    if (LAD) a.L[q.e] = a.C_lad * (lad < T(0) ? -lad : lad);
}

template <typename T>
__global__ void __launch_bounds__(256) k_c3_gauss(C3Args<T> a, int d, const T* __restrict__ in, T* out)
{
    C3Node q;
    if (!c3_node(a, q)) return;
    const Dims& D = a.D;
    Win<T> w;
    load_win<4>(w, in, q.e, q.st[d], q.c[d], D.n[d], D.per[d]);
    out[q.e] = gaussw(w, q.c[d], D.n[d], D.per[d]);
}

// EQ: 0 Poisson, 1 standard HJ, 2 LAD HJ, 3 eikonal (Gamma = 0)
template <typename T, int SCH, int EQ>
__global__ void __launch_bounds__(256) k_c3_stage(C3Args<T> a)
{
    C3Node q;
    if (!c3_node(a, q)) return;
    const Dims& D = a.D;
    const int e = q.e;
    constexpr int HD = C3Half<SCH>::HD;
    T lap = T(0);
#pragma unroll
    for (int l = 0; l < 3; l++) {
        Win<T> w;
        load_win<HD>(w, l == 0 ? a.U0 : (l == 1 ? a.U1 : a.U2), e, q.st[l], q.c[l], D.n[l], D.per[l]);
        lap += d1w<SCH>(w, q.c[l], D.n[l], D.per[l]) * a.ih[l];
    }
    T R, gam = T(0), gm = T(0);
    if (EQ == 0) {
        R = T(1) + lap;                                                  // Eq. 19
    } else {
        const T ux = a.U0[e], uy = a.U1[e], uz = a.U2[e];
        const T g2 = ux * ux + uy * uy + uz * uz;
        gm = sqrt(g2);
        const T ph = a.src[e];
        const T php = ph > T(0) ? ph : T(0);
        if (EQ == 1) gam = a.eps * php;                                  // Eq. 6
        else if (EQ == 2) {                                              // Eq. 7
            Win<T> w;
            load_win<4>(w, a.G2, e, q.st[2], q.c[2], D.n[2], D.per[2]);
            const T g1 = a.eps * php, gl = gaussw(w, q.c[2], D.n[2], D.per[2]);
            gam = g1 < gl ? g1 : gl;
        }
        R = T(1) + gam * lap - g2;                                       // Eqs. 5, 18
    }
    T dtv;
    if (a.stage == 0) {
        if (EQ == 0) dtv = a.cfl / a.sig2;
        else {
            const T am = gm > T(1) ? gm : T(1);
            dtv = a.cfl / (a.sig1 * am + gam * a.sig2);
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
    if (a.mask[e]) out = EQ == 0 ? T(0) : a.dval[e];
    a.dst[e] = out;
}

template <typename T, int SCH>
static void c3_launch_s(const C3Args<T>& a, int which, dim3 grd, dim3 blk, cudaStream_t st)
{
    if (which == C3_U) {
        if (a.lad) k_c3_u<T, SCH, 1><<<grd, blk, 0, st>>>(a);
        else k_c3_u<T, SCH, 0><<<grd, blk, 0, st>>>(a);
    } else {
        if (a.poisson) k_c3_stage<T, SCH, 0><<<grd, blk, 0, st>>>(a);
        else if (a.equation == WD_HJ_LAD) k_c3_stage<T, SCH, 2><<<grd, blk, 0, st>>>(a);
        else if (a.equation == WD_HJ_STD) k_c3_stage<T, SCH, 1><<<grd, blk, 0, st>>>(a);
        else k_c3_stage<T, SCH, 3><<<grd, blk, 0, st>>>(a);
    }
}

template <typename T>
cudaError_t c3_launch(const C3Args<T>& a, int which, cudaStream_t st)
{
    const dim3 blk(32, 8, 1);
    const dim3 grd((a.D.n[0] + 31) / 32, (a.D.n[1] + 7) / 8, a.D.n[2]);
    if (which == C3_GX) k_c3_gauss<T><<<grd, blk, 0, st>>>(a, 0, a.L, a.G1);
    else if (which == C3_GY) k_c3_gauss<T><<<grd, blk, 0, st>>>(a, 1, a.G1, a.G2);
    else if (a.scheme == WD_E6) c3_launch_s<T, WD_E6>(a, which, grd, blk, st);
    else if (a.scheme == WD_E4) c3_launch_s<T, WD_E4>(a, which, grd, blk, st);
    else c3_launch_s<T, WD_E2>(a, which, grd, blk, st);
    return cudaGetLastError();
}

template cudaError_t c3_launch<double>(const C3Args<double>&, int, cudaStream_t);
template cudaError_t c3_launch<float>(const C3Args<float>&, int, cudaStream_t);

}  // namespace wd
