// wd_cart3d.cu -- pseudo-step kernels for uniform Cartesian grids (3-D, and single 2-D grids
// whose faces rule out the fused 2-D path) with explicit schemes (E2 / E4 / E6).  The metrics are then the constants d(xi_l)/d(x_m) = delta_lm / h_l, so
//     U_l = D_l(phi) / h_l,   lap(phi) = sum_l D_l(U_l) / h_l   (Eq. 9 with diagonal metrics),
//     LAD term (Eq. 7) = C | sum_l d4_l(phi) s_l |   (s_l = h_l^(exponent - 4)),
// and every pass is a stencil along grid lines read straight from global memory (L1/L2 serve
// the neighbours).  One RK stage = three launches:
//   U   U_0, U_1, U_2 and the raw LAD term,
//   GXY Gaussian of the LAD term along directions 0 and 1 (one tiled pass; in 2-D: GX, along 0),
//   S   Gaussian along direction 2, Laplacian, Gamma, right-hand side, local time step, RK4
//       stage and the Dirichlet reset.
// Threads are laid out as the grid (x fastest, 32 x by per block (by autotuned), one z plane per block row
// of the launch), offsets are 32-bit, and a node whose stencil stays clear of the faces
// takes a branch-free path; the boundary rows are those of the line passes.  The formulas
// and the order of operations are those of the generic path.
#include "wd_api_internal.h"
#include "wd_cart3d.h"

#include <type_traits>

namespace wd {

// Line helpers.  A node whose stencil stays inside its line (or any node of a periodic line
// away from the wrap) loads its neighbours at constant offsets; the few nodes near a face
// (or the wrap) evaluate the same formulas with computed indices straight from memory.

template <typename T>
__device__ __forceinline__ T ld(const T* __restrict__ f, int e, int st, int t, int u, int N, int per)
{
    if (per) u = u < 0 ? u + N : (u >= N ? u - N : u);
    return __ldg(f + e + (u - t) * st);
}

// first derivative of Eq. 16 at line index t with its boundary rows (one-sided at the end
// node, centred 2nd order at the next, E4 at the third for E6); slow path
template <int SCH, typename T>
__device__ T d1_edge(const T* __restrict__ f, int e, int st, int t, int N, int per)
{
#define LV(u) ld(f, e, st, t, (u), N, per)
    if (!per) {
        if (t == 0) return (T(-25.0) * LV(0) + T(48.0) * LV(1) - T(36.0) * LV(2) + T(16.0) * LV(3) - T(3.0) * LV(4)) * T(1.0 / 12.0);
        if (t == N - 1)
            return -(T(-25.0) * LV(N - 1) + T(48.0) * LV(N - 2) - T(36.0) * LV(N - 3) + T(16.0) * LV(N - 4) - T(3.0) * LV(N - 5)) * T(1.0 / 12.0);
        if (t == 1 || t == N - 2) return T(0.5) * (LV(t + 1) - LV(t - 1));
    }
    const T a1 = LV(t + 1) - LV(t - 1);
    if (SCH == WD_E2) return T(0.5) * a1;
    const T a2 = LV(t + 2) - LV(t - 2);
    if (SCH == WD_E4 || (!per && (t == 2 || t == N - 3))) return T(2.0 / 3.0) * a1 - T(1.0 / 12.0) * a2;
    const T a3 = LV(t + 3) - LV(t - 3);
    return T(0.75) * a1 - T(0.15) * a2 + T(1.0 / 60.0) * a3;
}

// 5-point fourth difference, nearest complete stencil near non-periodic ends; slow path
template <typename T>
__device__ T d4_edge(const T* __restrict__ f, int e, int st, int t, int N, int per)
{
    int c = t;
    if (!per) c = c < 2 ? 2 : (c > N - 3 ? N - 3 : c);
    return LV(c - 2) - T(4) * LV(c - 1) + T(6) * LV(c) - T(4) * LV(c + 1) + LV(c + 2);
}

// truncated 9-point Gaussian (Kawai & Lele), even reflection at non-periodic ends; slow path
template <typename T>
__device__ T gauss_edge(const T* __restrict__ f, int e, int st, int t, int N, int per)
{
    const T c[5] = {T(3565.0 / 10368.0), T(3091.0 / 12960.0), T(1997.0 / 25920.0), T(149.0 / 12960.0),
                    T(107.0 / 103680.0)};
    T s = c[0] * LV(t);
    for (int m = 1; m <= 4; m++) {
        int up = t + m, um = t - m;
        if (!per) {
            up = up > N - 1 ? 2 * (N - 1) - up : up;
            um = um < 0 ? -um : um;
        }
        s += c[m] * (LV(up) + LV(um));
    }
    return s;
#undef LV
}

// interior values f[t + o], |o| <= H, at constant offsets
template <int H, typename T>
__device__ __forceinline__ void win(T (&v)[2 * H + 1], const T* __restrict__ f, int e, int st)
{
    const T* p = f + e;
#pragma unroll
    for (int o = -H; o <= H; o++) v[o + H] = __ldg(p + o * st);
}

template <int SCH, int H, typename T>
__device__ __forceinline__ T d1_in(const T (&v)[2 * H + 1])
{
    const T a1 = v[H + 1] - v[H - 1];
    if (SCH == WD_E2) return T(0.5) * a1;
    const T a2 = v[H + 2] - v[H - 2];
    if (SCH == WD_E4) return T(2.0 / 3.0) * a1 - T(1.0 / 12.0) * a2;
    const T a3 = v[H + 3] - v[H - 3];
    return T(0.75) * a1 - T(0.15) * a2 + T(1.0 / 60.0) * a3;
}

template <int H, typename T>
__device__ __forceinline__ T d4_in(const T (&v)[2 * H + 1])
{
    return v[H - 2] - T(4) * v[H - 1] + T(6) * v[H] - T(4) * v[H + 1] + v[H + 2];
}

template <typename T>
__device__ __forceinline__ T gauss_in(const T (&v)[9])
{
    return T(3565.0 / 10368.0) * v[4] + T(3091.0 / 12960.0) * (v[5] + v[3]) + T(1997.0 / 25920.0) * (v[6] + v[2])
         + T(149.0 / 12960.0) * (v[7] + v[1]) + T(107.0 / 103680.0) * (v[8] + v[0]);
}

// whether node t's stencil of half width H (and the one-sided rows, which reach 4) stays clear
// of the ends of a non-periodic line, or of the wrap of a periodic one
template <int H>
__device__ __forceinline__ bool inner(int t, int N, int per)
{
    return per ? (t >= H && t < N - H) : (t >= 4 && t < N - 4);
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
    q.c[1] = blockIdx.y * blockDim.y + threadIdx.y;
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

// U_0..2 (and the raw LAD term) of one node
template <typename T, int ND, int SCH, int LAD>
__device__ __forceinline__ void c3_u_node(const C3Args<T>& a, const C3Node& q)
{
    const Dims& D = a.D;
    constexpr int HD = C3Half<SCH>::HD;
    constexpr int H = LAD && HD < 2 ? 2 : HD;
    T lad = T(0);
#pragma unroll
    for (int l = 0; l < ND; l++) {
        const int t = q.c[l], N = D.n[l], per = D.per[l];
        T d1, d4 = T(0);
        if (inner<H>(t, N, per)) {
            T v[2 * H + 1];
            win<H>(v, a.src, q.e, q.st[l]);
            d1 = d1_in<SCH, H>(v);
            if (LAD) d4 = d4_in<H>(v);
        } else {
            d1 = d1_edge<SCH>(a.src, q.e, q.st[l], t, N, per);
            if (LAD) d4 = d4_edge(a.src, q.e, q.st[l], t, N, per);
        }
        (l == 0 ? a.U0 : (l == 1 ? a.U1 : a.U2))[q.e] = d1 * a.ih[l];
        if (LAD) lad += d4 * a.slad[l];
    }
    if (LAD) a.L[q.e] = a.C_lad * (lad < T(0) ? -lad : lad);
}

template <typename T, int ND, int SCH, int LAD>
__global__ void __launch_bounds__(512) k_c3_u(C3Args<T> a)
{
    C3Node q;
    if (!c3_node(a, q)) return;
    c3_u_node<T, ND, SCH, LAD>(a, q);
}

template <typename T>
__global__ void __launch_bounds__(512) k_c3_gauss(C3Args<T> a, int d, const T* __restrict__ in, T* out)
{
    C3Node q;
    if (!c3_node(a, q)) return;
    const Dims& D = a.D;
    const int t = q.c[d], N = D.n[d], per = D.per[d];
    T g;
    if (inner<4>(t, N, per)) {
        T v[9];
        win<4>(v, in, q.e, q.st[d]);
        g = gauss_in(v);
    } else {
        g = gauss_edge(in, q.e, q.st[d], t, N, per);
    }
    out[q.e] = g;
}

// Gaussians along directions 0 and 1 in one pass: a 32 x 32 tile of one z plane loads the LAD
// term with a halo of 4 nodes (wrapped on periodic directions, reflected at the others),
// smooths along x into shared memory for the tile's rows and the 4 halo rows on either side,
// then along y; the result equals the two separate passes.
template <typename T>
__device__ __forceinline__ int halo_index(int u, int N, int per)
{
    if (per) return u < 0 ? u + N : (u >= N ? u - N : u);
    u = u < 0 ? -u : u;
    return u > N - 1 ? 2 * (N - 1) - u : u;
}

constexpr int GXY_TY = 32;   // tile rows (4 consecutive per thread of a 32 x 8 block)
constexpr int GXY_LS = 44;   // row stride of the tile + halo (40 used; 16-byte rows)

template <typename T>
__device__ __forceinline__ T gauss9(const T* v)   // v[0..8] centred on v[4]
{
    return T(3565.0 / 10368.0) * v[4] + T(3091.0 / 12960.0) * (v[5] + v[3]) + T(1997.0 / 25920.0) * (v[6] + v[2]) +
           T(149.0 / 12960.0) * (v[7] + v[1]) + T(107.0 / 103680.0) * (v[8] + v[0]);
}

// Each smoothing phase gives a thread 4 neighbouring outputs from a 12-value window in
// registers: along x 4 consecutive columns of a row (three 16-byte shared loads in FP32),
// along y 4 consecutive rows of a column.
template <typename T>
__global__ void __launch_bounds__(256) k_c3_gauss_xy(C3Args<T> a)
{
    __shared__ __align__(16) T Ls[GXY_TY + 8][GXY_LS];
    __shared__ T Gx[GXY_TY + 8][33];
    const Dims& D = a.D;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * GXY_TY, k = blockIdx.z;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int st1 = D.pitch, st2 = D.pitch * D.n[1];
    const T* Lk = a.L + (size_t)st2 * k;
    // the tile + halo: in 16-byte groups of 4 columns where every group is whole (FP32 rows of a
    // periodic direction 0 of a multiple of 4 nodes, the groups wrapped by whole periods, or a
    // tile whose halo stays inside the row), else node by node
    bool vec = false;
    if constexpr (std::is_same<T, float>::value)
        vec = a.vec && (D.per[0] ? D.n[0] % 4 == 0 : (i0 >= 4 && i0 + 36 <= D.n[0]));
    if (vec) {
        if constexpr (std::is_same<T, float>::value)
            for (int q = tid; q < (GXY_TY + 8) * 10; q += 256) {
                const int r = q / 10, c4 = q - r * 10;
                const int gj = halo_index<T>(j0 - 4 + r, D.n[1], D.per[1]);
                int gx = i0 - 4 + 4 * c4;
                if (D.per[0]) gx = ((gx % D.n[0]) + D.n[0]) % D.n[0];
                *reinterpret_cast<float4*>(&Ls[r][4 * c4]) = __ldg(reinterpret_cast<const float4*>(Lk + gx + st1 * gj));
            }
    } else {
        for (int q = tid; q < (GXY_TY + 8) * 40; q += 256) {
            const int r = q / 40, c = q - r * 40;
            const int gi = halo_index<T>(i0 - 4 + c, D.n[0], D.per[0]);
            const int gj = halo_index<T>(j0 - 4 + r, D.n[1], D.per[1]);
            Ls[r][c] = __ldg(Lk + gi + st1 * gj);
        }
    }
    __syncthreads();
    // along x: rows 0 .. GXY_TY + 7, columns 4 c4 .. 4 c4 + 3 (c4 < 8)
    for (int q = tid; q < (GXY_TY + 8) * 8; q += 256) {
        const int r = q >> 3, c4 = q & 7;
        T v[12];
        if constexpr (std::is_same<T, float>::value) {
#pragma unroll
            for (int u = 0; u < 3; u++) {
                const float4 t = *reinterpret_cast<const float4*>(&Ls[r][4 * c4 + 4 * u]);
                v[4 * u] = t.x, v[4 * u + 1] = t.y, v[4 * u + 2] = t.z, v[4 * u + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 12; u++) v[u] = Ls[r][4 * c4 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) Gx[r][4 * c4 + u] = gauss9(v + u);
    }
    __syncthreads();
    // along y: column threadIdx.x, rows 4 threadIdx.y .. 4 threadIdx.y + 3 of the tile
    const int i = i0 + threadIdx.x;
    if (i >= D.n[0]) return;
    const int c = threadIdx.x, r0 = 4 * threadIdx.y;
    T v[12];
#pragma unroll
    for (int u = 0; u < 12; u++) v[u] = Gx[r0 + u][c];
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int j = j0 + r0 + u;
        if (j < D.n[1]) a.G2[i + st1 * j + (size_t)st2 * k] = gauss9(v + u);
    }
}

// the stage of one node; EQ: 0 Poisson, 1 standard HJ, 2 LAD HJ, 3 eikonal (Gamma = 0)
template <typename T, int ND, int SCH, int EQ>
__device__ __forceinline__ void c3_stage_node(const C3Args<T>& a, const C3Node& q)
{
    const Dims& D = a.D;
    const int e = q.e;
    constexpr int HD = C3Half<SCH>::HD;
    T lap = T(0);
#pragma unroll
    for (int l = 0; l < ND; l++) {
        const T* U = l == 0 ? a.U0 : (l == 1 ? a.U1 : a.U2);
        const int t = q.c[l], N = D.n[l], per = D.per[l];
        T d1;
        if (inner<HD>(t, N, per)) {
            T v[2 * HD + 1];
            win<HD>(v, U, e, q.st[l]);
            d1 = d1_in<SCH, HD>(v);
        } else {
            d1 = d1_edge<SCH>(U, e, q.st[l], t, N, per);
        }
        lap += d1 * a.ih[l];
    }
    T R, gam = T(0), gm = T(0);
    if (EQ == 0) {
        R = T(1) + lap;                                                  // Eq. 19
    } else {
        const T ux = __ldg(a.U0 + e), uy = __ldg(a.U1 + e), uz = ND == 3 ? __ldg(a.U2 + e) : T(0);
        const T g2 = ux * ux + uy * uy + uz * uz;
        gm = sqrt(g2);
        const T ph = a.src[e];   // also the stage output array (own node only)
        const T php = ph > T(0) ? ph : T(0);
        if (EQ == 1) gam = a.eps * php;                                  // Eq. 6
        else if (EQ == 2) {                                              // Eq. 7
            // the last direction's half of the separable Gaussian
            constexpr int L = ND - 1;
            const T* G = ND == 3 ? a.G2 : a.G1;
            const int t = q.c[L], N = D.n[L], per = D.per[L];
            T gl;
            if (inner<4>(t, N, per)) {
                T v[9];
                win<4>(v, G, e, q.st[L]);
                gl = gauss_in(v);
            } else {
                gl = gauss_edge(G, e, q.st[L], t, N, per);
            }
            const T g1 = a.eps * php;
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
    const T n = __ldg(a.phin + e);
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
    if (__ldg(a.mask + e)) out = EQ == 0 ? T(0) : __ldg(a.dval + e);
    a.dst[e] = out;
}

template <typename T, int ND, int SCH, int EQ>
__global__ void __launch_bounds__(512) k_c3_stage(C3Args<T> a)
{
    C3Node q;
    if (!c3_node(a, q)) return;
    c3_stage_node<T, ND, SCH, EQ>(a, q);
}

// ---- 4-wide passes (FP32, 3-D) ---------------------------------------------------------------
// The U and stage passes with 4 consecutive x nodes per thread: every stencil row is one
// 16-byte load (along x the node's group of 4 and its two neighbour groups; along y and z one
// group per offset), about a quarter of the load instructions of the per-node passes.  A
// group whose stencils along every direction are interior rows takes this path with the same
// formulas in the same order (on a periodic row of a multiple of 4 nodes the groups at the
// wrap too, with the neighbour group taken from the other end of the row); the others (within
// 4 nodes of a non-periodic face, and rows of other lengths along x) evaluate each node with
// the per-node bodies above.
// Rows must start on 16-byte boundaries: a pitch that is a multiple of 4.

__device__ __forceinline__ void ld4(float* v, const float* p)
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}

__device__ __forceinline__ void ldg4(float* v, const float* p)
{
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}

__device__ __forceinline__ void st4(float* p, const float* v)
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// the first node of this thread's group of 4; false when the group starts outside the grid
__device__ __forceinline__ bool c3_node4(const C3Args<float>& a, C3Node& q)
{
    const Dims& D = a.D;
    q.c[0] = 4 * (blockIdx.x * 32 + threadIdx.x);
    q.c[1] = blockIdx.y * blockDim.y + threadIdx.y;
    q.c[2] = blockIdx.z;
    if (q.c[0] >= D.n[0] || q.c[1] >= D.n[1]) return false;
    q.st[0] = 1;
    q.st[1] = D.pitch;
    q.st[2] = D.pitch * D.n[1];
    q.e = q.c[0] + q.st[1] * q.c[1] + q.st[2] * q.c[2];
    return true;
}

// whether the group's x stencils are interior rows, and the element offsets of its left and
// right neighbour groups: on a periodic row of a multiple of 4 nodes every group qualifies,
// its neighbours wrapped to the other end of the row (so all nodes of a row take one path)
__device__ __forceinline__ bool c3_x4(const Dims& D, int i, int& xl, int& xr)
{
    xl = -4;
    xr = 4;
    if (D.per[0] && D.n[0] % 4 == 0) {
        if (i == 0) xl = D.n[0] - 4;
        if (i + 4 == D.n[0]) xr = 4 - D.n[0];
        return true;
    }
    return i >= 4 && i + 8 <= D.n[0];
}

// node n (0..3) of the group
__device__ __forceinline__ C3Node c3_sub(const C3Node& q, int n)
{
    C3Node r = q;
    r.c[0] += n;
    r.e += n;
    return r;
}

template <int SCH, int LAD>
__global__ void __launch_bounds__(512) k_c3_u4(C3Args<float> a)
{
    C3Node q;
    if (!c3_node4(a, q)) return;
    const Dims& D = a.D;
    constexpr int HD = C3Half<SCH>::HD;
    constexpr int H = LAD && HD < 2 ? 2 : HD;
    int xl, xr;
    if (!(c3_x4(D, q.c[0], xl, xr) && inner<H>(q.c[1], D.n[1], D.per[1]) && inner<H>(q.c[2], D.n[2], D.per[2]))) {
        for (int n = 0; n < 4; n++)
            if (q.c[0] + n < D.n[0]) c3_u_node<float, 3, SCH, LAD>(a, c3_sub(q, n));
        return;
    }
    float lad[4] = {0.f, 0.f, 0.f, 0.f};
    {
        float v[12];
        ldg4(v, a.src + q.e + xl);
        ldg4(v + 4, a.src + q.e);
        ldg4(v + 8, a.src + q.e + xr);
        float u[4];
#pragma unroll
        for (int n = 0; n < 4; n++) {
            float w[2 * H + 1];
#pragma unroll
            for (int o = -H; o <= H; o++) w[o + H] = v[4 + n + o];
            u[n] = d1_in<SCH, H>(w) * a.ih[0];
            if (LAD) lad[n] += d4_in<H>(w) * a.slad[0];
        }
        st4(a.U0 + q.e, u);
    }
#pragma unroll
    for (int l = 1; l < 3; l++) {
        float v[2 * H + 1][4];
#pragma unroll
        for (int o = -H; o <= H; o++) ldg4(v[o + H], a.src + q.e + o * q.st[l]);
        float u[4];
#pragma unroll
        for (int n = 0; n < 4; n++) {
            float w[2 * H + 1];
#pragma unroll
            for (int o = 0; o <= 2 * H; o++) w[o] = v[o][n];
            u[n] = d1_in<SCH, H>(w) * a.ih[l];
            if (LAD) lad[n] += d4_in<H>(w) * a.slad[l];
        }
        st4(l == 1 ? a.U1 + q.e : a.U2 + q.e, u);
    }
    if (LAD) {
#pragma unroll
        for (int n = 0; n < 4; n++) lad[n] = a.C_lad * (lad[n] < 0.f ? -lad[n] : lad[n]);
        st4(a.L + q.e, lad);
    }
}

template <int SCH, int EQ>
__global__ void __launch_bounds__(512) k_c3_stage4(C3Args<float> a)
{
    using T = float;
    C3Node q;
    if (!c3_node4(a, q)) return;
    const Dims& D = a.D;
    constexpr int HD = C3Half<SCH>::HD;
    int xl, xr;
    bool fast = c3_x4(D, q.c[0], xl, xr) && inner<HD>(q.c[1], D.n[1], D.per[1]) && inner<HD>(q.c[2], D.n[2], D.per[2]);
    if (EQ == 2) fast = fast && inner<4>(q.c[2], D.n[2], D.per[2]);
    if (!fast) {
        for (int n = 0; n < 4; n++)
            if (q.c[0] + n < D.n[0]) c3_stage_node<float, 3, SCH, EQ>(a, c3_sub(q, n));
        return;
    }
    const int e = q.e;
    T lap[4] = {0.f, 0.f, 0.f, 0.f}, uo[3][4];
    {
        float v[12];
        ldg4(v, a.U0 + e + xl);
        ldg4(v + 4, a.U0 + e);
        ldg4(v + 8, a.U0 + e + xr);
#pragma unroll
        for (int n = 0; n < 4; n++) {
            float w[2 * HD + 1];
#pragma unroll
            for (int o = -HD; o <= HD; o++) w[o + HD] = v[4 + n + o];
            lap[n] += d1_in<SCH, HD>(w) * a.ih[0];
            uo[0][n] = v[4 + n];
        }
    }
#pragma unroll
    for (int l = 1; l < 3; l++) {
        const T* U = l == 1 ? a.U1 : a.U2;
        float v[2 * HD + 1][4];
#pragma unroll
        for (int o = -HD; o <= HD; o++) ldg4(v[o + HD], U + e + o * q.st[l]);
#pragma unroll
        for (int n = 0; n < 4; n++) {
            float w[2 * HD + 1];
#pragma unroll
            for (int o = 0; o <= 2 * HD; o++) w[o] = v[o][n];
            lap[n] += d1_in<SCH, HD>(w) * a.ih[l];
            uo[l][n] = v[HD][n];
        }
    }
    T gl[4];
    if (EQ == 2) {
        float v[9][4];
#pragma unroll
        for (int o = -4; o <= 4; o++) ldg4(v[o + 4], a.G2 + e + o * q.st[2]);
#pragma unroll
        for (int n = 0; n < 4; n++) {
            float w[9];
#pragma unroll
            for (int o = 0; o < 9; o++) w[o] = v[o][n];
            gl[n] = gauss_in(w);
        }
    }
    T ph[4], pn[4], dt[4], ac[4], dv[4];
    if (EQ != 0) ld4(ph, a.src + e);   // also the stage output array (own nodes only)
    ldg4(pn, a.phin + e);
    if (a.stage > 0) {
        ld4(dt, a.dtv + e);
        ld4(ac, a.acc + e);
    }
    const uchar4 mk = __ldg(reinterpret_cast<const uchar4*>(a.mask + e));
    const unsigned char mv[4] = {mk.x, mk.y, mk.z, mk.w};
    if (EQ != 0 && (mv[0] | mv[1] | mv[2] | mv[3])) ldg4(dv, a.dval + e);   // read only where used
    T out[4];
#pragma unroll
    for (int n = 0; n < 4; n++) {
        T R, gam = T(0), gm = T(0);
        if (EQ == 0) {
            R = T(1) + lap[n];                                               // Eq. 19
        } else {
            const T ux = uo[0][n], uy = uo[1][n], uz = uo[2][n];
            const T g2 = ux * ux + uy * uy + uz * uz;
            gm = sqrt(g2);
            const T php = ph[n] > T(0) ? ph[n] : T(0);
            if (EQ == 1) gam = a.eps * php;                                  // Eq. 6
            else if (EQ == 2) {                                              // Eq. 7
                const T g1 = a.eps * php;
                gam = g1 < gl[n] ? g1 : gl[n];
            }
            R = T(1) + gam * lap[n] - g2;                                    // Eqs. 5, 18
        }
        T dtv;
        if (a.stage == 0) {
            if (EQ == 0) dtv = a.cfl / a.sig2;
            else {
                const T am = gm > T(1) ? gm : T(1);
                dtv = a.cfl / (a.sig1 * am + gam * a.sig2);
            }
            dt[n] = dtv;
        } else {
            dtv = dt[n];
        }
        const T nn = pn[n];
        if (a.stage == 0) {
            ac[n] = R * T(1.0 / 6.0);
            out[n] = nn + T(0.5) * dtv * R;
        } else if (a.stage == 1) {
            ac[n] += R * T(1.0 / 3.0);
            out[n] = nn + T(0.5) * dtv * R;
        } else if (a.stage == 2) {
            ac[n] += R * T(1.0 / 3.0);
            out[n] = nn + dtv * R;
        } else {
            out[n] = nn + dtv * (ac[n] + R * T(1.0 / 6.0));
        }
        if (mv[n]) out[n] = EQ == 0 ? T(0) : dv[n];
    }
    if (a.stage == 0) st4(a.dtv + e, dt);
    if (a.stage < 3) st4(a.acc + e, ac);
    st4(a.dst + e, out);
}

template <int SCH>
static void c3_launch_v4(const C3Args<float>& a, int which, dim3 grd, dim3 blk, cudaStream_t st)
{
    if (which == C3_U) {
        if (a.lad) k_c3_u4<SCH, 1><<<grd, blk, 0, st>>>(a);
        else k_c3_u4<SCH, 0><<<grd, blk, 0, st>>>(a);
    } else {
        if (a.poisson) k_c3_stage4<SCH, 0><<<grd, blk, 0, st>>>(a);
        else if (a.equation == WD_HJ_LAD) k_c3_stage4<SCH, 2><<<grd, blk, 0, st>>>(a);
        else if (a.equation == WD_HJ_STD) k_c3_stage4<SCH, 1><<<grd, blk, 0, st>>>(a);
        else k_c3_stage4<SCH, 3><<<grd, blk, 0, st>>>(a);
    }
}

template <typename T, int ND, int SCH>
static void c3_launch_s(const C3Args<T>& a, int which, dim3 grd, dim3 blk, cudaStream_t st)
{
    if (which == C3_U) {
        if (a.lad) k_c3_u<T, ND, SCH, 1><<<grd, blk, 0, st>>>(a);
        else k_c3_u<T, ND, SCH, 0><<<grd, blk, 0, st>>>(a);
    } else {
        if (a.poisson) k_c3_stage<T, ND, SCH, 0><<<grd, blk, 0, st>>>(a);
        else if (a.equation == WD_HJ_LAD) k_c3_stage<T, ND, SCH, 2><<<grd, blk, 0, st>>>(a);
        else if (a.equation == WD_HJ_STD) k_c3_stage<T, ND, SCH, 1><<<grd, blk, 0, st>>>(a);
        else k_c3_stage<T, ND, SCH, 3><<<grd, blk, 0, st>>>(a);
    }
}

template <typename T, int ND>
static void c3_launch_nd(const C3Args<T>& a, int which, dim3 grd, dim3 blk, cudaStream_t st)
{
    if (a.scheme == WD_E6) c3_launch_s<T, ND, WD_E6>(a, which, grd, blk, st);
    else if (a.scheme == WD_E4) c3_launch_s<T, ND, WD_E4>(a, which, grd, blk, st);
    else c3_launch_s<T, ND, WD_E2>(a, which, grd, blk, st);
}

template <typename T>
cudaError_t c3_launch(const C3Args<T>& a, int which, cudaStream_t st)
{
    const int by = a.by > 0 ? a.by : 8;
    const dim3 blk(32, by, 1);
    const dim3 grd((a.D.n[0] + 31) / 32, (a.D.n[1] + by - 1) / by, a.D.n[2]);
    if constexpr (std::is_same<T, float>::value) {
        if (a.vec && a.D.ndim == 3 && a.D.pitch % 4 == 0 && (which == C3_U || which == C3_S)) {
            const dim3 g4(((a.D.n[0] + 3) / 4 + 31) / 32, grd.y, grd.z);
            if (a.scheme == WD_E6) c3_launch_v4<WD_E6>(a, which, g4, blk, st);
            else if (a.scheme == WD_E4) c3_launch_v4<WD_E4>(a, which, g4, blk, st);
            else c3_launch_v4<WD_E2>(a, which, g4, blk, st);
            return cudaGetLastError();
        }
    }
    if (which == C3_GXY) {
        const dim3 g2((a.D.n[0] + 31) / 32, (a.D.n[1] + GXY_TY - 1) / GXY_TY, a.D.n[2]);
        k_c3_gauss_xy<T><<<g2, dim3(32, 8, 1), 0, st>>>(a);
    }
    else if (which == C3_GX) k_c3_gauss<T><<<grd, blk, 0, st>>>(a, 0, a.L, a.G1);
    else if (which == C3_GY) k_c3_gauss<T><<<grd, blk, 0, st>>>(a, 1, a.G1, a.G2);
    else if (a.D.ndim == 3) c3_launch_nd<T, 3>(a, which, grd, blk, st);
    else c3_launch_nd<T, 2>(a, which, grd, blk, st);
    return cudaGetLastError();
}

template cudaError_t c3_launch<double>(const C3Args<double>&, int, cudaStream_t);
template cudaError_t c3_launch<float>(const C3Args<float>&, int, cudaStream_t);

}  // namespace wd
