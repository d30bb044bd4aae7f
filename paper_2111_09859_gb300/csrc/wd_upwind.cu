// wd_upwind.cu -- the baseline upwind advection term (Sec. 3.2.1, Eqs. UW1-UW5) and the
// level-set equation of the grain regression (Sec. 5.5), both built on the same upwind
// slopes.  One thread per node (a 3-D launch over i, j, k: no index division), padded SoA
// layout; every neighbour read is a +-1 step along one grid direction (wrapped on periodic
// directions), so consecutive threads read consecutive addresses and the rows above and
// below come from L1/L2.  Uniform Cartesian grids take the constant metrics delta_lm / h_l
// instead of the metric arrays.
#include "wd_api_internal.h"

namespace wd {

// Eqs. UW3-UW5: the slope is B where B >= 0 and B + F >= 0 (phi grows from the i-1 side),
// F where F < 0 and B + F < 0 (it grows from the i+1 side), and 0 at a local minimum of phi.
// Squared, this is Godunov's flux max(B+, F-)^2 of |grad phi| for a front moving towards
// increasing phi.
template <typename M>
__device__ __forceinline__ M uw_slope(M B, M F)
{
    const M s = F + B;
    return (B >= M(0) && s >= M(0)) ? B : ((F < M(0) && s < M(0)) ? F : M(0));
}

// backward and forward differences along direction l at node e (coordinates c), Eq. UW2
// with unit computational spacing; periodic directions wrap, the end node of an open line
// uses its one difference for both
template <typename T>
__device__ __forceinline__ void uw_diffs(const Dims& D, const T* __restrict__ f, long long e, const int c[3],
                                         int l, T& B, T& F)
{
    const int n = D.n[l], t = c[l];
    const long long s = D.stride(l);
    const bool hb = D.per[l] || t > 0, hf = D.per[l] || t < n - 1;
    const T v = f[e];
    T b = T(0), fw = T(0);
    if (hb) b = v - f[t > 0 ? e - s : e + (long long)(n - 1) * s];
    if (hf) fw = f[t < n - 1 ? e + s : e - (long long)(n - 1) * s] - v;
    B = hb ? b : fw;
    F = hf ? fw : b;
}

// contravariant metric d(xi_l)/d(x_m) at node e: the grid's array, or delta_lm / h_l on a
// uniform Cartesian grid (CART)
template <bool CART, typename M>
__device__ __forceinline__ M metric(const M* __restrict__ xi, const M* ih, int l, int m, long long e,
                                    long long tot)
{
    if (CART) return l == m ? ih[l] : M(0);
    return __ldg(xi + (long long)(l * 3 + m) * tot + e);
}

// one thread per node: blockIdx.x * blockDim.x + threadIdx.x runs along i, blockIdx.y is j,
// blockIdx.z is k (the stacked grid in 2-D)
__device__ __forceinline__ bool node_of(const Dims& D, int c[3])
{
    c[0] = blockIdx.x * blockDim.x + threadIdx.x;
    c[1] = blockIdx.y;
    c[2] = blockIdx.z;
    return c[0] < D.n[0];
}

static inline dim3 node_grid(const Dims& D, int threads)
{
    return dim3((unsigned)((D.n[0] + threads - 1) / threads), (unsigned)D.n[1], (unsigned)D.n[2]);
}

// U.grad(phi) of the baseline (Eq. UW1 summed over the directions): the contravariant
// components Uh_l = sum_m d(xi_l)/d(x_m) U_m of the upwind gradient U_m = sum_k
// d(xi_k)/d(x_m) s_k; direction l contributes Uh_l * B_l where Uh_l >= 0, Uh_l * F_l where
// Uh_l < 0 (the two halves of Eq. UW1)
template <typename T, typename M, bool CART, int ND>
__global__ void __launch_bounds__(128) k_uw_adv(Dims D, const T* __restrict__ phi, const M* __restrict__ xi,
                                                UwCart<M> cc, T* __restrict__ adv)
{
    int c[3];
    if (!node_of(D, c)) return;
    const long long tot = D.total;
    constexpr int nd = ND;
    const long long e = D.idx(c[0], c[1], c[2]);
    M B[3] = {M(0), M(0), M(0)}, F[3] = {M(0), M(0), M(0)}, s[3] = {M(0), M(0), M(0)};
#pragma unroll
    for (int l = 0; l < nd; l++) {
        T b, f;
        uw_diffs(D, phi, e, c, l, b, f);
        B[l] = M(b);
        F[l] = M(f);
        s[l] = uw_slope(B[l], F[l]);
    }
    M U[3] = {M(0), M(0), M(0)};
#pragma unroll
    for (int m = 0; m < nd; m++)
#pragma unroll
        for (int k = 0; k < nd; k++) U[m] += metric<CART>(xi, cc.ih, k, m, e, tot) * s[k];
    M a = M(0);
#pragma unroll
    for (int l = 0; l < nd; l++) {
        M uh = M(0);
    #pragma unroll
    for (int m = 0; m < nd; m++) uh += metric<CART>(xi, cc.ih, l, m, e, tot) * U[m];
        a += uh * (uh >= M(0) ? B[l] : F[l]);
    }
    adv[e] = T(a);
}

template <typename T, typename M>
cudaError_t launch_uw_adv(const Dims& D, const T* phi, const M* xi, const UwCart<M>& cc, T* adv,
                          cudaStream_t st)
{
    const dim3 grd = node_grid(D, 128);
    if (D.ndim == 2) {
        if (cc.cart) k_uw_adv<T, M, true, 2><<<grd, 128, 0, st>>>(D, phi, xi, cc, adv);
        else k_uw_adv<T, M, false, 2><<<grd, 128, 0, st>>>(D, phi, xi, cc, adv);
    } else {
        if (cc.cart) k_uw_adv<T, M, true, 3><<<grd, 128, 0, st>>>(D, phi, xi, cc, adv);
        else k_uw_adv<T, M, false, 3><<<grd, 128, 0, st>>>(D, phi, xi, cc, adv);
    }
    return cudaGetLastError();
}

// One classical RK4 stage of d(phi)/dt = -F |grad phi| (the level-set equation, right-hand
// side 0) with the global step dt, |grad phi| from the upwind slopes (of -phi when F < 0).
// The zero-gradient faces are folded in: the value at a node equals the stage value at the
// node with every non-periodic coordinate clamped to [1, n-2], which is what copying the
// neighbour face by face in the order of the directions produces (corners included).
// dst must not alias src or phin (face threads read their interior neighbour's phin).
template <typename T, typename M, bool CART, int ND>
__global__ void __launch_bounds__(128) k_ls_stage(Dims D, LsArgs<T, M> a, int stage)
{
    int c[3];
    if (!node_of(D, c)) return;
    const long long tot = D.total;
    constexpr int nd = ND;
    const long long e = D.idx(c[0], c[1], c[2]);
#pragma unroll
    for (int l = 0; l < nd; l++)
        if (!D.per[l]) c[l] = c[l] < 1 ? 1 : (c[l] > D.n[l] - 2 ? D.n[l] - 2 : c[l]);
    const long long q = D.idx(c[0], c[1], c[2]);
    const M sg = a.F < 0.0 ? M(-1) : M(1);
    M s[3] = {M(0), M(0), M(0)};
#pragma unroll
    for (int l = 0; l < nd; l++) {
        T b, f;
        uw_diffs(D, a.src, q, c, l, b, f);
        s[l] = uw_slope(sg * M(b), sg * M(f));
    }
    M g2 = M(0);
#pragma unroll
    for (int m = 0; m < nd; m++) {
        M u = M(0);
#pragma unroll
        for (int k = 0; k < nd; k++) u += metric<CART>(a.xi, a.cc.ih, k, m, q, tot) * s[k];
        g2 += u * u;
    }
    const T R = T(-a.F) * T(sqrt(g2));
    const T dt = T(a.dt);
    const T p0 = a.phin[q];
    T out;
    if (stage < 3) {
        if (q == e) {
            const T w = stage == 0 ? T(1.0 / 6.0) : T(1.0 / 3.0);
            a.acc[e] = stage == 0 ? R * w : a.acc[e] + R * w;
        }
        out = p0 + (stage == 2 ? dt : T(0.5) * dt) * R;
    } else {
        out = p0 + dt * (a.acc[q] + R * T(1.0 / 6.0));
    }
    a.dst[e] = out;
}

template <typename T, typename M>
cudaError_t launch_ls_stage(const Dims& D, const LsArgs<T, M>& a, int stage, cudaStream_t st)
{
    const dim3 grd = node_grid(D, 128);
    if (D.ndim == 2) {
        if (a.cc.cart) k_ls_stage<T, M, true, 2><<<grd, 128, 0, st>>>(D, a, stage);
        else k_ls_stage<T, M, false, 2><<<grd, 128, 0, st>>>(D, a, stage);
    } else {
        if (a.cc.cart) k_ls_stage<T, M, true, 3><<<grd, 128, 0, st>>>(D, a, stage);
        else k_ls_stage<T, M, false, 3><<<grd, 128, 0, st>>>(D, a, stage);
    }
    return cudaGetLastError();
}

template cudaError_t launch_uw_adv<double, double>(const Dims&, const double*, const double*,
                                                   const UwCart<double>&, double*, cudaStream_t);
template cudaError_t launch_uw_adv<float, float>(const Dims&, const float*, const float*, const UwCart<float>&,
                                                 float*, cudaStream_t);
template cudaError_t launch_ls_stage<double, double>(const Dims&, const LsArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_ls_stage<float, float>(const Dims&, const LsArgs<float, float>&, int, cudaStream_t);

}  // namespace wd
