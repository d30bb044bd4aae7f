// wd_upwind.cu -- the baseline upwind advection term (Sec. 3.2.1, Eqs. UW1-UW5) and the
// level-set equation of the grain regression (Sec. 5.5), both built on the same upwind
// slopes.  One thread per node, grid-stride, padded SoA layout; every neighbour read is a
// +-1 step along one grid direction (wrapped on periodic directions), so consecutive
// threads read consecutive addresses and the rows above and below come from L1/L2.
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

// node coordinates of padded index e
__device__ __forceinline__ void node_of(const Dims& D, long long e, int c[3])
{
    c[0] = (int)(e % D.pitch);
    const long long r = e / D.pitch;
    c[1] = (int)(r % D.n[1]);
    c[2] = (int)(r / D.n[1]);
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

// U.grad(phi) of the baseline (Eq. UW1 summed over the directions): the contravariant
// components Uh_l = sum_m d(xi_l)/d(x_m) U_m of the upwind gradient U_m = sum_k
// d(xi_k)/d(x_m) s_k; direction l contributes Uh_l * B_l where Uh_l >= 0, Uh_l * F_l where
// Uh_l < 0 (the two halves of Eq. UW1)
template <typename T, typename M>
__global__ void __launch_bounds__(256) k_uw_adv(Dims D, const T* __restrict__ phi, const M* __restrict__ xi,
                                                T* __restrict__ adv)
{
    const long long tot = D.total;
    const int nd = D.ndim;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int c[3];
        node_of(D, e, c);
        if (c[0] >= D.n[0]) continue;
        M B[3] = {M(0), M(0), M(0)}, F[3] = {M(0), M(0), M(0)}, s[3] = {M(0), M(0), M(0)};
        for (int l = 0; l < nd; l++) {
            T b, f;
            uw_diffs(D, phi, e, c, l, b, f);
            B[l] = M(b);
            F[l] = M(f);
            s[l] = uw_slope(B[l], F[l]);
        }
        M U[3] = {M(0), M(0), M(0)};
        for (int m = 0; m < nd; m++)
            for (int k = 0; k < nd; k++) U[m] += __ldg(xi + (long long)(k * 3 + m) * tot + e) * s[k];
        M a = M(0);
        for (int l = 0; l < nd; l++) {
            M uh = M(0);
            for (int m = 0; m < nd; m++) uh += __ldg(xi + (long long)(l * 3 + m) * tot + e) * U[m];
            a += uh * (uh >= M(0) ? B[l] : F[l]);
        }
        adv[e] = T(a);
    }
}

static inline int uw_grid(long long total)
{
    long long b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

template <typename T, typename M>
cudaError_t launch_uw_adv(const Dims& D, const T* phi, const M* xi, T* adv, cudaStream_t st)
{
    k_uw_adv<T, M><<<uw_grid(D.total), 256, 0, st>>>(D, phi, xi, adv);
    return cudaGetLastError();
}

// One classical RK4 stage of d(phi)/dt = -F |grad phi| (the level-set equation, right-hand
// side 0) with the global step dt, |grad phi| from the upwind slopes (of -phi when F < 0).
// The zero-gradient faces are folded in: the value at a node equals the stage value at the
// node with every non-periodic coordinate clamped to [1, n-2], which is what copying the
// neighbour face by face in the order of the directions produces (corners included).
// dst must not alias src or phin (face threads read their interior neighbour's phin).
template <typename T, typename M>
__global__ void __launch_bounds__(256) k_ls_stage(Dims D, LsArgs<T, M> a, int stage)
{
    const long long tot = D.total;
    const int nd = D.ndim;
    const M sg = a.F < 0.0 ? M(-1) : M(1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int c[3];
        node_of(D, e, c);
        if (c[0] >= D.n[0]) continue;
        for (int l = 0; l < nd; l++)
            if (!D.per[l]) c[l] = c[l] < 1 ? 1 : (c[l] > D.n[l] - 2 ? D.n[l] - 2 : c[l]);
        const long long q = D.idx(c[0], c[1], c[2]);
        M s[3] = {M(0), M(0), M(0)};
        for (int l = 0; l < nd; l++) {
            T b, f;
            uw_diffs(D, a.src, q, c, l, b, f);
            s[l] = uw_slope(sg * M(b), sg * M(f));
        }
        M g2 = M(0);
        for (int m = 0; m < nd; m++) {
            M u = M(0);
            for (int k = 0; k < nd; k++) u += __ldg(a.xi + (long long)(k * 3 + m) * tot + q) * s[k];
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
}

template <typename T, typename M>
cudaError_t launch_ls_stage(const Dims& D, const LsArgs<T, M>& a, int stage, cudaStream_t st)
{
    k_ls_stage<T, M><<<uw_grid(D.total), 256, 0, st>>>(D, a, stage);
    return cudaGetLastError();
}

template cudaError_t launch_uw_adv<double, double>(const Dims&, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_uw_adv<float, float>(const Dims&, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch_ls_stage<double, double>(const Dims&, const LsArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_ls_stage<float, float>(const Dims&, const LsArgs<float, float>&, int, cudaStream_t);

}  // namespace wd
