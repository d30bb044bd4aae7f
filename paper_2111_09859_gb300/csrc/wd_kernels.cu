// wd_kernels.cu -- sm_103a kernels of the HJ / LAD pseudo-HJ wall-distance solver.
//
//  k_line        one grid direction, whole lines staged in shared memory: explicit or
//                compact first derivatives (Sec. 3.2.2, Eq. 16), the implicit filter
//                (Sec. 3.4, Eq. 21) and the Gaussian smoothing of the LAD diffusivity;
//                tridiagonal systems are solved by the partition method (wd_linesys.cu);
//                the epilogue either stores each field or accumulates a metric-weighted
//                divergence (the Laplacian / curvature terms of Eqs. 9 and 25).
//  k_grad        chain rule U_m = sum_l d(xi_l)/d(x_m) d(phi)/d(xi_l) (Sec. 3.1) and the
//                unit normal n = U / (|U| + eps0) of Eq. 25.
//  k_lad_raw     C |sum_l (sum_m xi_{l,x_m}^2)^2 d4_l(phi) Delta x_l^e| of Eq. 7.
//  k_stage       HJ or Poisson right-hand side (Eqs. 5-7, 18-19, 25), local pseudo time
//                step and one classical RK4 stage (Sec. 3.3).
//  k_bc_face / k_bc_mask   boundary conditions (Sec. 3.5, Eqs. 22-23).
//  k_norms       RMS and max of the pseudo-step change over active nodes (Eq. 20),
//                double accumulation, deterministic order; also commits the new state.
//  metric kernels (Sec. 3.1), spacing ratios of far-field faces, masks.
#include <cstdio>

#include "wd_api_internal.h"

namespace wd {

// ------------------------------------------------------------------------------------
// line rows
// ------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T fat(const T* F, int S, int t, int N, int per)
{
    if (per) {
        if (t < 0) t += N;
        else if (t >= N) t -= N;
    }
    return F[t * S];
}

// first derivative row at t (explicit value, or the right-hand side of a compact row)
template <typename T>
__device__ __forceinline__ T deriv_row(const T* F, int S, int t, int N, int per, int scheme)
{
    if (!per) {
        if (t == 0)
            return (T(-25.0) * F[0] + T(48.0) * F[S] - T(36.0) * F[2 * S] + T(16.0) * F[3 * S]
                    - T(3.0) * F[4 * S]) * T(1.0 / 12.0);
        if (t == N - 1) {
            const T* G = F + (N - 1) * S;
            return -(T(-25.0) * G[0] + T(48.0) * G[-S] - T(36.0) * G[-2 * S]
                     + T(16.0) * G[-3 * S] - T(3.0) * G[-4 * S]) * T(1.0 / 12.0);
        }
        if (t == 1 || t == N - 2) return T(0.5) * (F[(t + 1) * S] - F[(t - 1) * S]);
    }
    T d1 = fat(F, S, t + 1, N, per) - fat(F, S, t - 1, N, per);
    if (scheme == WD_E2) return T(0.5) * d1;
    if (scheme == WD_C4) return T(0.75) * d1;
    T d2 = fat(F, S, t + 2, N, per) - fat(F, S, t - 2, N, per);
    if (scheme == WD_C6) return T(7.0 / 9.0) * d1 + T(1.0 / 36.0) * d2;
    if (scheme == WD_E4 || (!per && (t == 2 || t == N - 3)))
        return T(2.0 / 3.0) * d1 - T(1.0 / 12.0) * d2;
    T d3 = fat(F, S, t + 3, N, per) - fat(F, S, t - 3, N, per);
    return T(0.75) * d1 - T(0.15) * d2 + T(1.0 / 60.0) * d3;
}

// Filter right-hand side in delta form: with A fh = B f (Eq. 21) and sum_n a_n = 1 + 2 al,
// (B - A) f = sum_{n>=1} a_n/2 (f_{t+n} + f_{t-n} - 2 f_t) - al (f_{t+1} + f_{t-1} - 2 f_t),
// so A (fh - f) is built from second differences only; the line solve then yields the
// correction fh - f, whose rounding error scales with the correction rather than with f
// (the filter matrix amplifies high-frequency rounding by up to (1 + 2 al) / (1 - 2 al)).
template <typename T>
__device__ __forceinline__ T filter_row(const T* F, int S, int t, int N, int per, const LineOp& op)
{
    int hw = 5;
    if (!per) {
        int e = t < N - 1 - t ? t : N - 1 - t;
        if (e < hw) hw = e;
    }
    if (hw == 0) return T(0);
    const T f0 = F[t * S];
    T s = T(0);
    for (int m = hw; m >= 1; m--) {
        T s2 = (fat(F, S, t + m, N, per) - f0) + (fat(F, S, t - m, N, per) - f0);
        T cm = T(0.5 * op.fa[hw][m]) - (m == 1 ? T(op.fa[0][1]) : T(0));
        s += cm * s2;
    }
    return s;
}

// truncated 9-point Gaussian (Kawai & Lele's LAD smoothing); reflection at non-periodic ends
template <typename T>
__device__ __forceinline__ T gauss_row(const T* F, int S, int t, int N, int per)
{
    const T g0 = T(3565.0 / 10368.0), g1 = T(3091.0 / 12960.0), g2 = T(1997.0 / 25920.0),
            g3 = T(149.0 / 12960.0), g4 = T(107.0 / 103680.0);
    const T gw[5] = {g0, g1, g2, g3, g4};
    T s = gw[0] * F[t * S];
#pragma unroll
    for (int l = 1; l <= 4; l++) {
        int ip = t + l, im = t - l;
        if (per) {
            if (ip >= N) ip -= N;
            if (im < 0) im += N;
        } else {
            if (ip > N - 1) ip = 2 * (N - 1) - ip;
            if (im < 0) im = -im;
        }
        s += gw[l] * (F[ip * S] + F[im * S]);
    }
    return s;
}

// ------------------------------------------------------------------------------------
// k_line: one thread per (line, chunk).  A block holds LPB lines x P chunks (line index
// fastest, so that for strided directions neighbouring threads read neighbouring nodes).
// Each thread keeps its chunk (at most MAXM nodes) plus a 5-node halo in registers:
// right-hand side, local Thomas sweep and fix-up all run in registers; only the 2P
// chunk-end values of each line go through shared memory for the reduced system.
// ------------------------------------------------------------------------------------

constexpr int LH = 5;     // halo: E6 needs 3, the filter 5, the Gaussian 4
constexpr int MAXM = 16;  // nodes per chunk at most (host tables guarantee it)

// Row value at chunk position k (node t): the explicit derivative, the right-hand side of
// a compact row, the delta-form filter right-hand side, or the Gaussian.  F points at the
// register copy of node t (F[o] = node t + o).  cf[hw][m] holds the delta-form filter
// weights a_m/2 - alpha [m == 1] of the order-2hw member.
template <typename T>
__device__ __forceinline__ T row_value(int kind, int sch, const T (*cf)[6], const T* F, int t,
                                       int N, int per)
{
    if (kind == OPK_DERIV) {
        if (!per) {
            if (t == 0)
                return (T(-25.0) * F[0] + T(48.0) * F[1] - T(36.0) * F[2] + T(16.0) * F[3]
                        - T(3.0) * F[4]) * T(1.0 / 12.0);
            if (t == N - 1)
                return -(T(-25.0) * F[0] + T(48.0) * F[-1] - T(36.0) * F[-2] + T(16.0) * F[-3]
                         - T(3.0) * F[-4]) * T(1.0 / 12.0);
            if (t == 1 || t == N - 2) return T(0.5) * (F[1] - F[-1]);
        }
        T d1 = F[1] - F[-1];
        if (sch == WD_E2) return T(0.5) * d1;
        if (sch == WD_C4) return T(0.75) * d1;
        T d2 = F[2] - F[-2];
        if (sch == WD_C6) return T(7.0 / 9.0) * d1 + T(1.0 / 36.0) * d2;
        if (sch == WD_E4 || (!per && (t == 2 || t == N - 3)))
            return T(2.0 / 3.0) * d1 - T(1.0 / 12.0) * d2;
        T d3 = F[3] - F[-3];
        return T(0.75) * d1 - T(0.15) * d2 + T(1.0 / 60.0) * d3;
    }
    if (kind == OPK_FILTER) {
        // delta form of Eq. 21: with sum_m a_m = 1 + 2 alpha,
        //   A (fh - f) = sum_{m>=1} (a_m/2 - alpha [m==1]) (f_{t+m} + f_{t-m} - 2 f_t),
        // so the line solve returns the correction fh - f, whose rounding scales with the
        // correction instead of with f (the filter matrix amplifies high-frequency rounding
        // by up to (1 + 2 alpha) / (1 - 2 alpha))
        int hw = 5;
        if (!per) {
            int e = t < N - 1 - t ? t : N - 1 - t;
            if (e < hw) hw = e;
        }
        if (hw == 0) return T(0);
        const T f0 = F[0];
        T s = T(0);
#pragma unroll
        for (int m = 5; m >= 1; m--)
            if (m <= hw) s += cf[hw][m] * ((F[m] - f0) + (F[-m] - f0));
        return s;
    }
    // truncated 9-point Gaussian (Kawai & Lele's LAD smoothing); the even reflection at
    // non-periodic ends was applied when the halo was loaded
    return T(3565.0 / 10368.0) * F[0] + T(3091.0 / 12960.0) * (F[1] + F[-1])
         + T(1997.0 / 25920.0) * (F[2] + F[-2]) + T(149.0 / 12960.0) * (F[3] + F[-3])
         + T(107.0 / 103680.0) * (F[4] + F[-4]);
}

// position loaded into halo slot t (may lie outside [0, N)): periodic wrap, even
// reflection for the Gaussian, clamp otherwise (clamped values are never used by a row)
__device__ __forceinline__ int halo_pos(int t, int N, int per, int reflect)
{
    if (per) return t < 0 ? t + N : (t >= N ? t - N : t);
    if (reflect) return t < 0 ? -t : (t >= N ? 2 * (N - 1) - t : t);
    return t < 0 ? 0 : (t >= N ? N - 1 : t);
}

// ------------------------------------------------------------------------------------
// k_line: one thread per (line, chunk).  A block holds LPB lines x P chunks (line index
// fastest, so that for strided directions neighbouring threads read neighbouring nodes).
// Each thread keeps its chunk (at most 16 nodes) plus a 5-node halo in registers; the
// right-hand side, the local Thomas sweep and the fix-up run in registers and only the
// 2P chunk-end values of each line go through shared memory for the reduced system.
// Epilogue: store each field, or accumulate out0 (+)= sum_{m<nU} xi_{dir,m} F_m and
// out1 (+)= sum_m xi_{dir,m} F_{nU+m} (metric-weighted divergence, Eqs. 9 and 25).
// ------------------------------------------------------------------------------------

template <typename T, typename M, int NF, int EPI, int KIND>
__global__ void __launch_bounds__(256, 2)
k_line(Dims D, int dir, int nlines, int LPB, LineTab<T> tab, LineOp op, Fields<T> f,
       const M* __restrict__ xi, int nU, int accumulate)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Y = reinterpret_cast<T*>(smraw);              // LPB x 2P chunk-end values
    __shared__ T cf[6][6];
    for (int i = threadIdx.x; i < 36; i += blockDim.x) {
        int hw = i / 6, m = i % 6;
        double v = 0.0;
        if (KIND == OPK_FILTER && hw >= 1 && m >= 1 && m <= hw)
            v = 0.5 * op.fa[hw][m] - (m == 1 ? op.fa[0][1] : 0.0);
        cf[hw][m] = T(v);
    }
    __syncthreads();
    const int N = tab.N, P = tab.P, P2 = 2 * P;
    const int l = threadIdx.x % LPB, c = threadIdx.x / LPB;
    const int q = blockIdx.x * LPB + l;
    const bool act = q < nlines;
    const long long st = D.stride(dir);
    const int per = D.per[dir];
    constexpr int kind = KIND;
    const int sch = op.scheme;
    const int reflect = kind == OPK_GAUSS;
    const long long base = act ? D.line_base(dir, q) : 0;
    const int s = tab.bnd[c], Mc = tab.bnd[c + 1] - s;

    T acc[EPI ? MAXM : 1];
    T x[MAXM];

#pragma unroll 1
    for (int fi = 0; fi < NF; fi++) {
        const T* __restrict__ src = f.in[fi];
        if (act) {
            T fr[MAXM + 2 * LH];
#pragma unroll
            for (int k = 0; k < MAXM + 2 * LH; k++)
                if (k < Mc + 2 * LH) fr[k] = src[base + (long long)halo_pos(s + k - LH, N, per, reflect) * st];
#pragma unroll
            for (int k = 0; k < MAXM; k++)
                if (k < Mc) x[k] = row_value<T>(kind, sch, cf, fr + LH + k, s + k, N, per);
        }
        if (tab.implicit) {
            if (act) {
                T prev = T(0);
#pragma unroll
                for (int k = 0; k < MAXM; k++)
                    if (k < Mc) {
                        prev = (x[k] - tab.la[s + k] * prev) * tab.lib[s + k];
                        x[k] = prev;
                    }
#pragma unroll
                for (int k = MAXM - 2; k >= 0; k--)
                    if (k < Mc - 1) x[k] = x[k] - tab.lcp[s + k] * x[k + 1];
                T last = x[0];
#pragma unroll
                for (int k = 0; k < MAXM; k++)
                    if (k == Mc - 1) last = x[k];
                Y[l * P2 + 2 * c] = x[0];
                Y[l * P2 + 2 * c + 1] = last;
            }
            __syncthreads();
            if (act) {
                const T ac = tab.acoup[c], cc = tab.ccoup[c];
                const T* Yl = Y + l * P2;
                T qm = T(0), pp = T(0);
                if (ac != T(0)) {
                    const T* row = tab.Sinv + (size_t)(2 * ((c - 1 + P) % P) + 1) * P2;
                    for (int j = 0; j < P2; j++) qm += row[j] * Yl[j];
                }
                if (cc != T(0)) {
                    const T* row = tab.Sinv + (size_t)(2 * ((c + 1) % P)) * P2;
                    for (int j = 0; j < P2; j++) pp += row[j] * Yl[j];
                }
                const T aq = ac * qm, cp = cc * pp;
#pragma unroll
                for (int k = 0; k < MAXM; k++)
                    if (k < Mc) x[k] -= aq * tab.v[s + k] + cp * tab.w[s + k];
            }
            __syncthreads();   // Y is reused by the next field
        }
        if (!act) continue;
        if (kind == OPK_FILTER) {
#pragma unroll
            for (int k = 0; k < MAXM; k++)
                if (k < Mc) x[k] += src[base + (long long)(s + k) * st];
        }
        if (EPI == 0) {
            T* __restrict__ dst = f.out[fi];
#pragma unroll
            for (int k = 0; k < MAXM; k++)
                if (k < Mc) dst[base + (long long)(s + k) * st] = x[k];
        } else {
            const int grp = fi < nU ? 0 : 1, m = fi - grp * nU;
            const M* __restrict__ xm = xi + (long long)(dir * 3 + m) * D.total;
#pragma unroll
            for (int k = 0; k < MAXM; k++)
                if (k < Mc) {
                    T v = T(xm[base + (long long)(s + k) * st] * M(x[k]));
                    acc[EPI ? k : 0] = (m == 0 ? T(0) : acc[EPI ? k : 0]) + v;
                }
            if (m == nU - 1) {
                T* o = f.out[grp];
#pragma unroll
                for (int k = 0; k < MAXM; k++)
                    if (k < Mc) {
                        long long p = base + (long long)(s + k) * st;
                        o[p] = accumulate ? o[p] + acc[EPI ? k : 0] : acc[EPI ? k : 0];
                    }
            }
        }
    }
}

template <typename T, typename M, int NF, int EPI, int KIND>
static cudaError_t line_dispatch(const Dims& D, int dir, const HostLineTab& tab, const LineOp& op,
                                 const Fields<T>& f, const M* xi, int nU, int accumulate,
                                 cudaStream_t st)
{
    if (tab.maxm > MAXM) return cudaErrorInvalidConfiguration;
    const int P = tab.P;
    const int nlines = D.nlines(dir);
    // strided directions: up to 32 lines per block (coalesced rows); contiguous lines
    // gain nothing from wide blocks.  Shrink until the grid covers the 152 SMs twice.
    int LPB = dir == 0 ? 4 : 32;
    while (LPB > 1 && LPB * P > 256) LPB /= 2;
    const int min_lpb = dir == 0 ? 1 : (P <= 32 ? 8 : 2);
    while (LPB > min_lpb && (nlines + LPB - 1) / LPB < 2 * 152) LPB /= 2;
    if (LPB * P > 256 || LPB < 1) return cudaErrorInvalidConfiguration;
    int grid = (nlines + LPB - 1) / LPB;
    size_t sm = (size_t)LPB * 2 * P * sizeof(T);
    k_line<T, M, NF, EPI, KIND><<<grid, LPB * P, sm, st>>>(D, dir, nlines, LPB, tab.view<T>(), op, f,
                                                           xi, nU, accumulate);
    return cudaGetLastError();
}

template <typename T, typename M>
cudaError_t launch_line(const Dims& D, int dir, const HostLineTab& tab, const LineOp& op, int nf,
                        int epi, const Fields<T>& f, const M* xi, int nU, int accumulate,
                        cudaStream_t st)
{
    if (tab.N != D.n[dir]) return cudaErrorInvalidValue;
    if (op.kind == OPK_FILTER && nf == 1 && epi == 0)
        return line_dispatch<T, M, 1, 0, OPK_FILTER>(D, dir, tab, op, f, xi, nU, accumulate, st);
    if (op.kind == OPK_GAUSS && nf == 1 && epi == 0)
        return line_dispatch<T, M, 1, 0, OPK_GAUSS>(D, dir, tab, op, f, xi, nU, accumulate, st);
    if (op.kind != OPK_DERIV) return cudaErrorInvalidValue;
    if (epi == 0) {
        switch (nf) {
        case 1: return line_dispatch<T, M, 1, 0, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (nf) {
    case 2: return line_dispatch<T, M, 2, 1, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
    case 3: return line_dispatch<T, M, 3, 1, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
    case 4: return line_dispatch<T, M, 4, 1, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
    case 6: return line_dispatch<T, M, 6, 1, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------------------------
// pointwise kernels (grid-stride over the padded layout, padding skipped)
// ------------------------------------------------------------------------------------

static inline int pw_grid(long long total)
{
    long long b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T, typename M>
__global__ void k_grad(Dims D, const T* __restrict__ D0, const T* __restrict__ D1,
                       const T* __restrict__ D2, const M* __restrict__ xi, T* U0, T* U1, T* U2,
                       T* n0, T* n1, T* n2, double eps0)
{
    const long long tot = D.total;
    const int nd = D.ndim;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        M d[3] = {M(D0[e]), M(D1[e]), nd == 3 ? M(D2[e]) : M(0)};
        M u[3] = {M(0), M(0), M(0)};
        for (int m = 0; m < nd; m++) {
            M s = M(0);
            for (int l = 0; l < nd; l++) s += xi[(long long)(l * 3 + m) * tot + e] * d[l];
            u[m] = s;
        }
        U0[e] = T(u[0]);
        U1[e] = T(u[1]);
        if (nd == 3) U2[e] = T(u[2]);
        if (n0) {
            M g = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) + M(eps0);
            n0[e] = T(u[0] / g);
            n1[e] = T(u[1] / g);
            if (nd == 3) n2[e] = T(u[2] / g);
        }
    }
}

template <typename T, typename M>
cudaError_t launch_grad(const Dims& D, const T* const* Dl, const M* xi, T* const* U,
                        T* const* nv, double eps0, cudaStream_t st)
{
    k_grad<T, M><<<pw_grid(D.total), 256, 0, st>>>(D, Dl[0], Dl[1], Dl[2], xi, U[0], U[1], U[2],
                                                   nv ? nv[0] : nullptr, nv ? nv[1] : nullptr,
                                                   nv ? nv[2] : nullptr, eps0);
    return cudaGetLastError();
}

template <typename T, typename M>
__global__ void k_lad_raw(Dims D, const T* __restrict__ phi, const M* __restrict__ lads, double C,
                          T* out)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % D.pitch);
        if (i >= D.n[0]) continue;
        long long r = e / D.pitch;
        int crd[3] = {i, (int)(r % D.n[1]), (int)(r / D.n[1])};
        M s = M(0);
        for (int l = 0; l < D.ndim; l++) {
            int n = D.n[l], t = crd[l];
            int c = t;
            if (!D.per[l]) c = c < 2 ? 2 : (c > n - 3 ? n - 3 : c);
            long long sl = D.stride(l);
            long long base = e + (long long)(c - t) * sl;
            int o[5];
            for (int k = 0; k < 5; k++) {
                int q = c + k - 2;
                if (D.per[l]) q = q < 0 ? q + n : (q >= n ? q - n : q);
                o[k] = q - c;
            }
            M d4 = M(phi[base + o[0] * sl]) - M(4) * M(phi[base + o[1] * sl]) + M(6) * M(phi[base])
                 - M(4) * M(phi[base + o[3] * sl]) + M(phi[base + o[4] * sl]);
            s += lads[(long long)l * tot + e] * d4;
        }
        out[e] = T(M(C) * (s < M(0) ? -s : s));
    }
}

template <typename T, typename M>
cudaError_t launch_lad_raw(const Dims& D, const T* phi, const M* lads, double C, T* out,
                           cudaStream_t st)
{
    k_lad_raw<T, M><<<pw_grid(D.total), 256, 0, st>>>(D, phi, lads, C, out);
    return cudaGetLastError();
}

// HJ / Poisson right-hand side, local pseudo time step and one classical RK4 stage.
template <typename T, typename M>
__global__ void k_stage(Dims D, StageArgs<T, M> a, int stage)
{
    const long long tot = D.total;
    const int nd = D.ndim;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        T R, dtv;
        T gam = T(0), v = T(0), gm = T(0);
        if (a.poisson) {
            R = T(1) + a.lap[e];                                       // Eq. 19
        } else {
            T g2 = a.U[0][e] * a.U[0][e] + a.U[1][e] * a.U[1][e];
            if (nd == 3) g2 += a.U[2][e] * a.U[2][e];
            gm = sqrt(g2);
            T ph = a.src[e];
            T php = ph > T(0) ? ph : T(0);
            if (a.equation == WD_HJ_STD) gam = T(a.eps) * php;         // Eq. 6
            else if (a.equation == WD_HJ_LAD) {                        // Eq. 7
                T g1 = T(a.eps) * php, g2l = a.lad[e];
                gam = g1 < g2l ? g1 : g2l;
            }
            if (a.curvature) {                                         // Eq. 25
                v = T(0.001) * (T(1) - gm) * (T(1) - gm);
                T corr = gm * a.kap[e];
                corr = corr > T(0) ? corr : T(0);
                R = T(1) + (gam + v) * (a.lap[e] - corr) - g2;
            } else {
                R = T(1) + gam * a.lap[e] - g2;                        // Eqs. 5, 18
            }
        }
        if (stage <= 0) {
            if (a.poisson) dtv = T(a.cfl) / T(a.sig2[e]);
            else {
                T am = gm > T(1) ? gm : T(1);
                dtv = T(a.cfl) / (T(a.sig1[e]) * am + (gam + v) * T(a.sig2[e]));
            }
            a.dt[e] = dtv;
        } else {
            dtv = a.dt[e];
        }
        if (stage < 0) {
            a.dst[e] = R;
            continue;
        }
        T n = a.phin[e];
        T out;
        if (stage == 0) {
            a.acc[e] = R * T(1.0 / 6.0);
            out = n + T(0.5) * dtv * R;
        } else if (stage == 1) {
            a.acc[e] += R * T(1.0 / 3.0);
            out = n + T(0.5) * dtv * R;
        } else if (stage == 2) {
            a.acc[e] += R * T(1.0 / 3.0);
            out = n + dtv * R;
        } else {
            out = n + dtv * (a.acc[e] + R * T(1.0 / 6.0));
        }
        a.dst[e] = out;
    }
}

template <typename T, typename M>
cudaError_t launch_stage(const Dims& D, const StageArgs<T, M>& a, int stage, cudaStream_t st)
{
    k_stage<T, M><<<pw_grid(D.total), 256, 0, st>>>(D, a, stage);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_spalding(Dims D, const T* __restrict__ U0, const T* __restrict__ U1,
                           const T* __restrict__ U2, const T* __restrict__ phip, T* phi)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        T g2 = U0[e] * U0[e] + U1[e] * U1[e];
        if (D.ndim == 3) g2 += U2[e] * U2[e];
        // Eq. 4 with the minus root, -g + sqrt(g^2 + 2 phi'), evaluated in the equivalent
        // form 2 phi' / (g + sqrt(g^2 + 2 phi')) that does not cancel when 2 phi' << g^2
        T g = sqrt(g2);
        T arg = g2 + T(2) * phip[e];
        T r = sqrt(arg > T(0) ? arg : T(0));
        phi[e] = (arg > T(0) && g + r > T(0)) ? T(2) * phip[e] / (g + r) : -g;
    }
}

template <typename T, typename M>
cudaError_t launch_spalding(const Dims& D, const T* const* U, const T* phip, T* phi,
                            cudaStream_t st)
{
    k_spalding<T><<<pw_grid(D.total), 256, 0, st>>>(D, U[0], U[1], U[2], phip, phi);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// boundary conditions
// ------------------------------------------------------------------------------------

template <typename T>
__global__ void k_bc_face(Dims D, int d, int klo, int khi, const double* __restrict__ rlo,
                          const double* __restrict__ rhi, T* phi)
{
    const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
    const int fsize = D.n[o1] * D.n[o2];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * fsize; e += gridDim.x * blockDim.x) {
        int side = e / fsize, fidx = e - side * fsize;
        int kind = side ? khi : klo;
        if (kind != WD_BC_FARFIELD && kind != WD_BC_NEUMANN) continue;
        int c[3];
        c[o1] = fidx % D.n[o1];
        c[o2] = fidx / D.n[o1];
        c[d] = side ? D.n[d] - 1 : 0;
        long long p = D.idx(c[0], c[1], c[2]);
        long long s = side ? -D.stride(d) : D.stride(d);
        if (kind == WD_BC_NEUMANN) phi[p] = phi[p + s];
        else {
            T r = T((side ? rhi : rlo)[fidx]);
            T a1 = phi[p + s], a2 = phi[p + 2 * s];
            phi[p] = a1 + r * (a1 - a2);
        }
    }
}

template <typename T>
cudaError_t launch_bc_face(const Dims& D, int dir, int kind_lo, int kind_hi, const double* rlo,
                           const double* rhi, T* phi, cudaStream_t st)
{
    int o1 = (dir + 1) % 3, o2 = (dir + 2) % 3;
    int n = 2 * D.n[o1] * D.n[o2];
    k_bc_face<T><<<(n + 255) / 256, 256, 0, st>>>(D, dir, kind_lo, kind_hi, rlo, rhi, phi);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_bc_mask(Dims D, const uint8_t* __restrict__ mask, const T* __restrict__ dval, T* phi)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        if (mask[e]) phi[e] = dval ? dval[e] : T(0);
    }
}

template <typename T>
cudaError_t launch_bc_mask(const Dims& D, const uint8_t* mask, const T* dval, T* phi, cudaStream_t st)
{
    k_bc_mask<T><<<pw_grid(D.total), 256, 0, st>>>(D, mask, dval, phi);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// change norms (double, deterministic: fixed partition, fixed final order)
// ------------------------------------------------------------------------------------

template <typename T>
__global__ void k_norms(Dims D, const T* __restrict__ newp, T* oldp, const uint8_t* __restrict__ mask,
                        double* partial, unsigned* counter, double* result)
{
    __shared__ double s_ss[32], s_mx[32];
    __shared__ int s_last;
    const long long tot = D.total;
    double ss = 0.0, mx = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        T a = newp[e], b = oldp[e];
        oldp[e] = a;
        if (mask[e]) continue;
        double d = double(a) - double(b);
        ss += d * d;
        mx = fmax(mx, fabs(d));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        s_ss[wid] = ss;
        s_mx[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0;
        for (int w = 0; w < nw; w++) {
            a += s_ss[w];
            m = fmax(m, s_mx[w]);
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = m;
        __threadfence();
        unsigned v = atomicAdd(counter, 1u);
        s_last = (v == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ss = 0.0;
    mx = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        ss += __ldcg(partial + 2 * b);
        mx = fmax(mx, __ldcg(partial + 2 * b + 1));
    }
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    __syncthreads();
    if (lane == 0) {
        s_ss[wid] = ss;
        s_mx[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0;
        for (int w = 0; w < nw; w++) {
            a += s_ss[w];
            m = fmax(m, s_mx[w]);
        }
        result[0] = a;
        result[1] = m;
        *counter = 0u;
    }
}

template <typename T>
cudaError_t launch_norms(const Dims& D, const T* newp, T* oldp, const uint8_t* mask, double* partial,
                         unsigned* counter, double* result, int nblocks, cudaStream_t st)
{
    k_norms<T><<<nblocks, 256, 0, st>>>(D, newp, oldp, mask, partial, counter, result);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_fill(T* p, long long n, T v)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        p[e] = v;
}

template <typename T>
cudaError_t launch_fill(T* p, long long n, T v, cudaStream_t st)
{
    k_fill<T><<<pw_grid(n), 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// metrics (Sec. 3.1), computed once per grid in double
// ------------------------------------------------------------------------------------

__global__ void k_unwrap(Dims D, int dir, const double* __restrict__ x, double shift, double* out)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % D.pitch);
        if (i >= D.n[0]) continue;
        long long r = e / D.pitch;
        int crd[3] = {i, (int)(r % D.n[1]), (int)(r / D.n[1])};
        out[e] = x[e] - shift * (double)crd[dir] / (double)D.n[dir];
    }
}

cudaError_t launch_unwrap(const Dims& D, int dir, const double* x, double shift, double* out,
                          cudaStream_t st)
{
    k_unwrap<<<pw_grid(D.total), 256, 0, st>>>(D, dir, x, shift, out);
    return cudaGetLastError();
}

__global__ void k_add_const(Dims D, double* p, double c)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < D.total;
         e += (long long)gridDim.x * blockDim.x)
        if ((int)(e % D.pitch) < D.n[0]) p[e] += c;
}

cudaError_t launch_add_const(const Dims& D, double* p, double c, cudaStream_t st)
{
    k_add_const<<<pw_grid(D.total), 256, 0, st>>>(D, p, c);
    return cudaGetLastError();
}

// A[(m*3+l)*total + e] = dx_m/dxi_l (the periodic shift already added back).
template <typename M>
__global__ void k_metric_finish(Dims D, const double* __restrict__ A, double* xi_d, double* J,
                                double* dx, M* xi_m, M* sig1, M* sig2)
{
    const long long tot = D.total;
    const int nd = D.ndim;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        double a[3][3];
        for (int m = 0; m < 3; m++)
            for (int l = 0; l < 3; l++)
                a[m][l] = (m < nd && l < nd) ? A[(long long)(m * 3 + l) * tot + e] : (m == l ? 1.0 : 0.0);
        // cofactor expansion: inv[l][m] = cof[m][l] / det
        double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
        double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
        double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
        double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
        double inv[3][3];
        inv[0][0] = c00 / det;
        inv[1][0] = c01 / det;
        inv[2][0] = c02 / det;
        inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
        inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
        inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
        inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
        inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
        inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
        J[e] = det;
        double s1 = 0.0, s2 = 0.0;
        for (int l = 0; l < 3; l++) {
            double q = 0.0, col = 0.0;
            for (int m = 0; m < 3; m++) {
                double x = (l < nd && m < nd) ? inv[l][m] : 0.0;
                xi_d[(long long)(l * 3 + m) * tot + e] = x;
                if (xi_m) xi_m[(long long)(l * 3 + m) * tot + e] = M(x);
                q += x * x;
                if (m < nd && l < nd) col += a[m][l] * a[m][l];
            }
            dx[(long long)l * tot + e] = l < nd ? sqrt(col) : 0.0;
            if (l < nd) {
                s1 += sqrt(q);
                s2 += q;
            }
        }
        sig1[e] = M(s1);
        sig2[e] = M(s2);
    }
}

template <typename M>
cudaError_t launch_metric_finish(const Dims& D, const double* A, double* xi_d, double* J, double* dx,
                                 M* xi_m, M* sig1, M* sig2, cudaStream_t st)
{
    k_metric_finish<M><<<pw_grid(D.total), 256, 0, st>>>(D, A, xi_d, J, dx, xi_m, sig1, sig2);
    return cudaGetLastError();
}

// LAD scale s_l = (sum_m xi_{l,x_m}^2)^2 Delta x_l^ex of Eq. 7
template <typename M>
__global__ void k_lad_scale(Dims D, const double* __restrict__ xi_d, const double* __restrict__ dx,
                            double ex, M* lads)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        for (int l = 0; l < D.ndim; l++) {
            double q = 0.0;
            for (int m = 0; m < D.ndim; m++) {
                double x = xi_d[(long long)(l * 3 + m) * tot + e];
                q += x * x;
            }
            lads[(long long)l * tot + e] = M(q * q * pow(dx[(long long)l * tot + e], ex));
        }
    }
}

template <typename M>
cudaError_t launch_lad_scale(const Dims& D, const double* xi_d, const double* dx, double ex, M* lads,
                             cudaStream_t st)
{
    k_lad_scale<M><<<pw_grid(D.total), 256, 0, st>>>(D, xi_d, dx, ex, lads);
    return cudaGetLastError();
}

// spacing ratio |x_b - x_b1| / |x_b1 - x_b2| on the face nodes of both faces of every
// direction; ratio[(2d+side)*fmax + fidx]
__global__ void k_ff_ratio(Dims D, const double* __restrict__ xyz, double* ratio, long long fmax)
{
    for (int d = 0; d < D.ndim; d++) {
        const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
        const int fsize = D.n[o1] * D.n[o2];
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * fsize; e += gridDim.x * blockDim.x) {
            int side = e / fsize, fidx = e - side * fsize;
            int c[3];
            c[o1] = fidx % D.n[o1];
            c[o2] = fidx / D.n[o1];
            c[d] = side ? D.n[d] - 1 : 0;
            long long p = D.idx(c[0], c[1], c[2]);
            long long s = side ? -D.stride(d) : D.stride(d);
            double d1 = 0.0, d2 = 0.0;
            for (int m = 0; m < 3; m++) {
                const double* x = xyz + (long long)m * D.total;
                double a = x[p] - x[p + s], b = x[p + s] - x[p + 2 * s];
                d1 += a * a;
                d2 += b * b;
            }
            ratio[(long long)(2 * d + side) * fmax + fidx] = sqrt(d1) / sqrt(d2);
        }
    }
}

cudaError_t launch_ff_ratio(const Dims& D, const double* xyz, double* ratio, long long fmax,
                            cudaStream_t st)
{
    k_ff_ratio<<<(int)((2 * fmax + 255) / 256), 256, 0, st>>>(D, xyz, ratio, fmax);
    return cudaGetLastError();
}

// mask[e] = wall[e] | user (dense); dval[e] = wall ? 0 : user value (dense)
template <typename T>
__global__ void k_mask_merge(Dims D, const uint8_t* __restrict__ um, const T* __restrict__ uv,
                             uint8_t* mask, T* dval, const uint8_t* __restrict__ wall)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % D.pitch);
        if (i >= D.n[0]) continue;
        long long r = e / D.pitch;
        long long q = i + (long long)D.n[0] * r;     // dense index
        uint8_t w = wall[e];
        uint8_t u = um ? (um[q] != 0) : 0;
        mask[e] = w | u;
        dval[e] = (!w && u && uv) ? uv[q] : T(0);
    }
}

template <typename T>
cudaError_t launch_mask_merge(const Dims& D, const uint8_t* src_dense, const T* val_dense,
                              uint8_t* mask, T* dval, const uint8_t* wallmask, cudaStream_t st)
{
    k_mask_merge<T><<<pw_grid(D.total), 256, 0, st>>>(D, src_dense, val_dense, mask, dval, wallmask);
    return cudaGetLastError();
}

__global__ void k_count(Dims D, const uint8_t* __restrict__ mask, unsigned long long* out)
{
    unsigned long long c = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < D.total;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        if (!mask[e]) c++;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

cudaError_t launch_count(const Dims& D, const uint8_t* mask, unsigned long long* out, cudaStream_t st)
{
    k_count<<<pw_grid(D.total), 256, 0, st>>>(D, mask, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// explicit instantiations: (state, metric) = (double, double), (float, double), (float, float)
// ------------------------------------------------------------------------------------

#define WD_INST_TM(T, M)                                                                          \
    template cudaError_t launch_line<T, M>(const Dims&, int, const HostLineTab&, const LineOp&,   \
                                           int, int, const Fields<T>&, const M*, int, int,        \
                                           cudaStream_t);                                         \
    template cudaError_t launch_grad<T, M>(const Dims&, const T* const*, const M*, T* const*,     \
                                           T* const*, double, cudaStream_t);                      \
    template cudaError_t launch_lad_raw<T, M>(const Dims&, const T*, const M*, double, T*,        \
                                              cudaStream_t);                                      \
    template cudaError_t launch_stage<T, M>(const Dims&, const StageArgs<T, M>&, int,             \
                                            cudaStream_t);                                        \
    template cudaError_t launch_spalding<T, M>(const Dims&, const T* const*, const T*, T*,        \
                                               cudaStream_t);

WD_INST_TM(double, double)
WD_INST_TM(float, double)
WD_INST_TM(float, float)

#define WD_INST_T(T)                                                                              \
    template cudaError_t launch_bc_face<T>(const Dims&, int, int, int, const double*,             \
                                           const double*, T*, cudaStream_t);                      \
    template cudaError_t launch_bc_mask<T>(const Dims&, const uint8_t*, const T*, T*,             \
                                           cudaStream_t);                                         \
    template cudaError_t launch_norms<T>(const Dims&, const T*, T*, const uint8_t*, double*,      \
                                         unsigned*, double*, int, cudaStream_t);                  \
    template cudaError_t launch_fill<T>(T*, long long, T, cudaStream_t);                          \
    template cudaError_t launch_mask_merge<T>(const Dims&, const uint8_t*, const T*, uint8_t*,    \
                                              T*, const uint8_t*, cudaStream_t);

WD_INST_T(double)
WD_INST_T(float)

template cudaError_t launch_metric_finish<double>(const Dims&, const double*, double*, double*,
                                                  double*, double*, double*, double*, cudaStream_t);
template cudaError_t launch_metric_finish<float>(const Dims&, const double*, double*, double*,
                                                 double*, float*, float*, float*, cudaStream_t);
template cudaError_t launch_lad_scale<double>(const Dims&, const double*, const double*, double,
                                              double*, cudaStream_t);
template cudaError_t launch_lad_scale<float>(const Dims&, const double*, const double*, double,
                                             float*, cudaStream_t);
template cudaError_t launch_fill<uint8_t>(uint8_t*, long long, uint8_t, cudaStream_t);

}  // namespace wd
