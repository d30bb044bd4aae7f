// wd_pcr.cuh -- device building blocks of the line passes: block-local line layout in
// shared memory, the row formulas (first derivatives of Eq. 16 with their boundary rows,
// the delta form of the filter of Eq. 21, the Gaussian smoothing of the LAD diffusivity),
// and parallel cyclic reduction (PCR) with precomputed multipliers for the constant
// tridiagonal systems.
//
// A block owns `nl` (<= LPB) grid lines of one direction, N nodes each.  Slot s of a
// block-local array is node i of local line l with
//     s = l * N + i          for direction 0 (lines are contiguous rows), or
//     s = i * LPB + l        for directions 1, 2 (neighbouring lines are neighbouring i),
// which is also the thread mapping, so global loads and shared-memory accesses are both
// contiguous across a warp.
#pragma once

#include "wd_api_internal.h"

namespace wd {

struct LineMap {
    int dir, LPB, N, nl, q0;
    __device__ __forceinline__ int slot(int l, int i) const { return dir == 0 ? l * N + i : i * LPB + l; }
    __device__ __forceinline__ void decode(int s, int& l, int& i) const
    {
        if (dir == 0) {
            l = s / N;
            i = s - l * N;
        } else {
            i = s / LPB;
            l = s - i * LPB;
        }
    }
    __device__ __forceinline__ int size() const { return LPB * N; }
};

// block-local grid-line geometry for direction dir, lines q0 .. q0+nl-1
__device__ __forceinline__ LineMap make_map(const Dims& D, int dir, int LPB, int nlines, int q0)
{
    LineMap m;
    m.dir = dir;
    m.LPB = LPB;
    m.N = D.n[dir];
    m.q0 = q0;
    m.nl = min(LPB, nlines - q0);
    return m;
}

// value of row i + o of the same line (periodic wrap, optional even reflection; for other
// non-periodic offsets the caller guarantees 0 <= i + o < N)
template <typename T>
__device__ __forceinline__ T nb(const T* F, const LineMap& mp, int l, int i, int o, int per, int reflect)
{
    int j = i + o;
    const int N = mp.N;
    if (per) j = j < 0 ? j + N : (j >= N ? j - N : j);
    else if (reflect) j = j < 0 ? -j : (j >= N ? 2 * (N - 1) - j : j);
    return F[mp.slot(l, j)];
}

// first derivative row at node i (explicit value, or the right-hand side of a compact row);
// Sec. 3.2.2, Eq. 16.  Non-periodic ends: one-sided (-25,48,-36,16,-3)/12 at the end node,
// centred (f_2 - f_0)/2 at the next node; E6 uses E4 at the third node.
template <typename T>
__device__ __forceinline__ T deriv_rhs(const T* F, const LineMap& mp, int l, int i, int per, int sch)
{
    const int N = mp.N;
#define FV(o) nb(F, mp, l, i, (o), per, 0)
    if (!per) {
        if (i == 0)
            return (T(-25.0) * FV(0) + T(48.0) * FV(1) - T(36.0) * FV(2) + T(16.0) * FV(3)
                    - T(3.0) * FV(4)) * T(1.0 / 12.0);
        if (i == N - 1)
            return -(T(-25.0) * FV(0) + T(48.0) * FV(-1) - T(36.0) * FV(-2) + T(16.0) * FV(-3)
                     - T(3.0) * FV(-4)) * T(1.0 / 12.0);
        if (i == 1 || i == N - 2) return T(0.5) * (FV(1) - FV(-1));
    }
    T d1 = FV(1) - FV(-1);
    if (sch == WD_E2) return T(0.5) * d1;
    if (sch == WD_C4) return T(0.75) * d1;
    T d2 = FV(2) - FV(-2);
    if (sch == WD_C6) return T(7.0 / 9.0) * d1 + T(1.0 / 36.0) * d2;
    if (sch == WD_E4 || (!per && (i == 2 || i == N - 3))) return T(2.0 / 3.0) * d1 - T(1.0 / 12.0) * d2;
    T d3 = FV(3) - FV(-3);
    return T(0.75) * d1 - T(0.15) * d2 + T(1.0 / 60.0) * d3;
#undef FV
}

// Delta form of the filter of Eq. 21.  With sum_m a_m = 1 + 2 alpha the system
// A fh = B f is equivalent to
//     A (fh - f) = sum_{m>=1} (a_m/2 - alpha [m == 1]) (f_{i+m} + f_{i-m} - 2 f_i),
// whose right-hand side is built from second differences; the solve returns the
// correction fh - f, so rounding scales with the correction instead of with f (the filter
// matrix amplifies high-frequency rounding by up to (1 + 2 alpha) / (1 - 2 alpha)).
// cf[hw][m] holds a_m/2 - alpha [m == 1] of the order-2hw member; the order drops to
// 2 hw = 2 x (distance to a non-periodic end), and end nodes are not filtered (Sec. 3.4).
template <typename T>
__device__ __forceinline__ T filter_rhs(const T* F, const LineMap& mp, int l, int i, int per,
                                        const T (*cf)[6])
{
    int hw = 5;
    if (!per) {
        int e = i < mp.N - 1 - i ? i : mp.N - 1 - i;
        hw = e < 5 ? e : 5;
    }
    if (hw == 0) return T(0);
    const T f0 = F[mp.slot(l, i)];
    T s = T(0);
#pragma unroll
    for (int m = 5; m >= 1; m--)
        if (m <= hw) s += cf[hw][m] * ((nb(F, mp, l, i, m, per, 0) - f0) + (nb(F, mp, l, i, -m, per, 0) - f0));
    return s;
}

// truncated 9-point Gaussian of Kawai & Lele's LAD, even reflection at non-periodic ends
template <typename T>
__device__ __forceinline__ T gauss_rhs(const T* F, const LineMap& mp, int l, int i, int per)
{
#define GV(o) (nb(F, mp, l, i, (o), per, 1) + nb(F, mp, l, i, -(o), per, 1))
    return T(3565.0 / 10368.0) * F[mp.slot(l, i)] + T(3091.0 / 12960.0) * GV(1)
         + T(1997.0 / 25920.0) * GV(2) + T(149.0 / 12960.0) * GV(3) + T(107.0 / 103680.0) * GV(4);
#undef GV
}

// 5-point fourth difference at node i (one-sided near non-periodic ends: the nearest
// complete stencil), the d^4/dxi^4 of Eq. 7
template <typename T>
__device__ __forceinline__ T d4_row(const T* F, const LineMap& mp, int l, int i, int per)
{
    int c = i;
    if (!per) c = c < 2 ? 2 : (c > mp.N - 3 ? mp.N - 3 : c);
    return nb(F, mp, l, c, -2, per, 0) - T(4) * nb(F, mp, l, c, -1, per, 0) + T(6) * F[mp.slot(l, c)]
         - T(4) * nb(F, mp, l, c, 1, per, 0) + nb(F, mp, l, c, 2, per, 0);
}

// Parallel cyclic reduction of NF right-hand sides held in X (field f at X + f*S), with
// scratch Y of the same size.  Level s combines rows i -/+ 2^s with the precomputed
// multipliers alpha_s(i), gamma_s(i); after the last level x_i = d_i / b_i.  Periodic
// lines solve the corner-free matrix B and add the Sherman-Morrison correction
// x = y - (y_0 - a_0 y_{N-1}) / (1 + z_0 - a_0 z_{N-1}) z with z = B^-1 u precomputed.
// Returns the buffer holding the solution.  All threads of the block must call it.
template <typename T, int NF>
__device__ T* pcr_solve(T* X, T* Y, const LineMap& mp, const LineTab<T>& tb)
{
    const int S = mp.size(), N = mp.N;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int lev = 0; lev < tb.L; lev++) {
        const int h = 1 << lev;
        const T* al = tb.alpha + (size_t)lev * N;
        const T* ga = tb.gamma + (size_t)lev * N;
        for (int s = tid; s < S; s += nth) {
            int l, i;
            mp.decode(s, l, i);
            if (l >= mp.nl) continue;
            const T a = al[i], g = ga[i];
            const int sm = i - h >= 0 ? mp.slot(l, i - h) : s;
            const int sp = i + h < N ? mp.slot(l, i + h) : s;
#pragma unroll
            for (int f = 0; f < NF; f++) {
                const T* xf = X + (size_t)f * S;
                T v = xf[s];
                if (i - h >= 0) v += a * xf[sm];
                if (i + h < N) v += g * xf[sp];
                Y[(size_t)f * S + s] = v;
            }
        }
        __syncthreads();
        T* t = X;
        X = Y;
        Y = t;
    }
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        const T ib = tb.ib[i];
#pragma unroll
        for (int f = 0; f < NF; f++) X[(size_t)f * S + s] *= ib;
    }
    __syncthreads();
    if (tb.periodic) {
        for (int s = tid; s < S; s += nth) {
            int l, i;
            mp.decode(s, l, i);
            if (l >= mp.nl) continue;
            const T z = tb.z[i];
            const int s0 = mp.slot(l, 0), s1 = mp.slot(l, N - 1);
#pragma unroll
            for (int f = 0; f < NF; f++) {
                const T* xf = X + (size_t)f * S;
                T corr = (xf[s0] - tb.a0 * xf[s1]) * tb.inv_den;
                Y[(size_t)f * S + s] = xf[s] - corr * z;
            }
        }
        __syncthreads();
        return Y;
    }
    return X;
}

// threads per block and lines per block for a line pass with NF fields of type T
inline void line_launch_shape(int dir, int N, int nlines, int nf, size_t esize, int& LPB, int& threads,
                              size_t& smem)
{
    const size_t limit = 200 * 1024;
    LPB = dir == 0 ? 1 : 8;
    auto bytes = [&](int lpb) { return (size_t)2 * nf * lpb * N * esize; };
    while (LPB > 1 && bytes(LPB) > limit) LPB /= 2;
    while (LPB > 1 && (nlines + LPB - 1) / LPB < 2 * 152) LPB /= 2;
    int slots = LPB * N;
    threads = slots >= 512 ? 512 : ((slots + 31) / 32) * 32;
    smem = bytes(LPB);
}

}  // namespace wd
