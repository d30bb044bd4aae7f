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

// One grid-line node held by a thread: its slot s, node index i on the line, the slot of
// node 0 of the same line (nodes of a line sit at base + j * si in shared memory), and its
// global element index.
struct Slot {
    int s, i, base;
    long long node;
};

// Slots of this thread: s = threadIdx.x + r * blockDim.x, r < R (inactive: s = -1).
template <int R>
__device__ __forceinline__ void slots_init(Slot (&q)[R], const LineMap& mp, const Dims& D)
{
    const long long st = D.stride(mp.dir);
    const int si = mp.dir == 0 ? 1 : mp.LPB;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int s = threadIdx.x + r * blockDim.x;
        q[r].s = -1;
        q[r].i = 0;
        q[r].base = 0;
        q[r].node = 0;
        if (s < mp.size()) {
            int l, i;
            mp.decode(s, l, i);
            if (l < mp.nl) {
                q[r].s = s;
                q[r].i = i;
                q[r].base = s - i * si;
                q[r].node = D.line_base(mp.dir, mp.q0 + l) + (long long)i * st;
            }
        }
    }
}

// read-only view of one line in shared memory: node j at F[base + j * si]
template <typename T>
struct LineView {
    using value_type = T;
    const T* F;
    int base, si, N, per;
    __device__ __forceinline__ T at(int j) const   // 0 <= j < N, or wrapped when periodic
    {
        if (per) j = j < 0 ? j + N : (j >= N ? j - N : j);
        return F[base + j * si];
    }
    __device__ __forceinline__ T refl(int j) const  // even reflection at non-periodic ends
    {
        if (per) j = j < 0 ? j + N : (j >= N ? j - N : j);
        else j = j < 0 ? -j : (j >= N ? 2 * (N - 1) - j : j);
        return F[base + j * si];
    }
};

template <typename T>
__device__ __forceinline__ LineView<T> view_of(const T* F, const Slot& q, const LineMap& mp, int per)
{
    LineView<T> v;
    v.F = F;
    v.base = q.base;
    v.si = mp.dir == 0 ? 1 : mp.LPB;
    v.N = mp.N;
    v.per = per;
    return v;
}

// first derivative row at node i (explicit value, or the right-hand side of a compact row);
// Sec. 3.2.2, Eq. 16.  Non-periodic ends: one-sided (-25,48,-36,16,-3)/12 at the end node,
// centred (f_2 - f_0)/2 at the next node; E6 uses E4 at the third node.
template <typename V>
__device__ __forceinline__ typename V::value_type deriv_rhs(const V& v, int i, int sch)
{
    using T = typename V::value_type;
    const int N = v.N;
    if (!v.per) {
        if (i == 0)
            return (T(-25.0) * v.at(0) + T(48.0) * v.at(1) - T(36.0) * v.at(2) + T(16.0) * v.at(3)
                    - T(3.0) * v.at(4)) * T(1.0 / 12.0);
        if (i == N - 1)
            return -(T(-25.0) * v.at(N - 1) + T(48.0) * v.at(N - 2) - T(36.0) * v.at(N - 3)
                     + T(16.0) * v.at(N - 4) - T(3.0) * v.at(N - 5)) * T(1.0 / 12.0);
        if (i == 1 || i == N - 2) return T(0.5) * (v.at(i + 1) - v.at(i - 1));
    }
    const T d1 = v.at(i + 1) - v.at(i - 1);
    if (sch == WD_E2) return T(0.5) * d1;
    if (sch == WD_C4) return T(0.75) * d1;
    const T d2 = v.at(i + 2) - v.at(i - 2);
    if (sch == WD_C6) return T(7.0 / 9.0) * d1 + T(1.0 / 36.0) * d2;
    if (sch == WD_E4 || (!v.per && (i == 2 || i == N - 3))) return T(2.0 / 3.0) * d1 - T(1.0 / 12.0) * d2;
    const T d3 = v.at(i + 3) - v.at(i - 3);
    return T(0.75) * d1 - T(0.15) * d2 + T(1.0 / 60.0) * d3;
}

// Delta form of the filter of Eq. 21.  With sum_m a_m = 1 + 2 alpha the system
// A fh = B f is equivalent to
//     A (fh - f) = sum_{m>=1} (a_m/2 - alpha [m == 1]) (f_{i+m} + f_{i-m} - 2 f_i),
// whose right-hand side is built from second differences; the solve returns the
// correction fh - f, so rounding scales with the correction instead of with f (the filter
// matrix amplifies high-frequency rounding by up to (1 + 2 alpha) / (1 - 2 alpha)).
// cf[hw][m] holds a_m/2 - alpha [m == 1] of the order-2hw member; the order drops to
// 2 hw = 2 x (distance to a non-periodic end), and end nodes are not filtered (Sec. 3.4).
template <typename V>
__device__ __forceinline__ typename V::value_type filter_rhs(const V& v, int i,
                                                             const typename V::value_type (*cf)[6])
{
    using T = typename V::value_type;
    int hw = 5;
    if (!v.per) {
        const int e = i < v.N - 1 - i ? i : v.N - 1 - i;
        hw = e < 5 ? e : 5;
    }
    if (hw == 0) return T(0);
    const T f0 = v.at(i);
    T s = T(0);
#pragma unroll
    for (int m = 5; m >= 1; m--)
        if (m <= hw) s += cf[hw][m] * ((v.at(i + m) - f0) + (v.at(i - m) - f0));
    return s;
}

// truncated 9-point Gaussian of Kawai & Lele's LAD, even reflection at non-periodic ends
template <typename V>
__device__ __forceinline__ typename V::value_type gauss_rhs(const V& v, int i)
{
    using T = typename V::value_type;
    return T(3565.0 / 10368.0) * v.at(i) + T(3091.0 / 12960.0) * (v.refl(i + 1) + v.refl(i - 1))
         + T(1997.0 / 25920.0) * (v.refl(i + 2) + v.refl(i - 2))
         + T(149.0 / 12960.0) * (v.refl(i + 3) + v.refl(i - 3))
         + T(107.0 / 103680.0) * (v.refl(i + 4) + v.refl(i - 4));
}

// 5-point fourth difference at node i (one-sided near non-periodic ends: the nearest
// complete stencil), the d^4/dxi^4 of Eq. 7
template <typename V>
__device__ __forceinline__ typename V::value_type d4_row(const V& v, int i)
{
    using T = typename V::value_type;
    int c = i;
    if (!v.per) c = c < 2 ? 2 : (c > v.N - 3 ? v.N - 3 : c);
    return v.at(c - 2) - T(4) * v.at(c - 1) + T(6) * v.at(c) - T(4) * v.at(c + 1) + v.at(c + 2);
}

// Parallel cyclic reduction of NF right-hand sides held in X (field f at X + f*S), with
// scratch Y of the same size.  Level s combines rows i -/+ 2^s with the precomputed
// multipliers alpha_s(i), gamma_s(i) (zero where the neighbour is outside the line; the
// index is then clamped to the row itself so that no slot outside the line is read); after
// the last level x_i = d_i / b_i.  The next level's multipliers are loaded before the
// current level's barrier.  Periodic lines solve the corner-free matrix B and add the
// Sherman-Morrison correction x = y - (y_0 - a_0 y_{N-1}) / (1 + z_0 - a_0 z_{N-1}) z with
// z = B^-1 u precomputed.  Returns the buffer holding the solution.  Every thread of the
// block must call it.
template <typename T, int NF, int R>
__device__ T* pcr_solve(T* X, T* Y, const LineMap& mp, const LineTab<T>& tb, const Slot (&q)[R])
{
    const int S = mp.size(), N = mp.N;
    const int si = mp.dir == 0 ? 1 : mp.LPB;
    T an[R], gn[R], ib[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        an[r] = gn[r] = T(0);
        ib[r] = T(1);
        if (q[r].s >= 0) {
            ib[r] = tb.ib[q[r].i];
            if (tb.L > 0) {
                an[r] = tb.alpha[q[r].i];
                gn[r] = tb.gamma[q[r].i];
            }
        }
    }
    for (int lev = 0; lev < tb.L; lev++) {
        const int h = 1 << lev, hs = h * si;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int s = q[r].s;
            const T ac = an[r], gc = gn[r];
            if (s >= 0 && lev + 1 < tb.L) {
                an[r] = tb.alpha[(size_t)(lev + 1) * N + q[r].i];
                gn[r] = tb.gamma[(size_t)(lev + 1) * N + q[r].i];
            }
            if (s < 0) continue;
            const int i = q[r].i;
            const int sm = i - h >= 0 ? s - hs : s;
            const int sp = i + h < N ? s + hs : s;
#pragma unroll
            for (int f = 0; f < NF; f++) {
                const T* xf = X + (size_t)f * S;
                Y[(size_t)f * S + s] = xf[s] + ac * xf[sm] + gc * xf[sp];
            }
        }
        __syncthreads();
        T* t = X;
        X = Y;
        Y = t;
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int s = q[r].s;
        if (s < 0) continue;
#pragma unroll
        for (int f = 0; f < NF; f++) X[(size_t)f * S + s] *= ib[r];
    }
    __syncthreads();
    if (tb.periodic) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int s = q[r].s;
            if (s < 0) continue;
            const T z = tb.z[q[r].i];
            const int s0 = q[r].base, s1 = q[r].base + (N - 1) * si;
#pragma unroll
            for (int f = 0; f < NF; f++) {
                const T* xf = X + (size_t)f * S;
                const T corr = (xf[s0] - tb.a0 * xf[s1]) * tb.inv_den;
                Y[(size_t)f * S + s] = xf[s] - corr * z;
            }
        }
        __syncthreads();
        return Y;
    }
    return X;
}

// lines per block and threads per block for a line pass with NF fields of type T: at
// most 200 KB of shared memory for the two buffers and enough blocks to cover the 152 SMs
// twice when possible (strided directions prefer several lines per block for coalesced
// rows); one slot per thread up to 512 slots, otherwise R slots per 512 threads
inline void line_launch_shape(int dir, int N, int nlines, int nf, size_t esize, int& LPB, int& threads,
                              size_t& smem)
{
    const size_t limit = 200 * 1024;
    LPB = dir == 0 ? 1 : 4;
    auto bytes = [&](int lpb) { return (size_t)2 * nf * lpb * N * esize; };
    while (LPB > 1 && (bytes(LPB) > limit || LPB * N > 512)) LPB /= 2;
    while (LPB > 1 && (nlines + LPB - 1) / LPB < 2 * 152) LPB /= 2;
    const int slots = LPB * N;
    threads = slots > 512 ? 512 : ((slots + 31) / 32) * 32;
    smem = bytes(LPB);
}

// slots per thread needed by a block of `threads` threads holding `slots` slots
inline int slots_per_thread(int slots, int threads) { return (slots + threads - 1) / threads; }

}  // namespace wd
