// wd_partsolve.cuh -- the warp partition solve of a constant tridiagonal line system held
// in registers (lane l owns rows lR .. lR+R-1 of the line): Thomas elimination inside each
// lane's block, five PCR levels over shuffles for the 32 block-end rows (separators), and
// the back substitution; tables built and checked on the host (wd_linesys.cu, PartTab).
#pragma once

#include "wd_internal.cuh"

namespace wd {

// Solves the line system for NF right-hand sides held in x[f] (rows lane*R + k); see
// PartTab.  Each table value is loaded once for all NF fields.  Every lane of the warp must
// call it.
template <typename T, int R, int NF>
__device__ __forceinline__ void part_solve(T (&x)[NF][R], const PartTab<T>& tb, int lane)
{
    constexpr int m = R - 1;
    const T* __restrict__ loc = tb.loc;
    const T* __restrict__ sep = tb.sep;
    {
        const T iw = __ldg(loc + (1 * m + 0) * 32 + lane);
#pragma unroll
        for (int f = 0; f < NF; f++) x[f][0] *= iw;
    }
#pragma unroll
    for (int k = 1; k < m; k++) {
        const T la = __ldg(loc + (0 * m + k) * 32 + lane), iw = __ldg(loc + (1 * m + k) * 32 + lane);
#pragma unroll
        for (int f = 0; f < NF; f++) x[f][k] = (x[f][k] - la * x[f][k - 1]) * iw;
    }
#pragma unroll
    for (int k = m - 2; k >= 0; k--) {
        const T g = __ldg(loc + (2 * m + k) * 32 + lane);
#pragma unroll
        for (int f = 0; f < NF; f++) x[f][k] -= g * x[f][k + 1];
    }
    const T as = __ldg(sep + 0 * 32 + lane), cs = __ldg(sep + 1 * 32 + lane);
    T d[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) {
        const T ynext = __shfl_sync(0xffffffffu, x[f][0], (lane + 1) & 31);
        d[f] = x[f][R - 1] - as * x[f][m - 1] - cs * ynext;
    }
#pragma unroll
    for (int lev = 0; lev < 5; lev++) {
        const int h = 1 << lev;
        const T al = __ldg(sep + (2 + lev) * 32 + lane), ga = __ldg(sep + (7 + lev) * 32 + lane);
#pragma unroll
        for (int f = 0; f < NF; f++) {
            const T dm = __shfl_sync(0xffffffffu, d[f], (lane - h) & 31);
            const T dp = __shfl_sync(0xffffffffu, d[f], (lane + h) & 31);
            d[f] += al * dm + ga * dp;
        }
    }
    const T ib = __ldg(sep + 12 * 32 + lane);
    T s[NF], sp[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) {
        s[f] = d[f] * ib;
        sp[f] = __shfl_sync(0xffffffffu, s[f], (lane + 31) & 31);
    }
#pragma unroll
    for (int k = 0; k < m; k++) {
        const T P = __ldg(loc + (3 * m + k) * 32 + lane), Q = __ldg(loc + (4 * m + k) * 32 + lane);
#pragma unroll
        for (int f = 0; f < NF; f++) x[f][k] += P * sp[f] + Q * s[f];
    }
#pragma unroll
    for (int f = 0; f < NF; f++) x[f][R - 1] = s[f];
}

template <typename T, int R>
__device__ __forceinline__ void part_solve(T (&x)[R], const PartTab<T>& tb, int lane)
{
    part_solve<T, R, 1>(reinterpret_cast<T(&)[1][R]>(x), tb, lane);
}

}  // namespace wd
