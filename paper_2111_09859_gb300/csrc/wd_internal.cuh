// wd_internal.cuh -- internal types of libwd (GB300 / sm_103a wall-distance solver).
//
// Device layout: every field is stored padded, node (i, j, k) at
// i + pitch * (j + n[1] * k) with pitch = n[0] rounded up to 32 elements, so that every
// row starts on a 128-byte boundary.  Padding elements are never read into results.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace wd {

struct Dims {
    int ndim;
    int n[3];
    int pitch;          // row pitch in elements (>= n[0], multiple of 32)
    long long total;    // pitch * n[1] * n[2]
    int per[3];         // periodic flags

    __host__ __device__ __forceinline__ long long idx(int i, int j, int k) const
    {
        return i + (long long)pitch * (j + (long long)n[1] * k);
    }
    __host__ __device__ __forceinline__ long long stride(int d) const
    {
        return d == 0 ? 1 : (d == 1 ? (long long)pitch : (long long)pitch * n[1]);
    }
    // number of grid lines along direction d
    __host__ __device__ __forceinline__ int nlines(int d) const
    {
        return (n[0] * n[1] * n[2]) / n[d];
    }
    // first node of line q along direction d; consecutive q are consecutive i for d > 0
    __host__ __device__ __forceinline__ long long line_base(int d, int q) const
    {
        if (d == 0) return idx(0, q % n[1], q / n[1]);
        if (d == 1) return idx(q % n[0], 0, q / n[0]);
        return idx(q % n[0], q / n[0], 0);
    }
};

// Constant-coefficient tridiagonal system along one grid direction (unit diagonal except
// in boundary rows), prepared for parallel cyclic reduction: level s combines rows i -/+ 2^s
// with multipliers alpha[s][i], gamma[s][i]; ib = 1 / final diagonal.  Periodic systems are
// solved through the corner-free matrix plus a Sherman-Morrison correction along z with
// the scalars a0 (corner coefficient) and inv_den.  See wd_linesys.cu.
template <typename T>
struct LineTab {
    int N, L, implicit, periodic;
    const T* alpha;     // L x N
    const T* gamma;     // L x N
    const T* ib;        // N
    const T* z;         // N (periodic only)
    T a0, inv_den;
};

// The same system prepared for the warp partition solve (wd_part2d.cu): a line of N <= 32 R
// rows (rows N .. 32R-1 are decoupled identity rows) is split into 32 blocks of R rows, one
// per lane.  The first R-1 rows of a block are eliminated locally (Thomas factors la, iw, g)
// in terms of the last rows of the previous block and of the block itself (the
// separators): x = y + P s_prev + Q s.  The 32 separators form a tridiagonal (cyclic when
// periodic) system solved by five PCR levels over warp shuffles.
//   loc[(c * (R-1) + k) * 32 + lane], c = 0 la, 1 iw, 2 g, 3 P, 4 Q
//   sep[c * 32 + lane], c = 0 a_sep, 1 c_sep, 2..6 alpha of levels 0..4, 7..11 gamma, 12 1/b
template <typename T>
struct PartTab {
    int R, N, per, implicit, ok;
    const T* loc;
    const T* sep;
};

enum { OPK_DERIV = 0, OPK_FILTER = 1, OPK_GAUSS = 2 };

struct LineOp {
    int kind;           // OPK_*
    int scheme;         // WD_E2 .. WD_C6 for OPK_DERIV
    double fa[6][6];    // filter right-hand-side coefficients a_n of the order-2hw member
};

template <typename T>
struct Fields {
    const T* in[6];
    T* out[6];
};

// host-side owner of one LineTab (both precisions)
struct HostLineTab {
    int N = 0, L = 0, implicit = 0, periodic = 0;
    int L64 = 0, L32 = 0;     // levels after which the remaining coupling is below double /
                              // float rounding (L64 <= L, L32 <= L64)
    double* dtab = nullptr;   // (2L + 3) N doubles: alpha, gamma, ib (after L64 levels),
                              // ib (after L32 levels), z
    float* ftab = nullptr;    // same, float
    double a0 = 0.0, inv_den = 0.0;
    size_t bytes = 0;
    double key = 0.0;         // alpha_f the table was built for (filters)
    int valid = 0;
    // partition tables (pok = 0 when the line is not supported: N > 2048, R < 2, or a
    // periodic N that is not 32 R)
    int pR = 0, pok = 0;
    double* pdtab = nullptr;
    float* pftab = nullptr;
    template <typename T>
    LineTab<T> view() const;
    template <typename T>
    PartTab<T> pview() const
    {
        PartTab<T> t;
        const int m = pR - 1;
        const T* base = sizeof(T) == 8 ? (const T*)(const void*)pdtab : (const T*)(const void*)pftab;
        t.R = pR;
        t.N = N;
        t.per = periodic;
        t.implicit = implicit;
        t.ok = pok;
        t.loc = base;
        t.sep = base + (size_t)5 * (m > 0 ? m : 0) * 32;
        return t;
    }
};

}  // namespace wd
