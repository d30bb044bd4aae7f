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

// Constant-coefficient tridiagonal system along one grid direction, split into P chunks
// for the partition (divide-and-conquer) solve; see wd_linesys.cu.
template <typename T>
struct LineTab {
    int N, P, implicit, periodic;
    const int* bnd;     // P + 1 chunk bounds
    const T* la;        // N: local sub-diagonal (0 at every chunk start)
    const T* lib;       // N: inverse pivots of the local forward sweep
    const T* lcp;       // N: local modified super-diagonal
    const T* v;         // N: local response to a unit value in the chunk's first row
    const T* w;         // N: local response to a unit value in the chunk's last row
    const T* acoup;     // P: coupling of the chunk's first row to the previous node
    const T* ccoup;     // P: coupling of the chunk's last row to the next node
    const T* Sinv;      // (2P)^2: inverse of the reduced system for (first, last) values
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
    int N = 0, P = 0, implicit = 0, periodic = 0, maxm = 0;
    int* bnd = nullptr;
    double* dtab = nullptr;   // 5N + 2P + 4P^2 doubles
    float* ftab = nullptr;    // same, float
    size_t bytes = 0;
    double key = 0.0;         // alpha_f the table was built for (filters)
    int valid = 0;
    template <typename T>
    LineTab<T> view() const;
};

}  // namespace wd
