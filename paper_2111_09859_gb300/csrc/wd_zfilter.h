// wd_zfilter.h -- the implicit filter along direction 2 of a 3-D grid fused with the commit of
// the pseudo step, streamed along z (wd_zfilter.cu).
#pragma once

#include "wd_api_internal.h"

namespace wd {

template <typename T>
struct ZfArgs {
    Dims D;
    const T* src;            // filter input: the state after the RK stages (and the other filters)
    T* scratch;              // forward-sweep values, one per node
    const T* phin;           // phi^n: the state at the start of the pseudo step
    T* phin_w;               // committed state (the same array as phin)
    const uint8_t* mask;     // Dirichlet flags
    const T* dval;           // Dirichlet values
    int poisson;             // Poisson phase: Dirichlet nodes take 0
    const T* tab;            // 3 N values: a_t, c'_t, 1 / m_t (Thomas factors of the filter rows)
    T cf[6][6];              // delta-form right-hand-side coefficients of the order-2hw members
    double* partial;         // per block: sum of squared changes, largest change
    double* result;          // sum of squared changes, largest change
    int max_partials;
};

// whether the streamed pass applies: a 3-D grid, direction 2 not periodic (the filter rows
// are then a plain tridiagonal system), enough partial slots for its blocks
bool zfilter_supported(const Dims& D, int max_partials);

// Thomas factors of the filter system a_t x_{t-1} + x_t + c_t x_{t+1} = d_t of a line of N
// nodes (rows as filter_rows gives them): out[t] = a_t, out[N + t] = c'_t, out[2N + t] = 1 / m_t
void zfilter_factors(double alpha_f, int N, double* out);

template <typename T>
cudaError_t zfilter_commit(const ZfArgs<T>& a, cudaStream_t st);

}  // namespace wd
