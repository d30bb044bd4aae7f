// wd_fused2d.h -- arguments of the fused 2-D pseudo-step kernels (wd_fused2d.cu).
#pragma once

#include "wd_api_internal.h"

namespace wd {

enum { F2_DERIV = 0, F2_DIV = 1, F2_STAGE = 2, F2_FILTER = 3, P2_FILTER0 = 4 };

template <typename T, typename M>
struct F2Args {
    Dims D;
    int scheme;
    LineTab<T> dtab0, dtab1, ftab1;     // derivative tables (both directions), filter (dir 1)
    const M* xi;                         // 9 metric arrays d(xi_l)/d(x_m) at (l*3+m)
    const M* lads;                       // LAD scales s_l (Eq. 7)
    const M* sig1;                       // sum_l |grad xi_l|
    const M* sig2;                       // sum_l |grad xi_l|^2
    const T* src;                        // phi at which the stage / filter works
    T* dst;                              // stage output
    const T* phin;                       // state at the start of the pseudo step
    T* phin_w;                           // committed new state (filter pass)
    T* acc;                              // RK4 accumulator
    T* dtv;                              // local pseudo time step
    T *D0, *D1;                          // d(phi)/dxi_l
    T *L0, *L1;                          // s_l d4_l(phi)
    T *LAP0, *LAP1, *KAP0, *KAP1;        // divergence parts by direction
    T* G0;                               // C|LAD| smoothed along direction 0
    const uint8_t* mask;                 // Dirichlet nodes
    const T* dval;                       // Dirichlet values
    const double* ffr_lo;                // spacing ratios of the direction-1 faces
    const double* ffr_hi;
    int bclo1, bchi1;                    // boundary kinds of the direction-1 faces
    double eps, cfl, C_lad, eps0, alpha_f;
    double fa[6][6];                     // filter coefficients a_m of each order
    int equation, curvature, lad, poisson, stage, filter;
    double* partial;                     // 2 x blocks of the commit pass
    unsigned* counter;
    double* result;                      // sum of squares, max |change|
    int max_partials;
    int batch;                           // stacked grids (n[2]); result holds 2 per grid
    int lpb[3], nb[3];                   // filled by the launcher
    int stage_threads;                   // block size of the stage kernel (0: 256; autotuned)
};

template <typename T, typename M>
cudaError_t f2_launch(F2Args<T, M> a, int which, cudaStream_t st);

// the same passes with the warp partition solve (wd_part2d.cu), one direction per launch:
// F2_DERIV, F2_DIV, P2_FILTER0 (filter src into dst) or F2_FILTER (direction 1: filter,
// line boundary conditions, change norms, commit)
template <typename T, typename M>
cudaError_t p2_launch(const F2Args<T, M>& a, const PartTab<T>& tb, int which, int dir, cudaStream_t st);
template <typename T, typename M>
bool p2_supported(const F2Args<T, M>& a, const PartTab<T>& tb, int which, int dir);
// both directions' F2_DIV passes in one launch (cudaErrorNotSupported for other line pairs)
template <typename T, typename M>
cudaError_t p2_div2(const F2Args<T, M>& a, const PartTab<T>& t0, const PartTab<T>& t1, cudaStream_t st);

}  // namespace wd
