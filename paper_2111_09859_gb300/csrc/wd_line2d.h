// wd_line2d.h -- arguments and launchers of the line-resident 2-D pseudo-step passes
// (wd_line2d.cuh).
#pragma once

#include "wd_api_internal.h"

namespace wd {

enum { L2_Y0 = 0, L2_X = 1, L2_Y = 2, L2_FX = 3, L2_FY = 4 };

template <typename T, typename M>
struct L2Args {
    Dims D;
    T a1, a2;                            // interior rows: a1 (f+1 - f-1) + a2 (f+2 - f-2)
    int implicit;                        // compact scheme: the rows are solved along the line
    const M* xi;                         // 9 metric arrays d(xi_l)/d(x_m) at (l*3+m)
    const M* lads;                       // LAD scales s_0, s_1 (Eq. 7)
    const M* sig1;                       // sum_l |grad xi_l|
    const M* sig2;                       // Gershgorin bound of the second-order term
    const T* src;                        // stage input phi_s
    T* dst;                              // stage output phi_{s+1}
    const T* phin;                       // state at the start of the pseudo step
    T* acc;                              // RK4 accumulator
    T* dtv;                              // local pseudo time step
    T *D0, *D1;                          // d(phi_s)/dxi_0, d(phi_s)/dxi_1
    T* L1;                               // s_1 d4_1(phi_s)
    T *LAP0, *KAP0;                      // direction-0 parts of div(U) and div(n)
    T* G0;                               // C|LAD| smoothed along direction 0
    const uint8_t* mask;                 // Dirichlet nodes
    const T* dval;                       // Dirichlet values
    const double* ffr_lo;                // spacing ratios of the direction-1 faces, at k + n2 i
    const double* ffr_hi;
    int bclo1, bchi1;                    // boundary kinds of the direction-1 faces
    double eps, cfl, C_lad, eps0;
    int equation, lad, poisson, stage;
    int next;                            // Y: also D_1 and s_1 d4_1 of the stage output
    // filter passes (Eq. 21): FX filters src along direction 0 into dst; FY filters src along
    // direction 1, applies the line boundary conditions, commits the new state to phin_w and
    // reduces the change norms of every stacked grid into result (2 per grid: sum of squares,
    // max |change|), through per-block partial sums and a fixed-order final reduction
    T cf[6][6];                          // a_m / 2 - alpha_f [m == 1] of the order-2hw member
    int filter;                          // 0: FY only applies the BCs and commits
    int commit;                          // FY: 1 commit (BCs, norms); 0 filtered field into dst
    int fdir;                            // FY: line direction, 1 or 2 (3-D)
    T* phin_w;
    double* partial;
    unsigned* counter;                   // zero between launches (the last block resets it)
    double* result;
    int max_partials;                    // capacity of partial (blocks)
    int batch;
    // the stacked grids kbeg .. kbeg + kcnt - 1 of this launch (a contiguous range of lines in
    // both directions); the parts of a batch run as independent launches on separate streams
    int kbeg, kcnt;
};

// one launch of pass `which` (L2_Y0, L2_X, L2_Y, L2_FX or L2_FY) with the partition table of
// its line direction (the filter table for L2_FX / L2_FY); nf = 4 with the curvature correction
// (U and n), else 2
template <typename T, typename M>
cudaError_t l2_launch(const L2Args<T, M>& a, const PartTab<T>& tb, int which, int nf, cudaStream_t st);
// whether both directions have partition tables, n0 is a multiple of the vector row segment,
// and the widest pass fits in shared memory
template <typename T, typename M>
bool l2_supported(const Dims& D, const PartTab<T>& t0, const PartTab<T>& t1, int nf);

}  // namespace wd
