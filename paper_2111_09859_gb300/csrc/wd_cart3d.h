// wd_cart3d.h -- arguments of the uniform Cartesian 3-D pseudo-step kernels (wd_cart3d.cu).
#pragma once

#include "wd_api_internal.h"

namespace wd {

enum { C3_U = 0, C3_GX = 1, C3_GY = 2, C3_S = 3, C3_GXY = 4 };

template <typename T>
struct C3Args {
    Dims D;
    int scheme;                  // WD_E2 / WD_E4 / WD_E6
    T ih[3];                     // 1 / h_l
    T slad[3];                   // LAD scales s_l = h_l^(exponent - 4) (Eq. 7, diagonal metrics)
    T sig1, sig2;                // sum_l 1/h_l, sum_l 1/h_l^2
    const T* src;                // phi of the stage
    T* dst;                      // stage output
    const T* phin;               // state at the start of the pseudo step
    T* acc;                      // RK4 accumulator
    T* dtv;                      // local pseudo time step
    T *U0, *U1, *U2;             // grad(phi)
    T *L, *G1, *G2;              // C|LAD|, smoothed along 0, along 0 and 1
    const uint8_t* mask;
    const T* dval;
    T eps, cfl, C_lad;
    int equation, lad, stage, poisson;
    int by;                      // block rows of the stencil kernels (0: 8; autotuned)
    int vec;                     // FP32 3-D: the 4-wide U and stage passes (pitch a multiple of 4)
};

template <typename T>
cudaError_t c3_launch(const C3Args<T>& a, int which, cudaStream_t st);

}  // namespace wd
