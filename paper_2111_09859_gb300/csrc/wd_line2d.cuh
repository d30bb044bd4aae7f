// wd_line2d.cuh -- line-resident 2-D pseudo step: two line passes per RK4 stage (Sec. 3.3)
// for 2-D grids whose direction-0 faces are periodic or walls (O-grids, channels, plates,
// boxes, stacked grids), compact C4 / C6 or explicit E2 / E4 first derivatives (Eq. 16).
// Instantiated per precision in wd_line2d_f32.cu and wd_line2d_f64.cu.
//
// The work of one stage is split by the direction of the lines it needs:
//   X  (direction-0 lines, one warp per line, no block barrier)
//      D_0(phi) (line solve), C |s_0 d4_0(phi) + s_1 d4_1(phi)| smoothed along direction 0
//      (the first half of the separable Gaussian of the LAD diffusivity, Eq. 7), the
//      physical gradient U = grad(phi) and unit normal n = U / (|U| + eps_0) from D_0 and
//      D_1 (Sec. 3.1), and their direction-0 metric-weighted divergences (the direction-0
//      part of the Laplacian of Eq. 9 and of the curvature of Eq. 25, four line solves);
//   Y  (direction-1 lines, one warp per line, YW neighbouring lines per block so that the
//      global accesses are coalesced row segments)
//      the direction-1 divergences (four line solves), the Gaussian along direction 1, the
//      right-hand side (Eqs. 5-7, 18, 19, 25), the local pseudo time step, the RK4 stage,
//      the boundary conditions of the line (far-field / Neumann ends, Dirichlet nodes;
//      Eqs. 22-23), and, for the next stage, D_1 and s_1 d4_1 of the new stage value.
// A pseudo step is Y0 (D_1, s_1 d4_1 of phi^n), four X + Y pairs, the two filter passes of
// Eq. 21 with the change norms (wd_part2d.cuh): 11 launches, against 19 for the per-operator
// passes.  Every formula and the order of operations are those of the per-operator passes;
// only the kernel boundaries and the memory layout differ.
//
// Line layout in shared memory: the 32 R rows of a line (R = rows per lane of the partition
// solve) sit in 32 blocks of R rows, block b at (b + G) * S with the odd stride S = R or R + 1
// (lanes R rows apart hit distinct banks), and G ghost blocks on each side hold the wrapped
// rows of periodic lines.  A lane's R rows and every neighbour a stencil of half width <= 5
// reaches are then at compile-time offsets from the lane's block, so the interior row
// formulas are straight loads and FMAs; the rows within 5 of a non-periodic end take the
// general formulas (one-sided closures, even reflection, reduced filter order), evaluated
// by one lane per row into a small per-warp scratch and picked up by the owning lane.
#pragma once

#include <type_traits>

#include "wd_api_internal.h"
#include "wd_fused2d.h"
#include "wd_line2d.h"
#include "wd_partsolve.cuh"
#include "wd_pcr.cuh"

namespace wd {

// ---- layout -------------------------------------------------------------------------------
template <int R>
struct LL {
    static constexpr int H = 5;                          // widest half width (filter)
    static constexpr int NB = 5;                         // rows at a non-periodic end taking the general formulas
    static constexpr int G = (H + R - 1) / R;            // ghost blocks per side
    static constexpr int S = (R % 2 == 0) ? R + 1 : R;
    static constexpr int NS = (32 + 2 * G) * S;          // slots of one line buffer
    // line-buffer stride of the direction-1 passes, whose two threads per row segment take
    // lines 4 apart (16 bytes of lines each): NSY = 4 (mod 8) puts the two halves of a warp
    // on disjoint halves of the banks
    static constexpr int NSY = NS + ((12 - NS % 8) % 8);
    static constexpr int fdiv(int a) { return a >= 0 ? a / R : -((R - 1 - a) / R); }
    // slot offset of row k + m of a lane's block from the block's first slot
    static constexpr int off(int km) { return fdiv(km) * S + (km - fdiv(km) * R); }
    __device__ static __forceinline__ int slot(int i) { const int b = i / R; return (b + G) * S + (i - b * R); }
    __device__ static __forceinline__ int lane_base(int lane) { return (lane + G) * S; }
};

// general row access (runtime row index) for the rows near non-periodic ends
template <typename T, int R>
struct LView {
    using value_type = T;
    const T* F;
    int N, per;
    __device__ __forceinline__ T at(int j) const
    {
        if (per) j = j < 0 ? j + N : (j >= N ? j - N : j);
        return F[LL<R>::slot(j)];
    }
    __device__ __forceinline__ T refl(int j) const
    {
        if (per) j = j < 0 ? j + N : (j >= N ? j - N : j);
        else j = j < 0 ? -j : (j >= N ? 2 * (N - 1) - j : j);
        return F[LL<R>::slot(j)];
    }
};

// compile-time loop
template <int B, int E, typename F>
__device__ __forceinline__ void sfor(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

// ---- row operators ------------------------------------------------------------------------
// Each operator gives the row value at compile-time offsets from the lane's first slot Fb
// (`in`, interior rows), at any row of a non-periodic line from a runtime row index (`gen`),
// and at a compile-time row r of a line of compile-time length NC from the owning lane's Fb
// (`fixed`, the NH rows at each end whose formula differs from the interior one).

// first derivative of Eq. 16: interior a1 (f+1 - f-1) + a2 (f+2 - f-2); non-periodic ends:
// one-sided 4th order at the end node, centred 2nd order at the next
template <typename V>
__device__ __forceinline__ typename V::value_type gen_deriv(const V& v, int i, typename V::value_type a1,
                                                            typename V::value_type a2)
{
    using T = typename V::value_type;
    const int N = v.N;
    if (!v.per) {
        if (i == 0)
            return (T(-25.0) * v.at(0) + T(48.0) * v.at(1) - T(36.0) * v.at(2) + T(16.0) * v.at(3)
                    - T(3.0) * v.at(4)) * T(1.0 / 12.0);
        if (i == N - 1)
            return -(T(-25.0) * v.at(N - 1) + T(48.0) * v.at(N - 2) - T(36.0) * v.at(N - 3) + T(16.0) * v.at(N - 4)
                     - T(3.0) * v.at(N - 5)) * T(1.0 / 12.0);
        if (i == 1 || i == N - 2) return T(0.5) * (v.at(i + 1) - v.at(i - 1));
    }
    return a1 * (v.at(i + 1) - v.at(i - 1)) + a2 * (v.at(i + 2) - v.at(i - 2));
}

// value of compile-time row `row` seen from the lane owning compile-time row r
#define LROW(row) Fb[L::off(r % R + (row) - r)]

template <typename T>
struct OpDeriv {
    T a1, a2;
    static constexpr int NH = 2;
    template <int R, int K>
    __device__ __forceinline__ T in(const T* Fb) const
    {
        using L = LL<R>;
        return a1 * (Fb[L::off(K + 1)] - Fb[L::off(K - 1)]) + a2 * (Fb[L::off(K + 2)] - Fb[L::off(K - 2)]);
    }
    template <typename V>
    __device__ __forceinline__ T gen(const V& v, int i) const { return gen_deriv(v, i, a1, a2); }
    template <int R, int NC, int r>
    __device__ __forceinline__ T fixed(const T* Fb) const
    {
        using L = LL<R>;
        if constexpr (r == 0)
            return (T(-25.0) * LROW(0) + T(48.0) * LROW(1) - T(36.0) * LROW(2) + T(16.0) * LROW(3) - T(3.0) * LROW(4))
                 * T(1.0 / 12.0);
        else if constexpr (r == NC - 1)
            return -(T(-25.0) * LROW(NC - 1) + T(48.0) * LROW(NC - 2) - T(36.0) * LROW(NC - 3) + T(16.0) * LROW(NC - 4)
                     - T(3.0) * LROW(NC - 5)) * T(1.0 / 12.0);
        else
            return T(0.5) * (LROW(r + 1) - LROW(r - 1));   // rows 1 and NC - 2
    }
};

// 5-point fourth difference (the d4 of Eq. 7); within two nodes of a non-periodic end the
// nearest complete stencil
template <typename T>
struct OpD4 {
    static constexpr int NH = 2;
    template <int R, int K>
    __device__ __forceinline__ T in(const T* Fb) const
    {
        using L = LL<R>;
        return Fb[L::off(K - 2)] - T(4) * Fb[L::off(K - 1)] + T(6) * Fb[L::off(K)] - T(4) * Fb[L::off(K + 1)]
             + Fb[L::off(K + 2)];
    }
    template <typename V>
    __device__ __forceinline__ T gen(const V& v, int i) const { return d4_row(v, i); }
    template <int R, int NC, int r>
    __device__ __forceinline__ T fixed(const T* Fb) const
    {
        using L = LL<R>;
        constexpr int c = r < 2 ? 2 : NC - 3;
        return LROW(c - 2) - T(4) * LROW(c - 1) + T(6) * LROW(c) - T(4) * LROW(c + 1) + LROW(c + 2);
    }
};

// truncated 9-point Gaussian (Kawai & Lele's LAD smoothing), even reflection at
// non-periodic ends
template <int NC>
constexpr int lrefl(int j) { return j < 0 ? -j : (j > NC - 1 ? 2 * (NC - 1) - j : j); }

template <typename T>
struct OpGauss {
    static constexpr int NH = 4;
    template <int R, int K>
    __device__ __forceinline__ T in(const T* Fb) const
    {
        using L = LL<R>;
        return T(3565.0 / 10368.0) * Fb[L::off(K)] + T(3091.0 / 12960.0) * (Fb[L::off(K + 1)] + Fb[L::off(K - 1)])
             + T(1997.0 / 25920.0) * (Fb[L::off(K + 2)] + Fb[L::off(K - 2)])
             + T(149.0 / 12960.0) * (Fb[L::off(K + 3)] + Fb[L::off(K - 3)])
             + T(107.0 / 103680.0) * (Fb[L::off(K + 4)] + Fb[L::off(K - 4)]);
    }
    template <typename V>
    __device__ __forceinline__ T gen(const V& v, int i) const { return gauss_rhs(v, i); }
    template <int R, int NC, int r>
    __device__ __forceinline__ T fixed(const T* Fb) const
    {
        using L = LL<R>;
        return T(3565.0 / 10368.0) * LROW(r) + T(3091.0 / 12960.0) * (LROW(lrefl<NC>(r + 1)) + LROW(lrefl<NC>(r - 1)))
             + T(1997.0 / 25920.0) * (LROW(lrefl<NC>(r + 2)) + LROW(lrefl<NC>(r - 2)))
             + T(149.0 / 12960.0) * (LROW(lrefl<NC>(r + 3)) + LROW(lrefl<NC>(r - 3)))
             + T(107.0 / 103680.0) * (LROW(lrefl<NC>(r + 4)) + LROW(lrefl<NC>(r - 4)));
    }
};
// delta form of the filter of Eq. 21 (right-hand side from second differences; the solve
// gives the correction), order 2hw with hw = min(5, distance to a non-periodic end), end
// nodes unfiltered
template <typename T>
struct OpFilter {
    const T (*cf)[6];
    static constexpr int NH = 5;
    template <int R, int K>
    __device__ __forceinline__ T in(const T* Fb) const
    {
        using L = LL<R>;
        const T f0 = Fb[L::off(K)];
        T s = T(0);
        sfor<0, 5>([&](auto mc) {
            constexpr int m = 5 - decltype(mc)::value;
            s += cf[5][m] * ((Fb[L::off(K + m)] - f0) + (Fb[L::off(K - m)] - f0));
        });
        return s;
    }
    template <typename V>
    __device__ __forceinline__ T gen(const V& v, int i) const { return filter_rhs(v, i, cf); }
    template <int R, int NC, int r>
    __device__ __forceinline__ T fixed(const T* Fb) const
    {
        using L = LL<R>;
        constexpr int e = r < NC - 1 - r ? r : NC - 1 - r;
        constexpr int hw = e < 5 ? e : 5;
        if constexpr (hw == 0) {
            return T(0);
        } else {
            const T f0 = LROW(r);
            T s = T(0);
            sfor<0, hw>([&](auto mc) {
                constexpr int m = hw - decltype(mc)::value;
                s += cf[hw][m] * ((LROW(r + m) - f0) + (LROW(r - m) - f0));
            });
            return s;
        }
    }
};

#undef LROW

// x[k] = row lane*R + k of a line operator over buffer F (rows >= N give 0).
// NC > 0: a non-periodic line of compile-time length NC: every row takes the interior formula
// and the lanes owning the NH end rows at each end patch them at compile-time positions.
// NC == 0: runtime length N; on non-periodic lines the rows within NB of an end take the
// general formula, evaluated by lanes 0 .. 2NB-1 into the warp's scratch and picked up by the
// owning lane.
template <int NC, typename T, int R, typename Op>
__device__ __forceinline__ void rows_of(T (&x)[R], const T* F, int lane, int N, int per, T* scr, const Op& op)
{
    const T* Fb = F + LL<R>::lane_base(lane);
    if constexpr (NC > 0) {
        constexpr int E = (NC - 1) / R, KE = (NC - 1) % R;
        sfor<0, R>([&](auto kc) { x[decltype(kc)::value] = op.template in<R, decltype(kc)::value>(Fb); });
        if (lane > E) {
            sfor<0, R>([&](auto kc) { x[decltype(kc)::value] = T(0); });
        } else if (lane == E) {
            sfor<KE + 1, R>([&](auto kc) { x[decltype(kc)::value] = T(0); });
        }
        sfor<0, Op::NH>([&](auto tc) {
            constexpr int rh = decltype(tc)::value, rt = NC - 1 - decltype(tc)::value;
            if (lane == rh / R) x[rh % R] = op.template fixed<R, NC, rh>(Fb);
            if (lane == rt / R) x[rt % R] = op.template fixed<R, NC, rt>(Fb);
        });
    } else {
        constexpr int NB = LL<R>::NB;
        if (!per) {
            if (lane < 2 * NB) {
                const int i = lane < NB ? lane : N - 2 * NB + lane;
                scr[lane] = op.gen(LView<T, R>{F, N, per}, i);
            }
            __syncwarp();
        }
        sfor<0, R>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const int i = lane * R + k;
            T v = op.template in<R, k>(Fb);
            if (!per) {
                if (k < NB && i < NB) v = scr[i];
                const int t = i - (N - NB);
                if (t >= 0 && t < NB) v = scr[NB + t];
            }
            x[k] = i < N ? v : T(0);
        });
        if (!per) __syncwarp();
    }
}

template <typename T, int R>
__device__ __forceinline__ void store_rows(T* F, const T (&x)[R], int lane)
{
    T* Fb = F + LL<R>::lane_base(lane);
#pragma unroll
    for (int k = 0; k < R; k++) Fb[k] = x[k];
}

// wrapped rows of a periodic line (N = 32 R) into the ghost blocks; called by the whole warp
template <int R, typename T>
__device__ __forceinline__ void ghost_fill(T* F, int lane)
{
    using L = LL<R>;
    for (int t = lane; t < L::G * L::S; t += 32) {
        F[t] = F[32 * L::S + t];
        F[(32 + L::G) * L::S + t] = F[L::G * L::S + t];
    }
}

// fields solved together: one load of each partition-table value per group
template <int R, int NF>
struct LGroup {
    static constexpr int GF = R <= 9 ? NF : (R <= 17 ? (NF < 2 ? NF : 2) : 1);
};

// first derivatives (Eq. 16, solved along the line when compact) of the fields F[0 .. NF-1]
// in place: each group's rows are formed, solved and written back after the whole warp has
// read the group's fields
template <int NC, typename T, int R, int NF>
__device__ __forceinline__ void deriv_fields(T* const (&F)[NF], int lane, int N, int per, T* scr,
                                             const OpDeriv<T>& op, int implicit, const PartTab<T>& tb)
{
    constexpr int GF = LGroup<R, NF>::GF;
#pragma unroll
    for (int f0 = 0; f0 < NF; f0 += GF) {
        T x[GF][R];
#pragma unroll
        for (int f = 0; f < GF; f++) rows_of<NC, T, R>(x[f], F[f0 + f], lane, N, per, scr, op);
        if (implicit) part_solve<T, R, GF>(x, tb, lane);
        __syncwarp();
#pragma unroll
        for (int f = 0; f < GF; f++) store_rows<T, R>(F[f0 + f], x[f], lane);
        __syncwarp();
    }
}

// ---- 16-byte vector access: VW consecutive values of T along i ------------------------------
template <typename T>
struct VecT;
template <>
struct VecT<float> {
    using V = float4;
    using MV = uchar4;
    static constexpr int n = 4;
};
template <>
struct VecT<double> {
    using V = double2;
    using MV = uchar2;
    static constexpr int n = 2;
};

template <typename T>
__device__ __forceinline__ void unpack(const typename VecT<T>::V& v, T (&o)[VecT<T>::n])
{
    if constexpr (VecT<T>::n == 4) {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    } else {
        o[0] = v.x;
        o[1] = v.y;
    }
}
// read-only data of this launch
template <typename T>
__device__ __forceinline__ void vldg(const T* p, T (&o)[VecT<T>::n])
{
    unpack<T>(__ldg(reinterpret_cast<const typename VecT<T>::V*>(p)), o);
}
// data this launch also writes (each element by the thread that reads it)
template <typename T>
__device__ __forceinline__ void vld(const T* p, T (&o)[VecT<T>::n])
{
    unpack<T>(*reinterpret_cast<const typename VecT<T>::V*>(p), o);
}
template <typename T>
__device__ __forceinline__ void vst(T* p, const T (&o)[VecT<T>::n])
{
    typename VecT<T>::V v;
    if constexpr (VecT<T>::n == 4) {
        v.x = o[0];
        v.y = o[1];
        v.z = o[2];
        v.w = o[3];
    } else {
        v.x = o[0];
        v.y = o[1];
    }
    *reinterpret_cast<typename VecT<T>::V*>(p) = v;
}
template <typename T>
__device__ __forceinline__ void vldm(const uint8_t* p, uint8_t (&o)[VecT<T>::n])
{
    const typename VecT<T>::MV m = *reinterpret_cast<const typename VecT<T>::MV*>(p);
    if constexpr (VecT<T>::n == 4) {
        o[0] = m.x;
        o[1] = m.y;
        o[2] = m.z;
        o[3] = m.w;
    } else {
        o[0] = m.x;
        o[1] = m.y;
    }
}

// ---- X: direction-0 pass ------------------------------------------------------------------
// One warp per line; the line's global accesses are 16-byte vectors of VW consecutive nodes
// (lane v of the warp takes vectors v, v + 32, ...), needing n0 % VW == 0.
template <typename T>
struct LXShape {
    static constexpr int W = 4;          // warps (= lines) per block
};

template <typename T, typename M, int R, int NF>
__global__ void __launch_bounds__(32 * LXShape<T>::W) k_l2_x(L2Args<T, M> a, PartTab<T> tb)
{
    static_assert(std::is_same<T, M>::value, "the loop reads its metrics in the state precision");
    extern __shared__ __align__(16) unsigned char smraw[];
    using L = LL<R>;
    constexpr int W = LXShape<T>::W, VW = VecT<T>::n;
    const Dims& D = a.D;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = a.kbeg * D.n[1] + blockIdx.x * W + w;
    if (q >= (a.kbeg + a.kcnt) * D.n[1]) return;   // whole warps leave; no block barrier here
    const int N = D.n[0], per = D.per[0], nv = N / VW;
    T* base = reinterpret_cast<T*>(smraw) + (size_t)w * ((NF + 1) * L::NS + 16);
    T* P = base;                                    // phi, then C|LAD|, then its smoothed value
    T* F[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) F[f] = base + (f + 1) * L::NS;
    T* scr = base + (NF + 1) * L::NS;
    const long long e0 = D.line_base(0, q), tot = D.total;
    const M* xi = a.xi;
    const bool lad = a.lad;
    const OpDeriv<T> od{a.a1, a.a2};

    for (int v = lane; v < nv; v += 32) {
        T t[VW];
        vldg(a.src + e0 + (long long)v * VW, t);
#pragma unroll
        for (int u = 0; u < VW; u++) P[L::slot(v * VW + u)] = t[u];
    }
    __syncwarp();
    if (per) {
        ghost_fill<R>(P, lane);
        __syncwarp();
    }
    // D_0(phi) and d4_0(phi) of the lane's rows
    {
        T x[R];
        rows_of<0, T, R>(x, P, lane, N, per, scr, od);
        if (a.implicit) part_solve<T, R>(x, tb, lane);
        store_rows<T, R>(F[0], x, lane);
        if (lad) {
            rows_of<0, T, R>(x, P, lane, N, per, scr, OpD4<T>{});
            store_rows<T, R>(F[1], x, lane);
        }
    }
    __syncwarp();
    // D_0 out; C|s_0 d4_0 + s_1 d4_1| into P; U (and n) into F
    for (int v = lane; v < nv; v += 32) {
        const long long e = e0 + (long long)v * VW;
        T d1[VW], x0[VW], x1[VW], x3[VW], x4[VW], la[VW], l1[VW], d0[VW];
        vldg(a.D1 + e, d1);
        vldg(xi + e, x0);
        vldg(xi + tot + e, x1);
        vldg(xi + 3 * tot + e, x3);
        vldg(xi + 4 * tot + e, x4);
        if (lad) {
            vldg(a.lads + e, la);
            vldg(a.L1 + e, l1);
        }
#pragma unroll
        for (int u = 0; u < VW; u++) {
            const int s = L::slot(v * VW + u);
            d0[u] = F[0][s];
            if (lad) {
                const T v0 = T(la[u] * M(F[1][s])) + l1[u];
                P[s] = T(a.C_lad) * (v0 < T(0) ? -v0 : v0);
            }
            const M dd0 = M(d0[u]), dd1 = M(d1[u]);
            const M ux = x0[u] * dd0 + x3[u] * dd1;   // xi_x D0 + eta_x D1
            const M uy = x1[u] * dd0 + x4[u] * dd1;   // xi_y D0 + eta_y D1
            F[0][s] = T(ux);
            F[1][s] = T(uy);
            if constexpr (NF == 4) {
                const M ig = M(1) / (sqrt(ux * ux + uy * uy) + M(a.eps0));
                F[2][s] = T(ux * ig);
                F[3][s] = T(uy * ig);
            }
        }
        vst(a.D0 + e, d0);
    }
    __syncwarp();
    if (per) {
        if (lad) ghost_fill<R>(P, lane);
#pragma unroll
        for (int f = 0; f < NF; f++) ghost_fill<R>(F[f], lane);
        __syncwarp();
    }
    // Gaussian along direction 0 (even reflection at non-periodic ends)
    if (lad) {
        T x[R];
        rows_of<0, T, R>(x, P, lane, N, per, scr, OpGauss<T>{});
        __syncwarp();
        store_rows<T, R>(P, x, lane);
    }
    // direction-0 derivatives of U (and n)
    deriv_fields<0, T, R, NF>(F, lane, N, per, scr, od, a.implicit, tb);
    // metric weights: the direction-0 parts of div(U) and div(n)
    for (int v = lane; v < nv; v += 32) {
        const long long e = e0 + (long long)v * VW;
        T x0[VW], x1[VW], lp[VW], kp[VW], gg[VW];
        vldg(xi + e, x0);
        vldg(xi + tot + e, x1);
#pragma unroll
        for (int u = 0; u < VW; u++) {
            const int s = L::slot(v * VW + u);
            lp[u] = T(M(x0[u]) * M(F[0][s]) + M(x1[u]) * M(F[1][s]));
            if constexpr (NF == 4) kp[u] = T(M(x0[u]) * M(F[2][s]) + M(x1[u]) * M(F[3][s]));
            gg[u] = P[s];
        }
        vst(a.LAP0 + e, lp);
        if constexpr (NF == 4) vst(a.KAP0 + e, kp);
        if (lad) vst(a.G0 + e, gg);
    }
}

// ---- Y: direction-1 pass ------------------------------------------------------------------
// W neighbouring lines per block, one warp per line in the line phases; in the pointwise
// phases two threads share a row of the block's lines, each with a 16-byte vector of VW
// lines (W = 2 VW: a 32-byte row segment), rows tid/2, tid/2 + 16 W, ...  Needs n0 % W == 0,
// so that a block's lines are consecutive nodes of one row.  NC > 0: the lines have NC nodes
// (compile time; the O-grid radial sizes 32 (R - 1) + 1), else D.n[1].
template <typename T>
struct LYShape {
    static constexpr int W = 32 / sizeof(T);   // lines per block: 32-byte row segments
};

// resident blocks per SM asked of the compiler (lines up to 544 nodes: three)
constexpr int ly_minb(int R) { return R <= 17 ? 3 : 1; }

// buffers of a Y block, each W lines x NS slots: 0 U_x, 1 U_y, 2 |U|^2 then the stage value
// before the boundary conditions, 3 G0 then its smoothed value, 4 n_x, 5 n_y; buffer 0 then
// holds the stage value after the boundary conditions
template <int NF>
struct LYBufs {
    static constexpr int N = NF == 4 ? 6 : 4;
};

template <typename T, typename M, int R, int NF, int NC>
__global__ void __launch_bounds__(32 * LYShape<T>::W, ly_minb(R)) k_l2_y(L2Args<T, M> a, PartTab<T> tb)
{
    static_assert(std::is_same<T, M>::value, "the loop reads its metrics in the state precision");
    extern __shared__ __align__(16) unsigned char smraw[];
    using L = LL<R>;
    constexpr int W = LYShape<T>::W, VW = VecT<T>::n, JS = 16 * W;
    constexpr int NBUF = LYBufs<NF>::N;
    const Dims& D = a.D;
    const int N = NC > 0 ? NC : D.n[1], per = NC > 0 ? 0 : D.per[1];
    const int q0 = a.kbeg * D.n[0] + blockIdx.x * W;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    T* sm = reinterpret_cast<T*>(smraw);
    auto buf = [&](int b, int l) { return sm + (size_t)(b * W + l) * L::NSY; };
    T* scr = sm + (size_t)NBUF * W * L::NSY + 16 * w;
    const long long tot = D.total, st = D.pitch;
    const M* xi = a.xi;
    const bool lad = a.lad;
    const OpDeriv<T> od{a.a1, a.a2};
    const int lv0 = (tid & 1) * VW;                        // first of the thread's VW lines
    const long long lb = D.line_base(1, q0 + lv0);
    const int jr = tid >> 1;

    // U, |U|^2 (and n) of every node; G0
    for (int j = jr; j < N; j += JS) {
        const long long e = lb + (long long)j * st;
        const int s = L::slot(j);
        T d0[VW], d1[VW], x0[VW], x1[VW], x3[VW], x4[VW], gg[VW];
        vldg(a.D0 + e, d0);
        vldg(a.D1 + e, d1);
        vldg(xi + e, x0);
        vldg(xi + tot + e, x1);
        vldg(xi + 3 * tot + e, x3);
        vldg(xi + 4 * tot + e, x4);
        if (lad) vldg(a.G0 + e, gg);
#pragma unroll
        for (int u = 0; u < VW; u++) {
            const int l = lv0 + u;
            const M dd0 = M(d0[u]), dd1 = M(d1[u]);
            const M ux = x0[u] * dd0 + x3[u] * dd1;
            const M uy = x1[u] * dd0 + x4[u] * dd1;
            const T tx = T(ux), ty = T(uy);
            buf(0, l)[s] = tx;
            buf(1, l)[s] = ty;
            buf(2, l)[s] = tx * tx + ty * ty;
            if (lad) buf(3, l)[s] = gg[u];
            if constexpr (NF == 4) {
                const M ig = M(1) / (sqrt(ux * ux + uy * uy) + M(a.eps0));
                buf(4, l)[s] = T(ux * ig);
                buf(5, l)[s] = T(uy * ig);
            }
        }
    }
    __syncthreads();
    {
        if (per) {
            for (int b = 0; b < NBUF; b++) ghost_fill<R>(buf(b, w), lane);
            __syncwarp();
        }
        // Gaussian along direction 1: the second half of the LAD smoothing
        if (lad) {
            T x[R];
            rows_of<NC, T, R>(x, buf(3, w), lane, N, per, scr, OpGauss<T>{});
            __syncwarp();
            store_rows<T, R>(buf(3, w), x, lane);
        }
        if constexpr (NF == 4) {
            T* const F[4] = {buf(0, w), buf(1, w), buf(4, w), buf(5, w)};
            deriv_fields<NC, T, R, 4>(F, lane, N, per, scr, od, a.implicit, tb);
        } else {
            T* const F[2] = {buf(0, w), buf(1, w)};
            deriv_fields<NC, T, R, 2>(F, lane, N, per, scr, od, a.implicit, tb);
        }
    }
    __syncthreads();
    // right-hand side, local time step, RK4 stage and Dirichlet nodes (pointwise): the stage
    // value before the boundary conditions into buffer 2, after them into buffer 0 and out;
    // the far-field / Neumann end nodes are redone below from their neighbours
    for (int j = jr; j < N; j += JS) {
        const long long e = lb + (long long)j * st;
        const int s = L::slot(j);
        T x3[VW], x4[VW], lp0[VW], kp0[VW], src[VW], phn[VW], ac[VW], dt[VW], s1[VW], s2[VW], nv[VW];
        uint8_t mk[VW];
        vldg(xi + 3 * tot + e, x3);
        vldg(xi + 4 * tot + e, x4);
        vldg(a.LAP0 + e, lp0);
        vldg(a.phin + e, phn);
        vldm<T>(a.mask + e, mk);
        if (!a.poisson) {
            vldg(a.src + e, src);
            if constexpr (NF == 4) vldg(a.KAP0 + e, kp0);
        }
        if (a.stage == 0) {
            vldg(a.sig2 + e, s2);
            if (!a.poisson) vldg(a.sig1 + e, s1);
        } else {
            vld(a.dtv + e, dt);
            vld(a.acc + e, ac);
        }
#pragma unroll
        for (int u = 0; u < VW; u++) {
            const int l = lv0 + u;
            const T lap = lp0[u] + T(M(x3[u]) * M(buf(0, l)[s]) + M(x4[u]) * M(buf(1, l)[s]));
            T Rv, gam = T(0), v = T(0), gm = T(0);
            if (a.poisson) {
                Rv = T(1) + lap;                                                 // Eq. 19
            } else {
                const T g2 = buf(2, l)[s];
                gm = sqrt(g2);
                const T php = src[u] > T(0) ? src[u] : T(0);
                if (lad) {                                                       // Eq. 7
                    const T g1 = T(a.eps) * php, gl = buf(3, l)[s];
                    gam = g1 < gl ? g1 : gl;
                } else if (a.equation == WD_HJ_STD) {
                    gam = T(a.eps) * php;                                        // Eq. 6
                }
                if constexpr (NF == 4) {                                         // Eq. 25
                    const T kap = kp0[u] + T(M(x3[u]) * M(buf(4, l)[s]) + M(x4[u]) * M(buf(5, l)[s]));
                    v = T(0.001) * (T(1) - gm) * (T(1) - gm);
                    T corr = gm * kap;
                    corr = corr > T(0) ? corr : T(0);
                    Rv = T(1) + (gam + v) * (lap - corr) - g2;
                } else {
                    Rv = T(1) + gam * lap - g2;                                  // Eqs. 5, 18
                }
            }
            if (a.stage == 0) {
                if (a.poisson) dt[u] = T(a.cfl) / T(s2[u]);
                else {
                    const T am = gm > T(1) ? gm : T(1);
                    dt[u] = T(a.cfl) / (T(s1[u]) * am + (gam + v) * T(s2[u]));
                }
            }
            T out;
            if (a.stage == 0) {
                ac[u] = Rv * T(1.0 / 6.0);
                out = phn[u] + T(0.5) * dt[u] * Rv;
            } else if (a.stage == 1) {
                ac[u] += Rv * T(1.0 / 3.0);
                out = phn[u] + T(0.5) * dt[u] * Rv;
            } else if (a.stage == 2) {
                ac[u] += Rv * T(1.0 / 3.0);
                out = phn[u] + dt[u] * Rv;
            } else {
                out = phn[u] + dt[u] * (ac[u] + Rv * T(1.0 / 6.0));
            }
            buf(2, l)[s] = out;
            nv[u] = mk[u] ? (a.poisson ? T(0) : __ldg(a.dval + e + u)) : out;
            buf(0, l)[s] = nv[u];
        }
        if (a.stage == 0) vst(a.dtv + e, dt);
        if (a.stage < 3) vst(a.acc + e, ac);
        vst(a.dst + e, nv);
    }
    __syncthreads();
    // far-field / Neumann ends of the lines from the stage values of their inner neighbours
    // (before the Dirichlet reset), then the Dirichlet reset of the end node itself
    if (!per && tid < 2 * W) {
        const int l = tid >> 1, side = tid & 1;
        int kind = side ? a.bchi1 : a.bclo1;
        if (kind == WD_BC_FARFIELD || kind == WD_BC_NEUMANN) {
            if (a.poisson) kind = WD_BC_NEUMANN;
            const T* V = buf(2, l);
            const T v1 = V[L::slot(side ? N - 2 : 1)], v2 = V[L::slot(side ? N - 3 : 2)];
            T nv;
            if (kind == WD_BC_NEUMANN) nv = v1;
            else {
                const int qline = q0 + l;   // = i + n0 k
                const long long fi = (long long)(qline / D.n[0]) + (long long)D.n[2] * (qline % D.n[0]);
                nv = v1 + T((side ? a.ffr_hi : a.ffr_lo)[fi]) * (v1 - v2);
            }
            const int j = side ? N - 1 : 0;
            const long long e = D.line_base(1, q0 + l) + (long long)j * st;
            if (a.mask[e]) nv = a.poisson ? T(0) : __ldg(a.dval + e);
            buf(0, l)[L::slot(j)] = nv;
            a.dst[e] = nv;
        }
    }
    if (!a.next) return;
    __syncthreads();
    // D_1 and s_1 d4_1 of the stage value, for the next stage's direction-0 pass (into buffers
    // 1 and 3, then out with coalesced row segments)
    {
        T* P = buf(0, w);
        if (per) {
            ghost_fill<R>(P, lane);
            __syncwarp();
        }
        T x[R];
        rows_of<NC, T, R>(x, P, lane, N, per, scr, od);
        if (a.implicit) part_solve<T, R>(x, tb, lane);
        store_rows<T, R>(buf(1, w), x, lane);
        if (lad) {
            rows_of<NC, T, R>(x, P, lane, N, per, scr, OpD4<T>{});
            store_rows<T, R>(buf(3, w), x, lane);
        }
    }
    __syncthreads();
    for (int j = jr; j < N; j += JS) {
        const long long e = lb + (long long)j * st;
        const int s = L::slot(j);
        T ls[VW], o1[VW], o2[VW];
        if (lad) vldg(a.lads + tot + e, ls);
#pragma unroll
        for (int u = 0; u < VW; u++) {
            o1[u] = buf(1, lv0 + u)[s];
            if (lad) o2[u] = T(M(ls[u]) * M(buf(3, lv0 + u)[s]));
        }
        vst(a.D1 + e, o1);
        if (lad) vst(a.L1 + e, o2);
    }
}

// ---- Y0: D_1 and s_1 d4_1 of phi^n (the first stage's direction-0 pass needs them) ----------
template <typename T, typename M, int R, int NC>
__global__ void __launch_bounds__(32 * LYShape<T>::W, ly_minb(R)) k_l2_y0(L2Args<T, M> a, PartTab<T> tb)
{
    static_assert(std::is_same<T, M>::value, "the loop reads its metrics in the state precision");
    extern __shared__ __align__(16) unsigned char smraw[];
    using L = LL<R>;
    constexpr int W = LYShape<T>::W, VW = VecT<T>::n, JS = 16 * W;
    const Dims& D = a.D;
    const int N = NC > 0 ? NC : D.n[1], per = NC > 0 ? 0 : D.per[1];
    const int q0 = a.kbeg * D.n[0] + blockIdx.x * W;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    T* sm = reinterpret_cast<T*>(smraw);
    auto buf = [&](int b, int l) { return sm + (size_t)(b * W + l) * L::NSY; };
    T* scr = sm + (size_t)3 * W * L::NSY + 16 * w;
    const long long tot = D.total, st = D.pitch;
    const bool lad = a.lad;
    const int lv0 = (tid & 1) * VW;
    const long long lb = D.line_base(1, q0 + lv0);
    const int jr = tid >> 1;
    for (int j = jr; j < N; j += JS) {
        T t[VW];
        vldg(a.src + lb + (long long)j * st, t);
        const int s = L::slot(j);
#pragma unroll
        for (int u = 0; u < VW; u++) buf(0, lv0 + u)[s] = t[u];
    }
    __syncthreads();
    {
        T* P = buf(0, w);
        if (per) {
            ghost_fill<R>(P, lane);
            __syncwarp();
        }
        T x[R];
        rows_of<NC, T, R>(x, P, lane, N, per, scr, OpDeriv<T>{a.a1, a.a2});
        if (a.implicit) part_solve<T, R>(x, tb, lane);
        store_rows<T, R>(buf(1, w), x, lane);
        if (lad) {
            rows_of<NC, T, R>(x, P, lane, N, per, scr, OpD4<T>{});
            store_rows<T, R>(buf(2, w), x, lane);
        }
    }
    __syncthreads();
    for (int j = jr; j < N; j += JS) {
        const long long e = lb + (long long)j * st;
        const int s = L::slot(j);
        T ls[VW], o1[VW], o2[VW];
        if (lad) vldg(a.lads + tot + e, ls);
#pragma unroll
        for (int u = 0; u < VW; u++) {
            o1[u] = buf(1, lv0 + u)[s];
            if (lad) o2[u] = T(M(ls[u]) * M(buf(2, lv0 + u)[s]));
        }
        vst(a.D1 + e, o1);
        if (lad) vst(a.L1 + e, o2);
    }
}

// ---- change-norm accumulation ------------------------------------------------------------
// Sum of squares and max of a thread's changes.  A float state keeps the sum as an unevaluated
// pair hi + lo of floats (error-free products and sums), so that the per-thread partial is as
// exact as a double sum without double arithmetic (1/64 of the float rate on GB300); the
// sums across threads and blocks are taken in double.
template <typename T>
struct NormAcc {
    double ss = 0.0, mx = 0.0;
    __device__ __forceinline__ void add(T d)
    {
        ss += double(d) * double(d);
        mx = fmax(mx, fabs(double(d)));
    }
    __device__ __forceinline__ double sum() const { return ss; }
};
template <>
struct NormAcc<float> {
    float hi = 0.f, lo = 0.f, mx = 0.f;
    __device__ __forceinline__ void add(float d)
    {
        const float p = __fmul_rn(d, d);
        const float pe = fmaf(d, d, -p);                     // p + pe = d^2 exactly
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));   // hi + p = s + e
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, pe));
        mx = fmaxf(mx, fabsf(d));
    }
    __device__ __forceinline__ double sum() const { return double(hi) + double(lo); }
};

// ---- FX: filter along direction 0 (src into dst) ---------------------------------------------
template <typename T, typename M, int R>
__global__ void __launch_bounds__(32 * LXShape<T>::W) k_l2_fx(L2Args<T, M> a, PartTab<T> tb)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    using L = LL<R>;
    constexpr int W = LXShape<T>::W, VW = VecT<T>::n;
    const Dims& D = a.D;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = a.kbeg * D.n[1] + blockIdx.x * W + w;
    if (q >= (a.kbeg + a.kcnt) * D.n[1]) return;
    const int N = D.n[0], per = D.per[0], nv = N / VW;
    T* P = reinterpret_cast<T*>(smraw) + (size_t)w * (L::NS + 16);
    T* scr = P + L::NS;
    const long long e0 = D.line_base(0, q);
    for (int v = lane; v < nv; v += 32) {
        T t[VW];
        vldg(a.src + e0 + (long long)v * VW, t);
#pragma unroll
        for (int u = 0; u < VW; u++) P[L::slot(v * VW + u)] = t[u];
    }
    __syncwarp();
    if (per) {
        ghost_fill<R>(P, lane);
        __syncwarp();
    }
    T x[R];
    rows_of<0, T, R>(x, P, lane, N, per, scr, OpFilter<T>{a.cf});
    if (tb.implicit) part_solve<T, R>(x, tb, lane);
    const T* Fb = P + L::lane_base(lane);
#pragma unroll
    for (int k = 0; k < R; k++) x[k] += Fb[k];   // delta form: f + (fh - f)
    __syncwarp();
    store_rows<T, R>(P, x, lane);
    __syncwarp();
    for (int v = lane; v < nv; v += 32) {
        T t[VW];
#pragma unroll
        for (int u = 0; u < VW; u++) t[u] = P[L::slot(v * VW + u)];
        vst(a.dst + e0 + (long long)v * VW, t);
    }
}

// ---- FY: filter along a strided direction DIR (1, or 2 of a 3-D grid); with a.commit also
// the line boundary conditions (far-field / Neumann ends of 2-D direction-1 lines, Dirichlet
// nodes), the commit of the new state and the change norms, else the filtered field into dst
// Direction-2 lines of a 3-D grid lie a whole plane apart: their blocks take 32 neighbouring
// lines (128-byte row segments), each warp solving 32 / NW of them.
template <typename T, int DIR, bool WIDE = false>
struct LFShape {
    static constexpr int NW = LYShape<T>::W;                             // warps per block
    static constexpr int W = (DIR == 2 || WIDE) ? 32 : LYShape<T>::W;    // lines per block
};

template <typename T, typename M, int R, int NC, int DIR, bool WIDE = false>
__global__ void __launch_bounds__(32 * LFShape<T, DIR, WIDE>::NW, ly_minb(R)) k_l2_fy(L2Args<T, M> a, PartTab<T> tb)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double s_ss[LFShape<T, DIR, WIDE>::NW], s_mx[LFShape<T, DIR, WIDE>::NW];
    __shared__ int s_last;
    using L = LL<R>;
    constexpr int W = LFShape<T, DIR, WIDE>::W, NW = LFShape<T, DIR, WIDE>::NW, VW = VecT<T>::n;
    constexpr int TPR = W / VW;                 // threads per row segment
    constexpr int JS = 32 * NW / TPR;           // rows per sweep
    const Dims& D = a.D;
    const int N = NC > 0 ? NC : D.n[DIR], per = NC > 0 ? 0 : D.per[DIR];
    const int q0 = (DIR == 1 ? a.kbeg * D.n[0] : 0) + blockIdx.x * W;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    T* sm = reinterpret_cast<T*>(smraw);
    auto buf = [&](int l) { return sm + (size_t)l * L::NS; };
    T* scr = sm + (size_t)W * L::NS + 16 * w;
    const long long st = D.stride(DIR);
    const int lv0 = (tid % TPR) * VW;
    const long long lb = D.line_base(DIR, q0 + lv0);
    const int jr = tid / TPR;
    for (int j = jr; j < N; j += JS) {
        T t[VW];
        vldg(a.src + lb + (long long)j * st, t);
        const int s = L::slot(j);
#pragma unroll
        for (int u = 0; u < VW; u++) buf(lv0 + u)[s] = t[u];
    }
    __syncthreads();
    if (a.filter)
        for (int l = w; l < W; l += NW) {
            T* P = buf(l);
            if (per) {
                ghost_fill<R>(P, lane);
                __syncwarp();
            }
            T x[R];
            rows_of<NC, T, R>(x, P, lane, N, per, scr, OpFilter<T>{a.cf});
            if (tb.implicit) part_solve<T, R>(x, tb, lane);
            const T* Fb = P + L::lane_base(lane);
#pragma unroll
            for (int k = 0; k < R; k++) x[k] += Fb[k];
            __syncwarp();
            store_rows<T, R>(P, x, lane);
            __syncwarp();
        }
    __syncthreads();
    if (!a.commit) {
        for (int j = jr; j < N; j += JS) {
            const int s = L::slot(j);
            T nv[VW];
#pragma unroll
            for (int u = 0; u < VW; u++) nv[u] = buf(lv0 + u)[s];
            vst(a.dst + lb + (long long)j * st, nv);
        }
        return;
    }
    // far-field / Neumann end rows (2-D direction-1 lines) are committed by the end threads below
    const bool ff_lo = DIR == 1 && D.ndim == 2 && !per && (a.bclo1 == WD_BC_FARFIELD || a.bclo1 == WD_BC_NEUMANN);
    const bool ff_hi = DIR == 1 && D.ndim == 2 && !per && (a.bchi1 == WD_BC_FARFIELD || a.bchi1 == WD_BC_NEUMANN);
    NormAcc<T> acc;
    for (int j = jr; j < N; j += JS) {
        if ((j == 0 && ff_lo) || (j == N - 1 && ff_hi)) continue;
        const long long e = lb + (long long)j * st;
        const int s = L::slot(j);
        T ov[VW], nv[VW];
        uint8_t mk[VW];
        vld(a.phin + e, ov);
        vldm<T>(a.mask + e, mk);
#pragma unroll
        for (int u = 0; u < VW; u++) {
            nv[u] = buf(lv0 + u)[s];
            if (mk[u]) nv[u] = a.poisson ? T(0) : __ldg(a.dval + e + u);
            else acc.add(nv[u] - ov[u]);
        }
        vst(a.phin_w + e, nv);
    }
    if (tid < 2 * W) {
        const int l = tid >> 1, side = tid & 1;
        if (side ? ff_hi : ff_lo) {
            const int kind = a.poisson ? WD_BC_NEUMANN : (side ? a.bchi1 : a.bclo1);
            const T* V = buf(l);
            const T v1 = V[L::slot(side ? N - 2 : 1)], v2 = V[L::slot(side ? N - 3 : 2)];
            T nv;
            if (kind == WD_BC_NEUMANN) nv = v1;
            else {
                const int qline = q0 + l;   // = i + n0 k
                const long long fi = (long long)(qline / D.n[0]) + (long long)D.n[2] * (qline % D.n[0]);
                nv = v1 + T((side ? a.ffr_hi : a.ffr_lo)[fi]) * (v1 - v2);
            }
            const long long e = D.line_base(DIR, q0 + l) + (long long)(side ? N - 1 : 0) * st;
            const T ov = a.phin[e];
            if (a.mask[e]) nv = a.poisson ? T(0) : __ldg(a.dval + e);
            else acc.add(nv - ov);
            a.phin_w[e] = nv;
        }
    }
    // block partials, then the last block of the launch reduces the partials of each of its
    // stacked grids in a fixed order (the blocks of grid k are [k bpm, (k + 1) bpm))
    double ss = acc.sum(), mx = double(acc.mx);
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        s_ss[w] = ss;
        s_mx[w] = mx;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0, m = 0.0;
        for (int k = 0; k < NW; k++) {
            t += s_ss[k];
            m = fmax(m, s_mx[k]);
        }
        const int b = q0 / W;   // block index within the whole batch
        a.partial[2 * b] = t;
        a.partial[2 * b + 1] = m;
        __threadfence();
        s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // one warp per grid, whatever the part size, so that the order of the sums is the same
    // however the batch is split into parts
    const int bpm = (DIR == 1 ? D.n[0] : D.nlines(2)) / W;
    for (int k = a.kbeg + w; k < a.kbeg + a.kcnt; k += NW) {
        double t = 0.0, m = 0.0;
        for (int b = k * bpm + lane; b < (k + 1) * bpm; b += 32) {
            t += __ldcg(a.partial + 2 * b);
            m = fmax(m, __ldcg(a.partial + 2 * b + 1));
        }
        for (int o = 16; o > 0; o >>= 1) {
            t += __shfl_down_sync(0xffffffffu, t, o);
            m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        }
        if (lane == 0) {
            a.result[2 * k] = t;
            a.result[2 * k + 1] = m;
        }
    }
    __syncthreads();
    if (tid == 0) *a.counter = 0u;
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------

static const size_t L2_SMEM_LIMIT = 200 * 1024;

template <int R>
static size_t l2_ns() { return (size_t)LL<R>::NS; }

// shared memory of a launch (bytes)
template <typename T, int R>
static size_t l2_smem(int which, int nf)
{
    if (which == L2_X) return (size_t)LXShape<T>::W * ((nf + 1) * l2_ns<R>() + 16) * sizeof(T);
    if (which == L2_FX) return (size_t)LXShape<T>::W * (l2_ns<R>() + 16) * sizeof(T);
    if (which == L2_FY) return ((size_t)LYShape<T>::W * l2_ns<R>() + 16 * LYShape<T>::W) * sizeof(T);
    if (which == L2_Y) return ((size_t)(nf == 4 ? 6 : 4) * LYShape<T>::W * LL<R>::NSY + 16 * LYShape<T>::W) * sizeof(T);
    return ((size_t)3 * LYShape<T>::W * LL<R>::NSY + 16 * LYShape<T>::W) * sizeof(T);
}

template <typename K>
static cudaError_t l2_allow(K kern)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L2_SMEM_LIMIT);
}

// the O-grid radial line lengths 32 (R - 1) + 1 (65, 129, 257, 513, 1025) run the
// direction-1 passes with the length known at compile time
template <int R>
constexpr int l2_nc() { return (R == 3 || R == 5 || R == 9 || R == 17 || R == 33) ? 32 * (R - 1) + 1 : 0; }

template <typename T, typename M, int R, int NC>
static cudaError_t l2_allow_r()
{
    cudaError_t e;
    if ((e = l2_allow(k_l2_y<T, M, R, 2, NC>)) != cudaSuccess) return e;
    if ((e = l2_allow(k_l2_y<T, M, R, 4, NC>)) != cudaSuccess) return e;
    if ((e = l2_allow(k_l2_fy<T, M, R, NC, 1>)) != cudaSuccess) return e;
    if constexpr (NC == 0)
        if ((e = l2_allow(k_l2_fy<T, M, R, 0, 2>)) != cudaSuccess) return e;
    if ((e = l2_allow(k_l2_fy<T, M, R, NC, 1, true>)) != cudaSuccess) return e;
    return l2_allow(k_l2_y0<T, M, R, NC>);
}

// whether a direction-1 filter pass takes the 32-line blocks: rows of a multiple of 32 nodes
// (a block's lines are then consecutive nodes of one row of one grid) and lines of at most 17
// rows per lane (longer lines: too few blocks, one per SM; the 1025-node radial lines of the
// 1025 x 2048 ellipse measured 47 us against 38 us with 8 lines per block)
template <typename T, int R, typename A>
static bool l2_fy_wide(const A& a)
{
    using S = LFShape<T, 1, true>;
    return R <= 17 && a.fdir == 1 && a.D.n[0] % S::W == 0 &&
           ((size_t)S::W * LL<R>::NS + 16 * S::NW) * sizeof(T) <= L2_SMEM_LIMIT;
}

template <typename T, typename M, int R, int NC>
static void l2_launch_y(const L2Args<T, M>& a, const PartTab<T>& tb, int which, int nf, int nb, size_t sm,
                        cudaStream_t st)
{
    constexpr int W = LYShape<T>::W;
    if (which == L2_Y0) k_l2_y0<T, M, R, NC><<<nb, 32 * W, sm, st>>>(a, tb);
    else if (which == L2_FY) {
        if constexpr (NC == 0)
            if (a.fdir == 2) {
                constexpr int W2 = LFShape<T, 2>::W;
                const size_t sm2 = ((size_t)W2 * LL<R>::NS + 16 * LFShape<T, 2>::NW) * sizeof(T);
                k_l2_fy<T, M, R, 0, 2><<<a.D.nlines(2) / W2, 32 * LFShape<T, 2>::NW, sm2, st>>>(a, tb);
                return;
            }
        if (l2_fy_wide<T, R>(a)) {
            // 32 lines per block, so that every row access is a 128-byte segment (the lines'
            // rows lie a whole x-row apart)
            using S = LFShape<T, 1, true>;
            const size_t sm3 = ((size_t)S::W * LL<R>::NS + 16 * S::NW) * sizeof(T);
            k_l2_fy<T, M, R, NC, 1, true><<<a.kcnt * a.D.n[0] / S::W, 32 * S::NW, sm3, st>>>(a, tb);
            return;
        }
        k_l2_fy<T, M, R, NC, 1><<<nb, 32 * W, sm, st>>>(a, tb);
    }
    else if (nf == 4) k_l2_y<T, M, R, 4, NC><<<nb, 32 * W, sm, st>>>(a, tb);
    else k_l2_y<T, M, R, 2, NC><<<nb, 32 * W, sm, st>>>(a, tb);
}

template <typename T, typename M, int R>
static cudaError_t l2_launch_r(const L2Args<T, M>& a, const PartTab<T>& tb, int which, int nf, cudaStream_t st)
{
    constexpr int NC = l2_nc<R>();
    const size_t sm = l2_smem<T, R>(which, nf);
    if (sm > L2_SMEM_LIMIT) return cudaErrorNotSupported;
    static bool attr = false;
    if (!attr) {
        cudaError_t e;
        if ((e = l2_allow(k_l2_x<T, M, R, 2>)) != cudaSuccess) return e;
        if ((e = l2_allow(k_l2_x<T, M, R, 4>)) != cudaSuccess) return e;
        if ((e = l2_allow(k_l2_fx<T, M, R>)) != cudaSuccess) return e;
        if ((e = l2_allow_r<T, M, R, 0>()) != cudaSuccess) return e;
        if constexpr (NC > 0)
            if ((e = l2_allow_r<T, M, R, NC>()) != cudaSuccess) return e;
        attr = true;
    }
    const Dims& D = a.D;
    if (which == L2_X || which == L2_FX) {
        constexpr int W = LXShape<T>::W;
        const int nb = (a.kcnt * D.n[1] + W - 1) / W;
        if (which == L2_FX) k_l2_fx<T, M, R><<<nb, 32 * W, sm, st>>>(a, tb);
        else if (nf == 4) k_l2_x<T, M, R, 4><<<nb, 32 * W, sm, st>>>(a, tb);
        else k_l2_x<T, M, R, 2><<<nb, 32 * W, sm, st>>>(a, tb);
    } else {
        if (which == L2_FY && a.commit && (a.fdir == 2 ? D.nlines(2) / LFShape<T, 2>::W : D.nlines(1) / LYShape<T>::W) > a.max_partials)
            return cudaErrorNotSupported;
        if (which == L2_FY && a.fdir == 2 && (D.n[0] % LFShape<T, 2>::W != 0 ||
                                              ((size_t)LFShape<T, 2>::W * LL<R>::NS + 16 * LFShape<T, 2>::NW) * sizeof(T) > L2_SMEM_LIMIT))
            return cudaErrorNotSupported;
        const int nb = a.kcnt * D.n[0] / LYShape<T>::W;   // n0 % W == 0
        if constexpr (NC > 0) {
            if (D.n[1] == NC) {
                l2_launch_y<T, M, R, NC>(a, tb, which, nf, nb, sm, st);
                return cudaGetLastError();
            }
        }
        l2_launch_y<T, M, R, 0>(a, tb, which, nf, nb, sm, st);
    }
    return cudaGetLastError();
}

template <typename T, typename M>
cudaError_t l2_launch(const L2Args<T, M>& a, const PartTab<T>& tb, int which, int nf, cudaStream_t st)
{
    if (!tb.ok) return cudaErrorNotSupported;
    switch (tb.R) {
    case 3: return l2_launch_r<T, M, 3>(a, tb, which, nf, st);
    case 4: return l2_launch_r<T, M, 4>(a, tb, which, nf, st);
    case 5: return l2_launch_r<T, M, 5>(a, tb, which, nf, st);
    case 8: return l2_launch_r<T, M, 8>(a, tb, which, nf, st);
    case 9: return l2_launch_r<T, M, 9>(a, tb, which, nf, st);
    case 16: return l2_launch_r<T, M, 16>(a, tb, which, nf, st);
    case 17: return l2_launch_r<T, M, 17>(a, tb, which, nf, st);
    case 32: return l2_launch_r<T, M, 32>(a, tb, which, nf, st);
    case 33: return l2_launch_r<T, M, 33>(a, tb, which, nf, st);
    case 64: return l2_launch_r<T, M, 64>(a, tb, which, nf, st);
    default: return cudaErrorNotSupported;
    }
}

// whether both directions' passes fit: partition tables for both line lengths and the
// shared memory of the widest pass (curvature: four fields)
template <typename T, typename M>
bool l2_supported(const Dims& D, const PartTab<T>& t0, const PartTab<T>& t1, int nf)
{
    if (!t0.ok || !t1.ok) return false;
    // 16-byte vectors along i: the direction-0 lines in vectors, the direction-1 blocks in
    // 32-byte row segments of one stacked grid
    if (D.n[0] % LYShape<T>::W != 0) return false;
    auto fits = [&](int R, int which) -> bool {
        size_t sm = 0;
        switch (R) {
        case 3: sm = l2_smem<T, 3>(which, nf); break;
        case 4: sm = l2_smem<T, 4>(which, nf); break;
        case 5: sm = l2_smem<T, 5>(which, nf); break;
        case 8: sm = l2_smem<T, 8>(which, nf); break;
        case 9: sm = l2_smem<T, 9>(which, nf); break;
        case 16: sm = l2_smem<T, 16>(which, nf); break;
        case 17: sm = l2_smem<T, 17>(which, nf); break;
        case 32: sm = l2_smem<T, 32>(which, nf); break;
        case 33: sm = l2_smem<T, 33>(which, nf); break;
        case 64: sm = l2_smem<T, 64>(which, nf); break;
        default: return false;
        }
        return sm <= L2_SMEM_LIMIT;
    };
    return fits(t0.R, L2_X) && fits(t1.R, L2_Y) && fits(t1.R, L2_Y0);
}

}  // namespace wd
