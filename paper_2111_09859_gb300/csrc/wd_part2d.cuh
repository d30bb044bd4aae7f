// wd_part2d.cuh -- line passes of the fused 2-D pseudo step with the warp partition solve
// (instantiated per precision in wd_part2d_f32.cu and wd_part2d_f64.cu).
//
// A block holds 8 grid lines of one direction in shared memory (staged with coalesced
// loads: whole rows for direction 0, 32-byte segments of 8 neighbouring lines for
// direction 1) and gives each line to one warp.  Lane l owns the R consecutive rows
// lR .. lR+R-1 of its line in registers: it forms their right-hand sides from shared
// memory, eliminates its first R-1 rows locally with precomputed Thomas factors, and the
// warp solves the 32-unknown system of the block-end rows (separators) by five PCR levels
// over shuffles; two FMAs per row then give the solution (tables: wd_linesys.cu).  Per row
// and field this costs about a dozen instructions and no block barrier, where PCR over
// shared memory costs a barrier and a dozen instructions per row, field and level.
//
// The passes compute exactly what the PCR passes of wd_fused2d.cu compute (the same row
// formulas, the same tridiagonal systems, the same epilogues); only the elimination order
// of the tridiagonal solves differs.
#pragma once

#include <algorithm>

#include "wd_api_internal.h"
#include "wd_fused2d.h"
#include "wd_partsolve.cuh"
#include "wd_pcr.cuh"

namespace wd {

// lines per block = warps per block (direction 1 stages 32-byte segments of 8 neighbouring
// lines per row)
// resident blocks per SM asked of the compiler
#define P2_MINB(T, LPB) ((LPB) >= 32 ? 1 : (sizeof(T) == 8 ? 2 : 4))
#define P2_MINB_DIV(T, LPB) ((LPB) >= 32 ? 1 : (sizeof(T) == 8 ? 1 : 3))

// padded line layout in shared memory: row i at i + i / 32 when R is even (so that the 32
// lanes, R rows apart, fall in distinct banks); the line stride is 4 modulo 32, so that the
// 8 lines x 4 rows touched by a warp in the direction-1 staging order hit distinct banks
template <int R>
struct PLayout {
    static constexpr int NP = 32 * R;
    static constexpr int PAD = (R % 2 == 0);
    static constexpr int USED = NP + (PAD ? R : 0);
    static constexpr int LS = (USED + 27) / 32 * 32 + 4;
    __device__ static __forceinline__ int at(int i) { return PAD ? i + (i >> 5) : i; }
};

template <typename T, int R>
struct PView {
    using value_type = T;
    const T* F;
    int N, per;
    __device__ __forceinline__ T at(int j) const
    {
        if (per) j = j < 0 ? j + N : (j >= N ? j - N : j);
        return F[PLayout<R>::at(j)];
    }
    __device__ __forceinline__ T refl(int j) const
    {
        if (per) j = j < 0 ? j + N : (j >= N ? j - N : j);
        else j = j < 0 ? -j : (j >= N ? 2 * (N - 1) - j : j);
        return F[PLayout<R>::at(j)];
    }
};

// visits the nodes (l, i) of the block's lines in an order whose global accesses are
// coalesced; the same thread gets the same nodes in every call
template <int LPB, typename F>
__device__ __forceinline__ void p2_nodes(const Dims& D, int dir, int q0, int nl, F&& fn)
{
    const int N = D.n[dir];
    if (dir == 0) {
        for (int l = 0; l < nl; l++) {
            const long long base = D.line_base(0, q0 + l);
            for (int i = threadIdx.x; i < N; i += 32 * LPB) fn(l, i, base + i);
        }
    } else {
        const int l = threadIdx.x & (LPB - 1);
        if (l >= nl) return;
        const long long st = D.stride(dir);
        const long long base = D.line_base(dir, q0 + l);
        for (int i = threadIdx.x / LPB; i < N; i += 32) fn(l, i, base + (long long)i * st);
    }
}

// ---- A: derivative of phi along one direction (+ LAD fourth difference) -------------------
template <typename T, typename M, int R, int LPB>
__global__ void __launch_bounds__(32 * LPB, P2_MINB(T, LPB)) k_p2_deriv(F2Args<T, M> a, PartTab<T> tb, int dir)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    using Lay = PLayout<R>;
    T* Ph = reinterpret_cast<T*>(smraw);
    T* Dv = Ph + LPB * Lay::LS;
    const Dims& D = a.D;
    const int N = D.n[dir], per = D.per[dir];
    const int q0 = blockIdx.x * LPB, nl = min(LPB, D.nlines(dir) - q0);
    p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) { Ph[l * Lay::LS + Lay::at(i)] = a.src[e]; });
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < nl) {
        const PView<T, R> v{Ph + w * Lay::LS, N, per};
        T x[R];
#pragma unroll
        for (int k = 0; k < R; k++) {
            const int i = lane * R + k;
            x[k] = i < N ? deriv_rhs(v, i, a.scheme) : T(0);
        }
        if (tb.implicit) part_solve<T, R>(x, tb, lane);
#pragma unroll
        for (int k = 0; k < R; k++) {
            const int i = lane * R + k;
            if (i < N) Dv[w * Lay::LS + Lay::at(i)] = x[k];
        }
    }
    __syncthreads();
    T* Dout = dir == 0 ? a.D0 : a.D1;
    const long long tot = D.total;
    if (dir == 1 || !a.lad) {
        p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) {
            Dout[e] = Dv[l * Lay::LS + Lay::at(i)];
            if (a.lad) {
                const PView<T, R> v{Ph + l * Lay::LS, N, per};
                a.L1[e] = T(__ldg(a.lads + (long long)tot + e) * M(d4_row(v, i)));
            }
        });
        return;
    }
    // direction 0 after direction 1: C|s_0 d4_0 + s_1 d4_1| along the block's lines, then its
    // Gaussian along direction 0 (the first half of the separable smoothing of Eq. 7)
    T* Gb = Dv + LPB * Lay::LS;
    p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) {
        Dout[e] = Dv[l * Lay::LS + Lay::at(i)];
        const PView<T, R> v{Ph + l * Lay::LS, N, per};
        const T v0 = T(__ldg(a.lads + e) * M(d4_row(v, i))) + a.L1[e];
        Gb[l * Lay::LS + Lay::at(i)] = T(a.C_lad) * (v0 < T(0) ? -v0 : v0);
    });
    __syncthreads();
    p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) {
        a.G0[e] = gauss_rhs(PView<T, R>{Gb + l * Lay::LS, N, per}, i);
    });
}

// ---- B: metric-weighted divergence parts along one direction ------------------------------
template <typename T, typename M, int NF, int R, int LPB>
__device__ __forceinline__ void p2_div_body(const F2Args<T, M>& a, const PartTab<T>& tb, int dir, int bid,
                                            unsigned char* smraw)
{
    using Lay = PLayout<R>;
    constexpr int BUF = LPB * Lay::LS;
    T* U = reinterpret_cast<T*>(smraw);
    const Dims& D = a.D;
    const int N = D.n[dir], per = D.per[dir];
    const int q0 = bid * LPB, nl = min(LPB, D.nlines(dir) - q0);
    const long long tot = D.total;
    p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) {
        const int s = l * Lay::LS + Lay::at(i);
        const M d0 = M(a.D0[e]), d1 = M(a.D1[e]);
        const M ux = __ldg(a.xi + 0 * tot + e) * d0 + __ldg(a.xi + 3 * tot + e) * d1;   // xi_x D0 + eta_x D1
        const M uy = __ldg(a.xi + 1 * tot + e) * d0 + __ldg(a.xi + 4 * tot + e) * d1;   // xi_y D0 + eta_y D1
        U[s] = T(ux);
        U[BUF + s] = T(uy);
        if (NF == 4) {
            const M ig = M(1) / (sqrt(ux * ux + uy * uy) + M(a.eps0));
            U[2 * BUF + s] = T(ux * ig);
            U[3 * BUF + s] = T(uy * ig);
        }
    });
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // fields solved together (one load of each table value for the group); one at a time
    // keeps the registers low enough for two resident blocks
    constexpr int GF = 1;
    if (w < nl) {
#pragma unroll 1
        for (int f0 = 0; f0 < NF; f0 += GF) {
            T x[GF][R];
#pragma unroll
            for (int f = 0; f < GF; f++) {
                const PView<T, R> v{U + (f0 + f) * BUF + w * Lay::LS, N, per};
#pragma unroll
                for (int k = 0; k < R; k++) {
                    const int i = lane * R + k;
                    x[f][k] = i < N ? deriv_rhs(v, i, a.scheme) : T(0);
                }
            }
            if (tb.implicit) part_solve<T, R, GF>(x, tb, lane);
            __syncwarp();
#pragma unroll
            for (int f = 0; f < GF; f++) {
                T* F = U + (f0 + f) * BUF + w * Lay::LS;
#pragma unroll
                for (int k = 0; k < R; k++) {
                    const int i = lane * R + k;
                    if (i < N) F[Lay::at(i)] = x[f][k];
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    T* lap = dir == 0 ? a.LAP0 : a.LAP1;
    T* kap = dir == 0 ? a.KAP0 : a.KAP1;
    p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) {
        const int s = l * Lay::LS + Lay::at(i);
        const M x0 = __ldg(a.xi + (long long)(dir * 3 + 0) * tot + e);
        const M x1 = __ldg(a.xi + (long long)(dir * 3 + 1) * tot + e);
        lap[e] = T(x0 * M(U[s]) + x1 * M(U[BUF + s]));
        if (NF == 4) kap[e] = T(x0 * M(U[2 * BUF + s]) + x1 * M(U[3 * BUF + s]));
    });
}

template <typename T, typename M, int NF, int R, int LPB>
__global__ void __launch_bounds__(32 * LPB, P2_MINB_DIV(T, LPB)) k_p2_div(F2Args<T, M> a, PartTab<T> tb, int dir)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    p2_div_body<T, M, NF, R, LPB>(a, tb, dir, blockIdx.x, smraw);
}

// both directions' divergence passes in one launch (blocks [0, nb0) direction 0, the rest
// direction 1), so that the two passes fill each other's partial last waves
template <typename T, typename M, int NF, int R0, int R1>
__global__ void __launch_bounds__(256, P2_MINB_DIV(T, 8)) k_p2_div2(F2Args<T, M> a, PartTab<T> t0, PartTab<T> t1, int nb0)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    if ((int)blockIdx.x < nb0) p2_div_body<T, M, NF, R0, 8>(a, t0, 0, blockIdx.x, smraw);
    else p2_div_body<T, M, NF, R1, 8>(a, t1, 1, blockIdx.x - nb0, smraw);
}

// ---- F: filter along one direction; direction 1 with commit = 1 also applies the line
// boundary conditions, reduces the change norms (Eq. 20) and commits the new state ------
template <typename T, typename M, int R, int LPB>
__global__ void __launch_bounds__(32 * LPB, P2_MINB(T, LPB)) k_p2_filter(F2Args<T, M> a, PartTab<T> tb, int dir, int commit)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ T cf[6][6];
    __shared__ double s_ss[LPB], s_mx[LPB];
    using Lay = PLayout<R>;
    T* A = reinterpret_cast<T*>(smraw);
    T* O = A + LPB * Lay::LS;                                   // commit: old state
    uint8_t* MK = reinterpret_cast<uint8_t*>(O + LPB * Lay::LS);   // commit: Dirichlet flags
    const Dims& D = a.D;
    const int N = D.n[dir], per = D.per[dir];
    const int q0 = blockIdx.x * LPB, nl = min(LPB, D.nlines(dir) - q0);
    const int tid = threadIdx.x;
    for (int i = tid; i < 36; i += 32 * LPB) {
        const int hw = i / 6, mm = i % 6;
        double v = 0.0;
        if (hw >= 1 && mm >= 1 && mm <= hw) v = 0.5 * a.fa[hw][mm] - (mm == 1 ? a.alpha_f : 0.0);
        cf[hw][mm] = T(v);
    }
    // every global load of the pass happens here (the commit epilogue then only stores).  Off
    // direction 0 a thread's nodes (at most R: rows tid / LPB + 32 k of one line) are loaded
    // into registers first, so that their loads are in flight together, then stored
    if (dir != 0) {
        const int l = tid & (LPB - 1), i0 = tid / LPB;
        if (l < nl) {
            const long long st = D.stride(dir), base = D.line_base(dir, q0 + l);
            T v[R], o[R];
            uint8_t m[R];
#pragma unroll
            for (int k = 0; k < R; k++) {
                const int i = i0 + 32 * k;
                if (i < N) {
                    const long long e = base + (long long)i * st;
                    v[k] = a.src[e];
                    if (commit) {
                        o[k] = a.phin[e];
                        m[k] = a.mask[e];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < R; k++) {
                const int i = i0 + 32 * k;
                if (i < N) {
                    const int s = l * Lay::LS + Lay::at(i);
                    A[s] = v[k];
                    if (commit) {
                        O[s] = o[k];
                        MK[s] = m[k];
                    }
                }
            }
        }
    } else if (commit)
        p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) {
            const int s = l * Lay::LS + Lay::at(i);
            A[s] = a.src[e];
            O[s] = a.phin[e];
            MK[s] = a.mask[e];
        });
    else
        p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) { A[l * Lay::LS + Lay::at(i)] = a.src[e]; });
    __syncthreads();
    const int w = tid >> 5, lane = tid & 31;
    if (a.filter && w < nl) {
        T* F = A + w * Lay::LS;
        const PView<T, R> v{F, N, per};
        T x[R];
#pragma unroll
        for (int k = 0; k < R; k++) {
            const int i = lane * R + k;
            x[k] = i < N ? filter_rhs(v, i, cf) : T(0);
        }
        if (tb.implicit) part_solve<T, R>(x, tb, lane);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < R; k++) {
            const int i = lane * R + k;
            if (i < N) F[Lay::at(i)] += x[k];   // delta form: f + (fh - f)
        }
    }
    __syncthreads();
    if (!commit) {
        p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) { a.dst[e] = A[l * Lay::LS + Lay::at(i)]; });
        return;
    }
    // Epilogue: far-field / Neumann end nodes from the filtered values of their line (before
    // the Dirichlet reset), Dirichlet nodes, commit, change norms.  A thread sums its own
    // nodes' squared changes (at most R of them) in the state precision; the sums across
    // threads and blocks are taken in double.
    T ss_t = T(0), mx_t = T(0);
    p2_nodes<LPB>(D, dir, q0, nl, [&](int l, int i, long long e) {
        const T* F = A + l * Lay::LS;
        T nv = F[Lay::at(i)];
        if ((i == 0 || i == N - 1) && D.ndim == 2) {
            const int side = i == N - 1;
            int kind = side ? a.bchi1 : a.bclo1;
            if (kind == WD_BC_FARFIELD || kind == WD_BC_NEUMANN) {
                if (a.poisson) kind = WD_BC_NEUMANN;
                const T v1 = F[Lay::at(side ? N - 2 : 1)], v2 = F[Lay::at(side ? N - 3 : 2)];
                if (kind == WD_BC_NEUMANN) nv = v1;
                else {
                    const int qline = q0 + l;
                    const int line = (qline / D.n[0]) + D.n[2] * (qline % D.n[0]);   // face ratio index
                    nv = v1 + T((side ? a.ffr_hi : a.ffr_lo)[line]) * (v1 - v2);
                }
            }
        }
        const int s = l * Lay::LS + Lay::at(i);
        const bool dir_node = MK[s] != 0;
        if (dir_node) nv = a.poisson ? T(0) : __ldg(a.dval + e);
        const T ov = O[s];
        a.phin_w[e] = nv;
        if (dir_node) return;
        const T d = nv - ov;
        ss_t += d * d;
        mx_t = fmax(mx_t, fabs(d));
    });
    double ss = double(ss_t), mx = double(mx_t);
    // block reduction, then the last block reduces the block partials in a fixed order
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
        double t = 0.0, mm = 0.0;
        for (int k = 0; k < LPB; k++) {
            t += s_ss[k];
            mm = fmax(mm, s_mx[k]);
        }
        a.partial[2 * blockIdx.x] = t;
        a.partial[2 * blockIdx.x + 1] = mm;
    }
}

// Per-grid change norms from the block partials of the commit pass, in a fixed order: the
// blocks of stacked grid k are the contiguous range [k * bpm, (k + 1) * bpm); a group of
// tpm threads (a power of two, >= 32) reduces one grid at a time.
static __global__ void __launch_bounds__(1024) k_p2_reduce(const double* __restrict__ partial, int nblocks,
                                                    int batch, double* result)
{
    __shared__ double s_ss[32], s_mx[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int tpm = 1024;
    while (tpm > 32 && tpm * batch > 1024) tpm >>= 1;
    const int ngroups = 1024 / tpm, grp = tid / tpm, gt = tid % tpm, wpg = tpm / 32;
    const int bpm = nblocks / batch;
    const int rounds = (batch + ngroups - 1) / ngroups;
    for (int r = 0; r < rounds; r++) {
        const int k = r * ngroups + grp;
        double t = 0.0, mm = 0.0;
        if (k < batch)
            for (int b = k * bpm + gt; b < (k + 1) * bpm; b += tpm) {
                t += partial[2 * b];
                mm = fmax(mm, partial[2 * b + 1]);
            }
        for (int o = 16; o > 0; o >>= 1) {
            t += __shfl_down_sync(0xffffffffu, t, o);
            mm = fmax(mm, __shfl_down_sync(0xffffffffu, mm, o));
        }
        if (lane == 0) {
            s_ss[w] = t;
            s_mx[w] = mm;
        }
        __syncthreads();
        if (gt == 0 && k < batch) {
            double u = 0.0, v = 0.0;
            for (int q = 0; q < wpg; q++) {
                u += s_ss[grp * wpg + q];
                v = fmax(v, s_mx[grp * wpg + q]);
            }
            result[2 * k] = u;
            result[2 * k + 1] = v;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// launcher
// ------------------------------------------------------------------------------------

static const size_t P2_SMEM_LIMIT = 200 * 1024;

template <typename K>
static void p2_allow(K kern)
{
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P2_SMEM_LIMIT);
}

static size_t p2_ls(int R)
{
    const int used = 32 * R + (R % 2 == 0 ? R : 0);
    return (size_t)((used + 27) / 32 * 32 + 4);
}

// shared-memory buffers (lines x LS) of each pass
static int p2_bufs(int which, int dir, bool curv, bool lad)
{
    if (which == F2_DERIV) return 2 + (dir == 0 && lad ? 1 : 0);
    if (which == F2_DIV) return curv ? 4 : 2;
    if (which == F2_FILTER) return 3;   // field, old state, Dirichlet flags (rounded up)
    return 1;
}

template <typename T, typename M, int R, int LPB>
static cudaError_t p2_launch_rl(const F2Args<T, M>& a, const PartTab<T>& tb, int which, int dir,
                                cudaStream_t st)
{
    const Dims& D = a.D;
    const int nb = (D.nlines(dir) + LPB - 1) / LPB;
    const bool curv = a.curvature && !a.poisson;
    const size_t sm = (size_t)p2_bufs(which, dir, curv, a.lad) * LPB * PLayout<R>::LS * sizeof(T);
    if (sm > P2_SMEM_LIMIT) return cudaErrorNotSupported;
    if (which == F2_DERIV) {
        static bool attr = false;
        if (!attr) p2_allow(k_p2_deriv<T, M, R, LPB>), attr = true;
        k_p2_deriv<T, M, R, LPB><<<nb, 32 * LPB, sm, st>>>(a, tb, dir);
    } else if (which == F2_DIV) {
        static bool attr = false;
        if (!attr) p2_allow(k_p2_div<T, M, 2, R, LPB>), p2_allow(k_p2_div<T, M, 4, R, LPB>), attr = true;
        if (curv) k_p2_div<T, M, 4, R, LPB><<<nb, 32 * LPB, sm, st>>>(a, tb, dir);
        else k_p2_div<T, M, 2, R, LPB><<<nb, 32 * LPB, sm, st>>>(a, tb, dir);
    } else {
        static bool attr = false;
        if (!attr) p2_allow(k_p2_filter<T, M, R, LPB>), attr = true;
        const int commit = which == F2_FILTER;
        if (commit && (nb > a.max_partials || (D.ndim == 2 && (dir != 1 || D.n[0] % LPB))))
            return cudaErrorNotSupported;
        k_p2_filter<T, M, R, LPB><<<nb, 32 * LPB, sm, st>>>(a, tb, dir, commit);
        if (commit) {
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            k_p2_reduce<<<1, 1024, 0, st>>>(a.partial, nb, a.batch, a.result);
        }
    }
    return cudaGetLastError();
}

template <typename T, typename M, int R, int LPB>
static cudaError_t p2_launch_rl_filter(const F2Args<T, M>& a, const PartTab<T>& tb, int which, int dir,
                                       cudaStream_t st)
{
    const Dims& D = a.D;
    const int nb = (D.nlines(dir) + LPB - 1) / LPB;
    const int commit = which == F2_FILTER;
    const size_t sm = (size_t)(commit ? 3 : 1) * LPB * PLayout<R>::LS * sizeof(T);
    if (sm > P2_SMEM_LIMIT) return cudaErrorNotSupported;
    static bool attr = false;
    if (!attr) p2_allow(k_p2_filter<T, M, R, LPB>), attr = true;
    if (commit && (nb > a.max_partials || D.ndim == 2)) return cudaErrorNotSupported;
    k_p2_filter<T, M, R, LPB><<<nb, 32 * LPB, sm, st>>>(a, tb, dir, commit);
    if (commit) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_p2_reduce<<<1, 1024, 0, st>>>(a.partial, nb, a.batch, a.result);
    }
    return cudaGetLastError();
}

// lines per block of a pass: 8 (whole rows for direction 0, 32-byte row segments of 8
// neighbouring lines otherwise); the direction-2 filter of 3-D grids, whose rows lie a
// whole plane apart, takes 32 lines for full 128-byte segments
static int p2_lpb(int which, int dir, int R)
{
    if (R > 33) return 4;   // 2048-node lines: the shared-memory budget allows 4 per block
    return (dir == 2 && (which == F2_FILTER || which == P2_FILTER0)) ? 32 : 8;
}

template <typename T, typename M, int R>
static cudaError_t p2_launch_r(const F2Args<T, M>& a, const PartTab<T>& tb, int which, int dir,
                               cudaStream_t st)
{
    if constexpr (R > 33) {
        return p2_launch_rl<T, M, R, 4>(a, tb, which, dir, st);
    } else {
        if (p2_lpb(which, dir, R) == 32) {
            if (which == F2_DERIV || which == F2_DIV) return cudaErrorNotSupported;
            return p2_launch_rl_filter<T, M, R, 32>(a, tb, which, dir, st);
        }
        return p2_launch_rl<T, M, R, 8>(a, tb, which, dir, st);
    }
}

template <typename T, typename M>
cudaError_t p2_launch(const F2Args<T, M>& a, const PartTab<T>& tb, int which, int dir, cudaStream_t st)
{
    if (!tb.ok) return cudaErrorNotSupported;
    switch (tb.R) {
    case 3: return p2_launch_r<T, M, 3>(a, tb, which, dir, st);
    case 4: return p2_launch_r<T, M, 4>(a, tb, which, dir, st);
    case 5: return p2_launch_r<T, M, 5>(a, tb, which, dir, st);
    case 8: return p2_launch_r<T, M, 8>(a, tb, which, dir, st);
    case 9: return p2_launch_r<T, M, 9>(a, tb, which, dir, st);
    case 16: return p2_launch_r<T, M, 16>(a, tb, which, dir, st);
    case 17: return p2_launch_r<T, M, 17>(a, tb, which, dir, st);
    case 32: return p2_launch_r<T, M, 32>(a, tb, which, dir, st);
    case 33: return p2_launch_r<T, M, 33>(a, tb, which, dir, st);
    case 64: return p2_launch_r<T, M, 64>(a, tb, which, dir, st);
    default: return cudaErrorNotSupported;
    }
}

template <typename T, typename M, int R0, int R1>
static cudaError_t p2_div2_rr(const F2Args<T, M>& a, const PartTab<T>& t0, const PartTab<T>& t1, cudaStream_t st)
{
    const Dims& D = a.D;
    const bool curv = a.curvature && !a.poisson;
    const int nf = curv ? 4 : 2;
    const int nb0 = (D.nlines(0) + 7) / 8, nb1 = (D.nlines(1) + 7) / 8;
    const size_t sm0 = (size_t)nf * 8 * PLayout<R0>::LS * sizeof(T), sm1 = (size_t)nf * 8 * PLayout<R1>::LS * sizeof(T);
    const size_t sm = sm0 > sm1 ? sm0 : sm1;
    if (sm > P2_SMEM_LIMIT) return cudaErrorNotSupported;
    static bool attr = false;
    if (!attr) p2_allow(k_p2_div2<T, M, 2, R0, R1>), p2_allow(k_p2_div2<T, M, 4, R0, R1>), attr = true;
    if (curv) k_p2_div2<T, M, 4, R0, R1><<<nb0 + nb1, 256, sm, st>>>(a, t0, t1, nb0);
    else k_p2_div2<T, M, 2, R0, R1><<<nb0 + nb1, 256, sm, st>>>(a, t0, t1, nb0);
    return cudaGetLastError();
}

// both divergence passes in one launch for the line-length pairs of the O-grid sizes
// (periodic 128 .. 1024 around, 65 .. 513 radial); cudaErrorNotSupported otherwise
template <typename T, typename M>
cudaError_t p2_div2(const F2Args<T, M>& a, const PartTab<T>& t0, const PartTab<T>& t1, cudaStream_t st)
{
    if (!t0.ok || !t1.ok) return cudaErrorNotSupported;
    if (t0.R == 16 && t1.R == 9) return p2_div2_rr<T, M, 16, 9>(a, t0, t1, st);
    if (t0.R == 4 && t1.R == 3) return p2_div2_rr<T, M, 4, 3>(a, t0, t1, st);
    if (t0.R == 8 && t1.R == 5) return p2_div2_rr<T, M, 8, 5>(a, t0, t1, st);
    if (t0.R == 32 && t1.R == 17) return p2_div2_rr<T, M, 32, 17>(a, t0, t1, st);
    return cudaErrorNotSupported;
}

// whether the pass `which` (F2_DERIV, F2_DIV, P2_FILTER0 or F2_FILTER) fits direction dir
template <typename T, typename M>
bool p2_supported(const F2Args<T, M>& a, const PartTab<T>& tb, int which, int dir)
{
    if (!tb.ok) return false;
    const int lpb = p2_lpb(which, dir, tb.R);
    const int bufs = which == F2_DIV ? 4 : (which == F2_DERIV ? 3 : p2_bufs(which, dir, false, false));
    if ((size_t)bufs * lpb * p2_ls(tb.R) * sizeof(T) > P2_SMEM_LIMIT) return false;
    if (which == F2_FILTER) {
        const int nb = (a.D.nlines(dir) + lpb - 1) / lpb;
        if (nb > a.max_partials || (a.D.ndim == 2 && (dir != 1 || a.D.n[0] % lpb))) return false;
    }
    return true;
}

}  // namespace wd
