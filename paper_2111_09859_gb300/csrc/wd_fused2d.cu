// wd_fused2d.cu -- fused pseudo step for 2-D grids whose non-wall, non-periodic faces lie
// only at the ends of direction 1 (O-grids around bodies, channels, plates).
//
// One RK4 stage (Sec. 3.3) = three launches:
//   A  both directions' first derivatives of phi (Eq. 16; compact rows solved by PCR) and,
//      for LAD, both directions' s_l d4_l(phi) terms of Eq. 7;
//   B  both directions' metric-weighted divergences of U = grad(phi) (and of the unit normal
//      for the curvature correction, Eq. 25), i.e. the Laplacian of Eq. 9 split by
//      direction; the same launch smooths C|LAD| along direction 0;
//   C  direction-1 lines: Gaussian smoothing along direction 1, HJ (or Poisson) right-hand
//      side, local time step, RK4 stage update, then the boundary conditions of the line
//      (far-field / Neumann ends, Dirichlet nodes) in shared memory.
// After the fourth stage: the direction-0 filter (generic line pass) and one direction-1
// launch that filters, applies the boundary conditions, reduces the change norms (Eq. 20)
// and commits the new state.  The sequence of operations and every formula are those of
// the generic path in wd_api.cu / wd_kernels.cu; only the kernel boundaries differ.
#include <algorithm>

#include "wd_api_internal.h"
#include "wd_fused2d.h"
#include "wd_pcr.cuh"

namespace wd {

template <typename T, typename M>
__device__ __forceinline__ void grad_at(const F2Args<T, M>& a, long long node, M& ux, M& uy)
{
    const long long tot = a.D.total;
    const M d0 = M(__ldg(a.D0 + node)), d1 = M(__ldg(a.D1 + node));
    ux = __ldg(a.xi + 0 * tot + node) * d0 + __ldg(a.xi + 3 * tot + node) * d1;   // xi_x D0 + eta_x D1
    uy = __ldg(a.xi + 1 * tot + node) * d0 + __ldg(a.xi + 4 * tot + node) * d1;   // xi_y D0 + eta_y D1
}

// ---- A: derivatives of phi along both directions (+ LAD fourth differences) ---------------
template <typename T, typename M, int R>
__global__ void __launch_bounds__(512) k_f2_deriv(F2Args<T, M> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int dir = blockIdx.x < a.nb[0] ? 0 : 1;
    const int bidx = dir == 0 ? blockIdx.x : blockIdx.x - a.nb[0];
    const Dims& D = a.D;
    const LineMap mp = make_map(D, dir, a.lpb[dir], D.nlines(dir), bidx * a.lpb[dir]);
    const int S = mp.size(), per = D.per[dir];
    T* A = reinterpret_cast<T*>(smraw);
    T* B = A + S;
    Slot q[R];
    slots_init<R>(q, mp, D);
#pragma unroll
    for (int r = 0; r < R; r++)
        if (q[r].s >= 0) A[q[r].s] = a.src[q[r].node];
    __syncthreads();
    T* Lout = dir == 0 ? a.L0 : a.L1;
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (q[r].s < 0) continue;
        const LineView<T> v = view_of<T>(A, q[r], mp, per);
        B[q[r].s] = deriv_rhs(v, q[r].i, a.scheme);
        if (a.lad) Lout[q[r].node] = T(a.lads[(long long)dir * D.total + q[r].node] * M(d4_row(v, q[r].i)));
    }
    __syncthreads();
    T* X = B;
    const LineTab<T>& tb = dir == 0 ? a.dtab0 : a.dtab1;
    if (tb.implicit) X = pcr_solve<T, 1, R>(B, A, mp, tb, q);
    T* Dout = dir == 0 ? a.D0 : a.D1;
#pragma unroll
    for (int r = 0; r < R; r++)
        if (q[r].s >= 0) Dout[q[r].node] = X[q[r].s];
}

// ---- B: divergence passes along both directions (+ Gaussian along direction 0) ----------
template <typename T, typename M, int NF, int R>
__device__ void f2_div_line(const F2Args<T, M>& a, int dir, int bidx, T* A, T* B)
{
    const Dims& D = a.D;
    const LineMap mp = make_map(D, dir, a.lpb[dir], D.nlines(dir), bidx * a.lpb[dir]);
    const int S = mp.size(), per = D.per[dir];
    Slot q[R];
    slots_init<R>(q, mp, D);
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int s = q[r].s;
        if (s < 0) continue;
        M ux, uy;
        grad_at(a, q[r].node, ux, uy);
        A[s] = T(ux);
        A[S + s] = T(uy);
        if (NF == 4) {
            const M g = sqrt(ux * ux + uy * uy) + M(a.eps0);
            A[2 * S + s] = T(ux / g);
            A[3 * S + s] = T(uy / g);
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (q[r].s < 0) continue;
#pragma unroll
        for (int f = 0; f < NF; f++)
            B[(size_t)f * S + q[r].s] = deriv_rhs(view_of<T>(A + (size_t)f * S, q[r], mp, per), q[r].i, a.scheme);
    }
    __syncthreads();
    T* X = B;
    const LineTab<T>& tb = dir == 0 ? a.dtab0 : a.dtab1;
    if (tb.implicit) X = pcr_solve<T, NF, R>(B, A, mp, tb, q);
    T* lap = dir == 0 ? a.LAP0 : a.LAP1;
    T* kap = dir == 0 ? a.KAP0 : a.KAP1;
    const long long tot = D.total;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int s = q[r].s;
        if (s < 0) continue;
        const long long node = q[r].node;
        const M x0 = a.xi[(long long)(dir * 3 + 0) * tot + node];
        const M x1 = a.xi[(long long)(dir * 3 + 1) * tot + node];
        lap[node] = T(x0 * M(X[s]) + x1 * M(X[S + s]));
        if (NF == 4) kap[node] = T(x0 * M(X[2 * S + s]) + x1 * M(X[3 * S + s]));
    }
}

template <typename T, typename M, int R>
__device__ void f2_gauss0(const F2Args<T, M>& a, int bidx, T* A)
{
    const Dims& D = a.D;
    const LineMap mp = make_map(D, 0, a.lpb[0], D.nlines(0), bidx * a.lpb[0]);
    const int per = D.per[0];
    Slot q[R];
    slots_init<R>(q, mp, D);
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (q[r].s < 0) continue;
        const T v = a.L0[q[r].node] + a.L1[q[r].node];
        A[q[r].s] = T(a.C_lad) * (v < T(0) ? -v : v);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; r++)
        if (q[r].s >= 0) a.G0[q[r].node] = gauss_rhs(view_of<T>(A, q[r], mp, per), q[r].i);
}

template <typename T, typename M, int NF, int R>
__global__ void __launch_bounds__(512) k_f2_div(F2Args<T, M> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T* A = reinterpret_cast<T*>(smraw);
    int b = blockIdx.x;
    if (b < a.nb[0]) {
        f2_div_line<T, M, NF, R>(a, 0, b, A, A + (size_t)NF * a.lpb[0] * a.D.n[0]);
        return;
    }
    b -= a.nb[0];
    if (b < a.nb[1]) {
        f2_div_line<T, M, NF, R>(a, 1, b, A, A + (size_t)NF * a.lpb[1] * a.D.n[1]);
        return;
    }
    f2_gauss0<T, M, R>(a, b - a.nb[1], A);
}

// boundary conditions of the direction-1 lines held in shared memory: far-field / Neumann
// ends, then Dirichlet nodes (poisson: value 0, faces Neumann)
template <typename T, typename M, int R>
__device__ void f2_line_bc(const F2Args<T, M>& a, const LineMap& mp, const Slot (&q)[R], T* V)
{
    const int N = mp.N;
    for (int l = threadIdx.x; l < mp.nl; l += blockDim.x) {
        // line q = i + n0 k of direction 1; the face spacing ratios are stored at k + n2 i
        const int qline = mp.q0 + l;
        const int line = (qline / a.D.n[0]) + a.D.n[2] * (qline % a.D.n[0]);
        for (int side = 0; side < 2; side++) {
            int kind = side ? a.bchi1 : a.bclo1;
            if (kind != WD_BC_FARFIELD && kind != WD_BC_NEUMANN) continue;
            if (a.poisson) kind = WD_BC_NEUMANN;
            const int b = side ? N - 1 : 0, s1 = side ? N - 2 : 1, s2 = side ? N - 3 : 2;
            const T v1 = V[mp.slot(l, s1)], v2 = V[mp.slot(l, s2)];
            if (kind == WD_BC_NEUMANN) V[mp.slot(l, b)] = v1;
            else V[mp.slot(l, b)] = v1 + T((side ? a.ffr_hi : a.ffr_lo)[line]) * (v1 - v2);
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; r++)
        if (q[r].s >= 0 && a.mask[q[r].node]) V[q[r].s] = a.poisson ? T(0) : a.dval[q[r].node];
    __syncthreads();
}

// ---- C: Gaussian along direction 1, right-hand side, RK4 stage, BCs (pointwise) ----------
// Node (i, j) of stacked grid k.  The Gaussian along direction 1 reads the nine G0 values of
// its column directly (even reflection at non-periodic ends); a far-field / Neumann node
// recomputes the stage values of its two inner neighbours (the same code, the same inputs
// as their own threads, which write them too) to extrapolate, so no barrier is needed.
template <typename T, typename M, bool POIS, bool LAD, bool CURV>
__device__ __forceinline__ T f2_stage_value(const F2Args<T, M>& a, long long e, int j, bool own)
{
    const Dims& D = a.D;
    const int N1 = D.n[1];
    const long long st = D.stride(1);
    T Rv, dtv, gam = T(0), v = T(0), gm = T(0);
    const T lap = __ldg(a.LAP0 + e) + __ldg(a.LAP1 + e);
    if (POIS) {
        Rv = T(1) + lap;                                                     // Eq. 19
    } else {
        M ux, uy;
        grad_at(a, e, ux, uy);
        const T tx = T(ux), ty = T(uy);
        const T g2 = tx * tx + ty * ty;
        gm = sqrt(g2);
        const T ph = __ldg(a.src + e);   // the stage input is never the stage output
        const T php = ph > T(0) ? ph : T(0);
        if (!LAD && a.equation == WD_HJ_STD) gam = T(a.eps) * php;           // Eq. 6
        else if (LAD) {                                                      // Eq. 7
            // truncated Gaussian (Kawai & Lele) along direction 1 of C|LAD| smoothed along 0
            const T w[5] = {T(3565.0 / 10368.0), T(3091.0 / 12960.0), T(1997.0 / 25920.0),
                            T(149.0 / 12960.0), T(107.0 / 103680.0)};
            const long long e0 = e - (long long)j * st;
            T gl = w[0] * __ldg(a.G0 + e);
#pragma unroll
            for (int m = 1; m <= 4; m++) {
                int jp = j + m, jm = j - m;
                if (D.per[1]) {
                    jp = jp >= N1 ? jp - N1 : jp;
                    jm = jm < 0 ? jm + N1 : jm;
                } else {
                    jp = jp > N1 - 1 ? 2 * (N1 - 1) - jp : jp;
                    jm = jm < 0 ? -jm : jm;
                }
                gl += w[m] * (__ldg(a.G0 + e0 + (long long)jp * st) + __ldg(a.G0 + e0 + (long long)jm * st));
            }
            const T g1 = T(a.eps) * php;
            gam = g1 < gl ? g1 : gl;
        }
        if (CURV) {                                                          // Eq. 25
            v = T(0.001) * (T(1) - gm) * (T(1) - gm);
            T corr = gm * (__ldg(a.KAP0 + e) + __ldg(a.KAP1 + e));
            corr = corr > T(0) ? corr : T(0);
            Rv = T(1) + (gam + v) * (lap - corr) - g2;
        } else {
            Rv = T(1) + gam * lap - g2;                                      // Eqs. 5, 18
        }
    }
    if (a.stage == 0) {
        if (POIS) dtv = T(a.cfl) / T(__ldg(a.sig2 + e));
        else {
            const T am = gm > T(1) ? gm : T(1);
            dtv = T(a.cfl) / (T(__ldg(a.sig1 + e)) * am + (gam + v) * T(__ldg(a.sig2 + e)));
        }
        if (own) a.dtv[e] = dtv;
    } else {
        dtv = a.dtv[e];
    }
    const T n = __ldg(a.phin + e);
    T out;
    if (a.stage == 0) {
        if (own) a.acc[e] = Rv * T(1.0 / 6.0);
        out = n + T(0.5) * dtv * Rv;
    } else if (a.stage == 1) {
        if (own) a.acc[e] += Rv * T(1.0 / 3.0);
        out = n + T(0.5) * dtv * Rv;
    } else if (a.stage == 2) {
        if (own) a.acc[e] += Rv * T(1.0 / 3.0);
        out = n + dtv * Rv;
    } else {
        out = n + dtv * (a.acc[e] + Rv * T(1.0 / 6.0));
    }
    return out;
}

template <typename T, typename M, bool POIS, bool LAD, bool CURV>
__global__ void __launch_bounds__(512) k_f2_stage(F2Args<T, M> a)
{
    // one thread per node: i from the x-blocks, j = blockIdx.y, the stacked grid = blockIdx.z
    const Dims& D = a.D;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.n[0]) return;
    const int N1 = D.n[1];
    const int j = blockIdx.y;
    const long long st = D.stride(1);
    const long long e = D.idx(i, j, blockIdx.z);
    T out = f2_stage_value<T, M, POIS, LAD, CURV>(a, e, j, true);
    const int side = j == 0 ? 0 : (j == N1 - 1 ? 1 : -1);
    if (side >= 0) {
        int kind = side ? a.bchi1 : a.bclo1;
        if (kind == WD_BC_FARFIELD || kind == WD_BC_NEUMANN) {
            if (POIS) kind = WD_BC_NEUMANN;
            const long long s = side ? -st : st;
            const T v1 = f2_stage_value<T, M, POIS, LAD, CURV>(a, e + s, j + (side ? -1 : 1), false);
            if (kind == WD_BC_NEUMANN) out = v1;
            else {
                const T v2 = f2_stage_value<T, M, POIS, LAD, CURV>(a, e + 2 * s, j + (side ? -2 : 2), false);
                const long long q = blockIdx.z;   // stacked grid
                out = v1 + T((side ? a.ffr_hi : a.ffr_lo)[q + (long long)D.n[2] * i]) * (v1 - v2);
            }
        }
    }
    if (a.mask[e]) out = POIS ? T(0) : a.dval[e];
    a.dst[e] = out;
}

// ---- F: direction-1 filter, line BCs, change norms and commit ----------------------------
template <typename T, typename M, int R>
__global__ void __launch_bounds__(512) k_f2_filter_commit(F2Args<T, M> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ T cf[6][6];
    __shared__ double s_ss[32], s_mx[32];
    __shared__ int s_last;
    const Dims& D = a.D;
    const LineMap mp = make_map(D, 1, a.lpb[1], D.nlines(1), blockIdx.x * a.lpb[1]);
    const int S = mp.size(), per = D.per[1];
    T* A = reinterpret_cast<T*>(smraw);
    T* B = A + S;
    T* Cb = B + S;
    const int tid = threadIdx.x, nth = blockDim.x;
    Slot q[R];
    slots_init<R>(q, mp, D);
    for (int i = tid; i < 36; i += nth) {
        const int hw = i / 6, m = i % 6;
        double v = 0.0;
        if (hw >= 1 && m >= 1 && m <= hw) v = 0.5 * a.fa[hw][m] - (m == 1 ? a.alpha_f : 0.0);
        cf[hw][m] = T(v);
    }
    T ov[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        ov[r] = T(0);
        if (q[r].s < 0) continue;
        A[q[r].s] = a.src[q[r].node];
        ov[r] = a.phin[q[r].node];
    }
    __syncthreads();
    T* V = A;
    if (a.filter) {
#pragma unroll
        for (int r = 0; r < R; r++)
            if (q[r].s >= 0) B[q[r].s] = filter_rhs(view_of<T>(A, q[r], mp, per), q[r].i, cf);
        __syncthreads();
        T* X = B;
        if (a.ftab1.implicit) X = pcr_solve<T, 1, R>(B, Cb, mp, a.ftab1, q);
#pragma unroll
        for (int r = 0; r < R; r++)
            if (q[r].s >= 0) X[q[r].s] += A[q[r].s];
        __syncthreads();
        V = X;
    }
    f2_line_bc<T, M, R>(a, mp, q, V);
    double ss = 0.0, mx = 0.0;
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (q[r].s < 0) continue;
        const long long e = q[r].node;
        const T nv = V[q[r].s];
        a.phin_w[e] = nv;
        if (a.mask[e]) continue;
        const double d = double(nv) - double(ov[r]);
        ss += d * d;
        mx = fmax(mx, fabs(d));
    }
    // block reduction, then the last block reduces the block partials in a fixed order
    const int lane = tid & 31, wid = tid >> 5, nw = (nth + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        s_ss[wid] = ss;
        s_mx[wid] = mx;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0, m = 0.0;
        for (int w = 0; w < nw; w++) {
            t += s_ss[w];
            m = fmax(m, s_mx[w]);
        }
        a.partial[2 * blockIdx.x] = t;
        a.partial[2 * blockIdx.x + 1] = m;
        __threadfence();
        unsigned v = atomicAdd(a.counter, 1u);
        s_last = (v == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // blocks of stacked grid k are the contiguous range [k * bpm, (k + 1) * bpm)
    const int bpm = gridDim.x / a.batch;
    for (int k = 0; k < a.batch; k++) {
        ss = 0.0;
        mx = 0.0;
        for (int b = k * bpm + tid; b < (k + 1) * bpm; b += nth) {
            ss += __ldcg(a.partial + 2 * b);
            mx = fmax(mx, __ldcg(a.partial + 2 * b + 1));
        }
        for (int o = 16; o > 0; o >>= 1) {
            ss += __shfl_down_sync(0xffffffffu, ss, o);
            mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        }
        __syncthreads();
        if (lane == 0) {
            s_ss[wid] = ss;
            s_mx[wid] = mx;
        }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0, m = 0.0;
            for (int w = 0; w < nw; w++) {
                t += s_ss[w];
                m = fmax(m, s_mx[w]);
            }
            a.result[2 * k] = t;
            a.result[2 * k + 1] = m;
        }
    }
    if (tid == 0) *a.counter = 0u;
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------

static const size_t F2_SMEM_LIMIT = 200 * 1024;

template <typename K>
static cudaError_t allow_smem(K kern)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F2_SMEM_LIMIT);
}

// line shape of direction d for a pass holding `bufs` block-local arrays of T
static void f2_shape(const Dims& D, int d, int bufs, size_t es, int& lpb, int& thr, size_t& sm)
{
    line_launch_shape(d, D.n[d], D.nlines(d), bufs / 2 > 0 ? bufs / 2 : 1, es, lpb, thr, sm);
    sm = (size_t)bufs * lpb * D.n[d] * es;
}

template <typename T, typename M, int R>
static cudaError_t f2_launch_r(F2Args<T, M> a, int which, cudaStream_t st, int thr, size_t sm)
{
    static int attr = 0;
    if (!attr) {
        cudaError_t e;
        if ((e = allow_smem(k_f2_deriv<T, M, R>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_f2_div<T, M, 2, R>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_f2_div<T, M, 4, R>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_f2_filter_commit<T, M, R>)) != cudaSuccess) return e;
        attr = 1;
    }
    if (which == F2_DERIV) k_f2_deriv<T, M, R><<<a.nb[0] + a.nb[1], thr, sm, st>>>(a);
    else if (which == F2_DIV) {
        if (a.curvature && !a.poisson) k_f2_div<T, M, 4, R><<<a.nb[0] + a.nb[1] + a.nb[2], thr, sm, st>>>(a);
        else k_f2_div<T, M, 2, R><<<a.nb[0] + a.nb[1] + a.nb[2], thr, sm, st>>>(a);
    } else k_f2_filter_commit<T, M, R><<<a.nb[1], thr, sm, st>>>(a);
    return cudaGetLastError();
}

template <typename T, typename M>
cudaError_t f2_launch(F2Args<T, M> a, int which, cudaStream_t st)
{
    const Dims& D = a.D;
    if (which == F2_STAGE) {
        int thr = a.stage_threads > 0 ? a.stage_threads : 256;
        const int row = (D.n[0] + 31) / 32 * 32;
        if (thr > row) thr = row;
        const dim3 grd((unsigned)((D.n[0] + thr - 1) / thr), (unsigned)D.n[1], (unsigned)D.n[2]);
        // the equation's branches as template flags, so that every load they guard can be
        // issued ahead of the arithmetic
        const bool lad = a.equation == WD_HJ_LAD, curv = a.curvature != 0;
        if (a.poisson) k_f2_stage<T, M, true, false, false><<<grd, thr, 0, st>>>(a);
        else if (lad && curv) k_f2_stage<T, M, false, true, true><<<grd, thr, 0, st>>>(a);
        else if (lad) k_f2_stage<T, M, false, true, false><<<grd, thr, 0, st>>>(a);
        else if (curv) k_f2_stage<T, M, false, false, true><<<grd, thr, 0, st>>>(a);
        else k_f2_stage<T, M, false, false, false><<<grd, thr, 0, st>>>(a);
        return cudaGetLastError();
    }
    const size_t es = sizeof(T);
    int l0 = 1, t0 = 0, l1 = 1, t1 = 0;
    size_t m0 = 0, m1 = 0;
    int rmax = 1;
    if (which == F2_DERIV || which == F2_DIV) {
        const int bufs = which == F2_DERIV ? 2 : 2 * (a.curvature && !a.poisson ? 4 : 2);
        f2_shape(D, 0, bufs, es, l0, t0, m0);
        f2_shape(D, 1, bufs, es, l1, t1, m1);
        a.lpb[0] = l0;
        a.lpb[1] = l1;
        a.nb[0] = (D.nlines(0) + l0 - 1) / l0;
        a.nb[1] = (D.nlines(1) + l1 - 1) / l1;
        a.nb[2] = (which == F2_DIV && a.lad && !a.poisson) ? a.nb[0] : 0;
    } else {
        f2_shape(D, 1, which == F2_STAGE ? 2 : 3, es, l1, t1, m1);
        while (l1 > 1 && D.n[0] % l1) l1 /= 2;   // blocks never straddle two stacked grids
        a.lpb[1] = l1;
        a.nb[1] = (D.nlines(1) + l1 - 1) / l1;
        if (which == F2_FILTER && a.nb[1] > a.max_partials) return cudaErrorInvalidConfiguration;
    }
    const int thr = t0 > t1 ? t0 : t1;
    const size_t sm = m0 > m1 ? m0 : m1;
    if (sm > F2_SMEM_LIMIT) return cudaErrorInvalidConfiguration;
    if (t0) rmax = slots_per_thread(l0 * D.n[0], thr);
    if (t1) rmax = std::max(rmax, slots_per_thread(l1 * D.n[1], thr));
    if (rmax <= 1) return f2_launch_r<T, M, 1>(a, which, st, thr, sm);
    if (rmax <= 2) return f2_launch_r<T, M, 2>(a, which, st, thr, sm);
    if (rmax <= 4) return f2_launch_r<T, M, 4>(a, which, st, thr, sm);
    return cudaErrorInvalidConfiguration;
}

template cudaError_t f2_launch<double, double>(F2Args<double, double>, int, cudaStream_t);
template cudaError_t f2_launch<float, float>(F2Args<float, float>, int, cudaStream_t);

}  // namespace wd
