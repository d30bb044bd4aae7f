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
#include "wd_api_internal.h"
#include "wd_fused2d.h"
#include "wd_pcr.cuh"

namespace wd {

template <typename T, typename M>
__device__ __forceinline__ void grad_at(const F2Args<T, M>& a, long long node, M& ux, M& uy)
{
    const long long tot = a.D.total;
    const M d0 = M(a.D0[node]), d1 = M(a.D1[node]);
    ux = a.xi[0 * tot + node] * d0 + a.xi[3 * tot + node] * d1;   // xi_x D0 + eta_x D1
    uy = a.xi[1 * tot + node] * d0 + a.xi[4 * tot + node] * d1;   // xi_y D0 + eta_y D1
}

// ---- A: derivatives of phi along both directions (+ LAD fourth differences) ---------------
template <typename T, typename M>
__global__ void __launch_bounds__(512) k_f2_deriv(F2Args<T, M> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int set = blockIdx.x < a.nb[0] ? 0 : 1;
    const int dir = set;
    const int bidx = set == 0 ? blockIdx.x : blockIdx.x - a.nb[0];
    const Dims& D = a.D;
    const LineMap mp = make_map(D, dir, a.lpb[dir], D.nlines(dir), bidx * a.lpb[dir]);
    const int S = mp.size();
    T* A = reinterpret_cast<T*>(smraw);
    T* B = A + S;
    const int tid = threadIdx.x, nth = blockDim.x, per = D.per[dir];
    const long long st = D.stride(dir);
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        A[s] = a.src[D.line_base(dir, mp.q0 + l) + (long long)i * st];
    }
    __syncthreads();
    T* Lout = dir == 0 ? a.L0 : a.L1;
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        B[s] = deriv_rhs(A, mp, l, i, per, a.scheme);
        if (a.lad) {
            const long long node = D.line_base(dir, mp.q0 + l) + (long long)i * st;
            Lout[node] = T(a.lads[(long long)dir * D.total + node] * M(d4_row(A, mp, l, i, per)));
        }
    }
    __syncthreads();
    T* X = B;
    const LineTab<T>& tb = dir == 0 ? a.dtab0 : a.dtab1;
    if (tb.implicit) X = pcr_solve<T, 1>(B, A, mp, tb);
    T* Dout = dir == 0 ? a.D0 : a.D1;
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        Dout[D.line_base(dir, mp.q0 + l) + (long long)i * st] = X[s];
    }
}

// ---- B: divergence passes along both directions (+ Gaussian along direction 0) ----------
template <typename T, typename M, int NF>
__device__ void f2_div_line(const F2Args<T, M>& a, int dir, int bidx, T* A, T* B)
{
    const Dims& D = a.D;
    const LineMap mp = make_map(D, dir, a.lpb[dir], D.nlines(dir), bidx * a.lpb[dir]);
    const int S = mp.size();
    const int tid = threadIdx.x, nth = blockDim.x, per = D.per[dir];
    const long long st = D.stride(dir);
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        const long long node = D.line_base(dir, mp.q0 + l) + (long long)i * st;
        M ux, uy;
        grad_at(a, node, ux, uy);
        A[s] = T(ux);
        A[S + s] = T(uy);
        if (NF == 4) {
            const M g = sqrt(ux * ux + uy * uy) + M(a.eps0);
            A[2 * S + s] = T(ux / g);
            A[3 * S + s] = T(uy / g);
        }
    }
    __syncthreads();
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
#pragma unroll
        for (int f = 0; f < NF; f++) B[(size_t)f * S + s] = deriv_rhs(A + (size_t)f * S, mp, l, i, per, a.scheme);
    }
    __syncthreads();
    T* X = B;
    const LineTab<T>& tb = dir == 0 ? a.dtab0 : a.dtab1;
    if (tb.implicit) X = pcr_solve<T, NF>(B, A, mp, tb);
    T* lap = dir == 0 ? a.LAP0 : a.LAP1;
    T* kap = dir == 0 ? a.KAP0 : a.KAP1;
    const long long tot = D.total;
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        const long long node = D.line_base(dir, mp.q0 + l) + (long long)i * st;
        const M x0 = a.xi[(long long)(dir * 3 + 0) * tot + node];
        const M x1 = a.xi[(long long)(dir * 3 + 1) * tot + node];
        lap[node] = T(x0 * M(X[s]) + x1 * M(X[S + s]));
        if (NF == 4) kap[node] = T(x0 * M(X[2 * S + s]) + x1 * M(X[3 * S + s]));
    }
}

template <typename T, typename M>
__device__ void f2_gauss0(const F2Args<T, M>& a, int bidx, T* A, T* B)
{
    const Dims& D = a.D;
    const int dir = 0;
    const LineMap mp = make_map(D, dir, a.lpb[dir], D.nlines(dir), bidx * a.lpb[dir]);
    const int S = mp.size();
    const int tid = threadIdx.x, nth = blockDim.x, per = D.per[dir];
    const long long st = D.stride(dir);
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        const long long node = D.line_base(dir, mp.q0 + l) + (long long)i * st;
        T v = a.L0[node] + a.L1[node];
        A[s] = T(a.C_lad) * (v < T(0) ? -v : v);
    }
    __syncthreads();
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        const long long node = D.line_base(dir, mp.q0 + l) + (long long)i * st;
        a.G0[node] = gauss_rhs(A, mp, l, i, per);
    }
}

template <typename T, typename M, int NF>
__global__ void __launch_bounds__(512) k_f2_div(F2Args<T, M> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T* A = reinterpret_cast<T*>(smraw);
    int b = blockIdx.x;
    if (b < a.nb[0]) {
        T* B = A + (size_t)NF * a.lpb[0] * a.D.n[0];
        f2_div_line<T, M, NF>(a, 0, b, A, B);
        return;
    }
    b -= a.nb[0];
    if (b < a.nb[1]) {
        T* B = A + (size_t)NF * a.lpb[1] * a.D.n[1];
        f2_div_line<T, M, NF>(a, 1, b, A, B);
        return;
    }
    b -= a.nb[1];
    f2_gauss0<T, M>(a, b, A, A + (size_t)a.lpb[0] * a.D.n[0]);
}

// boundary conditions of one direction-1 line held in shared memory (slot s of node i):
// far-field / Neumann ends, then Dirichlet nodes (poisson: value 0, faces Neumann)
template <typename T, typename M>
__device__ void f2_line_bc(const F2Args<T, M>& a, const LineMap& mp, T* V)
{
    const Dims& D = a.D;
    const int N = mp.N, tid = threadIdx.x;
    const long long st = D.stride(1);
    for (int l = tid; l < mp.nl; l += blockDim.x) {
        const int q = mp.q0 + l;         // = i index of the line (2-D, direction 1)
        for (int side = 0; side < 2; side++) {
            int kind = side ? a.bchi1 : a.bclo1;
            if (kind != WD_BC_FARFIELD && kind != WD_BC_NEUMANN) continue;
            if (a.poisson) kind = WD_BC_NEUMANN;
            const int b = side ? N - 1 : 0, s1 = side ? N - 2 : 1, s2 = side ? N - 3 : 2;
            T v1 = V[mp.slot(l, s1)], v2 = V[mp.slot(l, s2)];
            if (kind == WD_BC_NEUMANN) V[mp.slot(l, b)] = v1;
            else V[mp.slot(l, b)] = v1 + T((side ? a.ffr_hi : a.ffr_lo)[q]) * (v1 - v2);
        }
    }
    __syncthreads();
    for (int s = tid; s < mp.size(); s += blockDim.x) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        const long long node = D.line_base(1, mp.q0 + l) + (long long)i * st;
        if (a.mask[node]) V[s] = a.poisson ? T(0) : a.dval[node];
    }
    __syncthreads();
}

// ---- C: Gaussian along direction 1, right-hand side, RK4 stage, line BCs ----------------
template <typename T, typename M>
__global__ void __launch_bounds__(512) k_f2_stage(F2Args<T, M> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Dims& D = a.D;
    const int dir = 1;
    const LineMap mp = make_map(D, dir, a.lpb[1], D.nlines(1), blockIdx.x * a.lpb[1]);
    const int S = mp.size();
    T* A = reinterpret_cast<T*>(smraw);
    T* V = A + S;
    const int tid = threadIdx.x, nth = blockDim.x, per = D.per[1];
    const long long st = D.stride(1);
    if (a.lad && !a.poisson) {
        for (int s = tid; s < S; s += nth) {
            int l, i;
            mp.decode(s, l, i);
            if (l >= mp.nl) continue;
            A[s] = a.G0[D.line_base(dir, mp.q0 + l) + (long long)i * st];
        }
        __syncthreads();
    }
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        const long long e = D.line_base(dir, mp.q0 + l) + (long long)i * st;
        T R, dtv, gam = T(0), v = T(0), gm = T(0);
        const T lap = a.LAP0[e] + a.LAP1[e];
        if (a.poisson) {
            R = T(1) + lap;                                                  // Eq. 19
        } else {
            M ux, uy;
            grad_at(a, e, ux, uy);
            const T tx = T(ux), ty = T(uy);
            const T g2 = tx * tx + ty * ty;
            gm = sqrt(g2);
            const T ph = a.src[e];
            const T php = ph > T(0) ? ph : T(0);
            if (a.equation == WD_HJ_STD) gam = T(a.eps) * php;               // Eq. 6
            else if (a.equation == WD_HJ_LAD) {                              // Eq. 7
                const T g1 = T(a.eps) * php, gl = gauss_rhs(A, mp, l, i, per);
                gam = g1 < gl ? g1 : gl;
            }
            if (a.curvature) {                                               // Eq. 25
                v = T(0.001) * (T(1) - gm) * (T(1) - gm);
                T corr = gm * (a.KAP0[e] + a.KAP1[e]);
                corr = corr > T(0) ? corr : T(0);
                R = T(1) + (gam + v) * (lap - corr) - g2;
            } else {
                R = T(1) + gam * lap - g2;                                   // Eqs. 5, 18
            }
        }
        if (a.stage == 0) {
            if (a.poisson) dtv = T(a.cfl) / T(a.sig2[e]);
            else {
                const T am = gm > T(1) ? gm : T(1);
                dtv = T(a.cfl) / (T(a.sig1[e]) * am + (gam + v) * T(a.sig2[e]));
            }
            a.dtv[e] = dtv;
        } else {
            dtv = a.dtv[e];
        }
        const T n = a.phin[e];
        T out;
        if (a.stage == 0) {
            a.acc[e] = R * T(1.0 / 6.0);
            out = n + T(0.5) * dtv * R;
        } else if (a.stage == 1) {
            a.acc[e] += R * T(1.0 / 3.0);
            out = n + T(0.5) * dtv * R;
        } else if (a.stage == 2) {
            a.acc[e] += R * T(1.0 / 3.0);
            out = n + dtv * R;
        } else {
            out = n + dtv * (a.acc[e] + R * T(1.0 / 6.0));
        }
        V[s] = out;
    }
    __syncthreads();
    f2_line_bc(a, mp, V);
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        a.dst[D.line_base(dir, mp.q0 + l) + (long long)i * st] = V[s];
    }
}

// ---- F: direction-1 filter, line BCs, change norms and commit ----------------------------
template <typename T, typename M>
__global__ void __launch_bounds__(512) k_f2_filter_commit(F2Args<T, M> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ T cf[6][6];
    __shared__ double s_ss[32], s_mx[32];
    __shared__ int s_last;
    const Dims& D = a.D;
    const int dir = 1;
    const LineMap mp = make_map(D, dir, a.lpb[1], D.nlines(1), blockIdx.x * a.lpb[1]);
    const int S = mp.size();
    T* A = reinterpret_cast<T*>(smraw);
    T* B = A + S;
    T* Cb = B + S;
    const int tid = threadIdx.x, nth = blockDim.x, per = D.per[1];
    const long long st = D.stride(1);
    for (int i = tid; i < 36; i += nth) {
        int hw = i / 6, m = i % 6;
        double v = 0.0;
        if (hw >= 1 && m >= 1 && m <= hw) v = 0.5 * a.fa[hw][m] - (m == 1 ? a.alpha_f : 0.0);
        cf[hw][m] = T(v);
    }
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        A[s] = a.src[D.line_base(dir, mp.q0 + l) + (long long)i * st];
    }
    __syncthreads();
    T* V = A;
    if (a.filter) {
        for (int s = tid; s < S; s += nth) {
            int l, i;
            mp.decode(s, l, i);
            if (l >= mp.nl) continue;
            B[s] = filter_rhs(A, mp, l, i, per, cf);
        }
        __syncthreads();
        T* X = B;
        if (a.ftab1.implicit) X = pcr_solve<T, 1>(B, Cb, mp, a.ftab1);
        for (int s = tid; s < S; s += nth) {
            int l, i;
            mp.decode(s, l, i);
            if (l >= mp.nl) continue;
            X[s] += A[s];
        }
        __syncthreads();
        V = X;
    }
    f2_line_bc(a, mp, V);
    double ss = 0.0, mx = 0.0;
    for (int s = tid; s < S; s += nth) {
        int l, i;
        mp.decode(s, l, i);
        if (l >= mp.nl) continue;
        const long long e = D.line_base(dir, mp.q0 + l) + (long long)i * st;
        const T nv = V[s], ov = a.phin[e];
        a.phin_w[e] = nv;
        if (a.mask[e]) continue;
        const double d = double(nv) - double(ov);
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
    ss = 0.0;
    mx = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += nth) {
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
        a.result[0] = t;
        a.result[1] = m;
        *a.counter = 0u;
    }
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

template <typename T, typename M>
cudaError_t f2_launch(F2Args<T, M> a, int which, cudaStream_t st)
{
    static int attr = 0;
    if (!attr) {
        cudaError_t e;
        if ((e = allow_smem(k_f2_deriv<T, M>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_f2_div<T, M, 2>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_f2_div<T, M, 4>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_f2_stage<T, M>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_f2_filter_commit<T, M>)) != cudaSuccess) return e;
        attr = 1;
    }
    const Dims& D = a.D;
    const size_t es = sizeof(T);
    int l0, t0, l1, t1;
    size_t m0, m1;
    if (which == F2_DERIV) {
        f2_shape(D, 0, 2, es, l0, t0, m0);
        f2_shape(D, 1, 2, es, l1, t1, m1);
        a.lpb[0] = l0;
        a.lpb[1] = l1;
        a.nb[0] = (D.nlines(0) + l0 - 1) / l0;
        a.nb[1] = (D.nlines(1) + l1 - 1) / l1;
        size_t sm = m0 > m1 ? m0 : m1;
        if (sm > F2_SMEM_LIMIT) return cudaErrorInvalidConfiguration;
        k_f2_deriv<T, M><<<a.nb[0] + a.nb[1], t0 > t1 ? t0 : t1, sm, st>>>(a);
    } else if (which == F2_DIV) {
        const int nf = a.curvature && !a.poisson ? 4 : 2;
        f2_shape(D, 0, 2 * nf, es, l0, t0, m0);
        f2_shape(D, 1, 2 * nf, es, l1, t1, m1);
        a.lpb[0] = l0;
        a.lpb[1] = l1;
        a.nb[0] = (D.nlines(0) + l0 - 1) / l0;
        a.nb[1] = (D.nlines(1) + l1 - 1) / l1;
        a.nb[2] = (a.lad && !a.poisson) ? a.nb[0] : 0;
        size_t sm = m0 > m1 ? m0 : m1;
        if (sm > F2_SMEM_LIMIT) return cudaErrorInvalidConfiguration;
        int thr = t0 > t1 ? t0 : t1;
        if (nf == 4) k_f2_div<T, M, 4><<<a.nb[0] + a.nb[1] + a.nb[2], thr, sm, st>>>(a);
        else k_f2_div<T, M, 2><<<a.nb[0] + a.nb[1] + a.nb[2], thr, sm, st>>>(a);
    } else if (which == F2_STAGE) {
        f2_shape(D, 1, 2, es, l1, t1, m1);
        a.lpb[1] = l1;
        a.nb[1] = (D.nlines(1) + l1 - 1) / l1;
        if (m1 > F2_SMEM_LIMIT) return cudaErrorInvalidConfiguration;
        k_f2_stage<T, M><<<a.nb[1], t1, m1, st>>>(a);
    } else {
        f2_shape(D, 1, 3, es, l1, t1, m1);
        a.lpb[1] = l1;
        a.nb[1] = (D.nlines(1) + l1 - 1) / l1;
        if (m1 > F2_SMEM_LIMIT || a.nb[1] > a.max_partials) return cudaErrorInvalidConfiguration;
        k_f2_filter_commit<T, M><<<a.nb[1], t1, m1, st>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t f2_launch<double, double>(F2Args<double, double>, int, cudaStream_t);
template cudaError_t f2_launch<float, double>(F2Args<float, double>, int, cudaStream_t);
template cudaError_t f2_launch<float, float>(F2Args<float, float>, int, cudaStream_t);

}  // namespace wd
