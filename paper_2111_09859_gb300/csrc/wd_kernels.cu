// wd_kernels.cu -- sm_103a kernels of the HJ / LAD pseudo-HJ wall-distance solver.
//
//  k_line        one grid direction, whole lines staged in shared memory: explicit or
//                compact first derivatives (Sec. 3.2.2, Eq. 16), the implicit filter
//                (Sec. 3.4, Eq. 21) and the Gaussian smoothing of the LAD diffusivity;
//                tridiagonal systems are solved by the partition method (wd_linesys.cu);
//                the epilogue either stores each field or accumulates a metric-weighted
//                divergence (the Laplacian / curvature terms of Eqs. 9 and 25).
//  k_grad        chain rule U_m = sum_l d(xi_l)/d(x_m) d(phi)/d(xi_l) (Sec. 3.1) and the
//                unit normal n = U / (|U| + eps0) of Eq. 25.
//  k_lad_raw     C |sum_l (sum_m xi_{l,x_m}^2)^2 d4_l(phi) Delta x_l^e| of Eq. 7.
//  k_stage       HJ or Poisson right-hand side (Eqs. 5-7, 18-19, 25), local pseudo time
//                step and one classical RK4 stage (Sec. 3.3).
//  k_bc_face / k_bc_mask   boundary conditions (Sec. 3.5, Eqs. 22-23).
//  k_norms       RMS and max of the pseudo-step change over active nodes (Eq. 20),
//                double accumulation, deterministic order; also commits the new state.
//  metric kernels (Sec. 3.1), spacing ratios of far-field faces, masks.
#include <cstdio>

#include "wd_api_internal.h"
#include "wd_pcr.cuh"

namespace wd {

// ------------------------------------------------------------------------------------
// k_line: generic line pass.  A block loads its lines into shared memory, evaluates the
// rows (derivative, delta-form filter or Gaussian), solves the tridiagonal systems by PCR
// (compact derivatives, filter) and either stores every field or accumulates the
// metric-weighted divergence out0 (+)= sum_{m<nU} xi_{dir,m} F_m,
// out1 (+)= sum_m xi_{dir,m} F_{nU+m} (Laplacian and curvature terms of Eqs. 9 and 25).
// ------------------------------------------------------------------------------------

template <typename T, typename M, int NF, int EPI, int KIND, int R>
__global__ void __launch_bounds__(512)
k_line(Dims D, int dir, int nlines, int LPB, LineTab<T> tab, LineOp op, Fields<T> f,
       const M* __restrict__ xi, int nU, int accumulate)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ T cf[6][6];
    const LineMap mp = make_map(D, dir, LPB, nlines, blockIdx.x * LPB);
    const int S = mp.size();
    T* A = reinterpret_cast<T*>(smraw);
    T* B = A + (size_t)NF * S;
    const int per = D.per[dir];
    Slot q[R];
    slots_init<R>(q, mp, D);
    if (KIND == OPK_FILTER)
        for (int i = threadIdx.x; i < 36; i += blockDim.x) {
            const int hw = i / 6, m = i % 6;
            double v = 0.0;
            if (hw >= 1 && m >= 1 && m <= hw) v = 0.5 * op.fa[hw][m] - (m == 1 ? op.fa[0][1] : 0.0);
            cf[hw][m] = T(v);
        }
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (q[r].s < 0) continue;
#pragma unroll
        for (int fi = 0; fi < NF; fi++) A[(size_t)fi * S + q[r].s] = f.in[fi][q[r].node];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (q[r].s < 0) continue;
#pragma unroll
        for (int fi = 0; fi < NF; fi++) {
            const LineView<T> v = view_of<T>(A + (size_t)fi * S, q[r], mp, per);
            T x;
            if (KIND == OPK_DERIV) x = deriv_rhs(v, q[r].i, op.scheme);
            else if (KIND == OPK_FILTER) x = filter_rhs(v, q[r].i, cf);
            else x = gauss_rhs(v, q[r].i);
            B[(size_t)fi * S + q[r].s] = x;
        }
    }
    __syncthreads();
    T* X = B;
    if (tab.implicit) X = pcr_solve<T, NF, R>(B, A, mp, tab, q);
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int sl = q[r].s;
        if (sl < 0) continue;
        const long long node = q[r].node;
        if (EPI == 0) {
#pragma unroll
            for (int fi = 0; fi < NF; fi++) {
                T v = X[(size_t)fi * S + sl];
                if (KIND == OPK_FILTER) v += f.in[fi][node];
                f.out[fi][node] = v;
            }
        } else {
            M s0 = M(0), s1 = M(0);
            for (int m = 0; m < nU; m++) {
                const M x = xi[(long long)(dir * 3 + m) * D.total + node];
                s0 += x * M(X[(size_t)m * S + sl]);
                if (NF > nU) s1 += x * M(X[(size_t)(nU + m) * S + sl]);
            }
            T* o0 = f.out[0];
            o0[node] = accumulate ? T(M(o0[node]) + s0) : T(s0);
            if (NF > nU) {
                T* o1 = f.out[1];
                o1[node] = accumulate ? T(M(o1[node]) + s1) : T(s1);
            }
        }
    }
}

template <typename T, typename M, int NF, int EPI, int KIND, int R>
static cudaError_t line_dispatch_r(const Dims& D, int dir, const HostLineTab& tab, const LineOp& op,
                                   const Fields<T>& f, const M* xi, int nU, int accumulate,
                                   cudaStream_t st, int LPB, int threads, size_t sm)
{
    static int attr_done = 0;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_line<T, M, NF, EPI, KIND, R>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_done = 1;
    }
    const int nlines = D.nlines(dir);
    int grid = (nlines + LPB - 1) / LPB;
    k_line<T, M, NF, EPI, KIND, R><<<grid, threads, sm, st>>>(D, dir, nlines, LPB, tab.view<T>(), op,
                                                              f, xi, nU, accumulate);
    return cudaGetLastError();
}

template <typename T, typename M, int NF, int EPI, int KIND>
static cudaError_t line_dispatch(const Dims& D, int dir, const HostLineTab& tab, const LineOp& op,
                                 const Fields<T>& f, const M* xi, int nU, int accumulate,
                                 cudaStream_t st)
{
    const int nlines = D.nlines(dir);
    int LPB, threads;
    size_t sm;
    line_launch_shape(dir, D.n[dir], nlines, NF, sizeof(T), LPB, threads, sm);
    if (sm > 200 * 1024) return cudaErrorInvalidConfiguration;
    const int R = slots_per_thread(LPB * D.n[dir], threads);
    if (R <= 1) return line_dispatch_r<T, M, NF, EPI, KIND, 1>(D, dir, tab, op, f, xi, nU, accumulate, st, LPB, threads, sm);
    if (R <= 2) return line_dispatch_r<T, M, NF, EPI, KIND, 2>(D, dir, tab, op, f, xi, nU, accumulate, st, LPB, threads, sm);
    if (R <= 4) return line_dispatch_r<T, M, NF, EPI, KIND, 4>(D, dir, tab, op, f, xi, nU, accumulate, st, LPB, threads, sm);
    return cudaErrorInvalidConfiguration;
}

template <typename T, typename M>
cudaError_t launch_line(const Dims& D, int dir, const HostLineTab& tab, const LineOp& op, int nf,
                        int epi, const Fields<T>& f, const M* xi, int nU, int accumulate,
                        cudaStream_t st)
{
    if (tab.N != D.n[dir]) return cudaErrorInvalidValue;
    if (op.kind == OPK_FILTER && nf == 1 && epi == 0)
        return line_dispatch<T, M, 1, 0, OPK_FILTER>(D, dir, tab, op, f, xi, nU, accumulate, st);
    if (op.kind == OPK_GAUSS && nf == 1 && epi == 0)
        return line_dispatch<T, M, 1, 0, OPK_GAUSS>(D, dir, tab, op, f, xi, nU, accumulate, st);
    if (op.kind != OPK_DERIV) return cudaErrorInvalidValue;
    if (epi == 0) {
        switch (nf) {
        case 1: return line_dispatch<T, M, 1, 0, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (nf) {
    case 2: return line_dispatch<T, M, 2, 1, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
    case 3: return line_dispatch<T, M, 3, 1, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
    case 4: return line_dispatch<T, M, 4, 1, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
    case 6: return line_dispatch<T, M, 6, 1, OPK_DERIV>(D, dir, tab, op, f, xi, nU, accumulate, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------------------------
// pointwise kernels (grid-stride over the padded layout, padding skipped)
// ------------------------------------------------------------------------------------

static inline int pw_grid(long long total)
{
    long long b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T, typename M>
__global__ void k_grad(Dims D, const T* __restrict__ D0, const T* __restrict__ D1,
                       const T* __restrict__ D2, const M* __restrict__ xi, T* U0, T* U1, T* U2,
                       T* n0, T* n1, T* n2, double eps0)
{
    const long long tot = D.total;
    const int nd = D.ndim;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        M d[3] = {M(D0[e]), M(D1[e]), nd == 3 ? M(D2[e]) : M(0)};
        M u[3] = {M(0), M(0), M(0)};
        for (int m = 0; m < nd; m++) {
            M s = M(0);
            for (int l = 0; l < nd; l++) s += xi[(long long)(l * 3 + m) * tot + e] * d[l];
            u[m] = s;
        }
        U0[e] = T(u[0]);
        U1[e] = T(u[1]);
        if (nd == 3) U2[e] = T(u[2]);
        if (n0) {
            M g = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) + M(eps0);
            n0[e] = T(u[0] / g);
            n1[e] = T(u[1] / g);
            if (nd == 3) n2[e] = T(u[2] / g);
        }
    }
}

template <typename T, typename M>
cudaError_t launch_grad(const Dims& D, const T* const* Dl, const M* xi, T* const* U,
                        T* const* nv, double eps0, cudaStream_t st)
{
    k_grad<T, M><<<pw_grid(D.total), 256, 0, st>>>(D, Dl[0], Dl[1], Dl[2], xi, U[0], U[1], U[2],
                                                   nv ? nv[0] : nullptr, nv ? nv[1] : nullptr,
                                                   nv ? nv[2] : nullptr, eps0);
    return cudaGetLastError();
}

template <typename T, typename M>
__global__ void k_lad_raw(Dims D, const T* __restrict__ phi, const M* __restrict__ lads, double C,
                          T* out)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % D.pitch);
        if (i >= D.n[0]) continue;
        long long r = e / D.pitch;
        int crd[3] = {i, (int)(r % D.n[1]), (int)(r / D.n[1])};
        M s = M(0);
        for (int l = 0; l < D.ndim; l++) {
            int n = D.n[l], t = crd[l];
            int c = t;
            if (!D.per[l]) c = c < 2 ? 2 : (c > n - 3 ? n - 3 : c);
            long long sl = D.stride(l);
            long long base = e + (long long)(c - t) * sl;
            int o[5];
            for (int k = 0; k < 5; k++) {
                int q = c + k - 2;
                if (D.per[l]) q = q < 0 ? q + n : (q >= n ? q - n : q);
                o[k] = q - c;
            }
            M d4 = M(phi[base + o[0] * sl]) - M(4) * M(phi[base + o[1] * sl]) + M(6) * M(phi[base])
                 - M(4) * M(phi[base + o[3] * sl]) + M(phi[base + o[4] * sl]);
            s += lads[(long long)l * tot + e] * d4;
        }
        out[e] = T(M(C) * (s < M(0) ? -s : s));
    }
}

template <typename T, typename M>
cudaError_t launch_lad_raw(const Dims& D, const T* phi, const M* lads, double C, T* out,
                           cudaStream_t st)
{
    k_lad_raw<T, M><<<pw_grid(D.total), 256, 0, st>>>(D, phi, lads, C, out);
    return cudaGetLastError();
}

// HJ / Poisson right-hand side, local pseudo time step and one classical RK4 stage.
template <typename T, typename M>
__global__ void k_stage(Dims D, StageArgs<T, M> a, int stage)
{
    const long long tot = D.total;
    const int nd = D.ndim;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        T R, dtv;
        T gam = T(0), v = T(0), gm = T(0);
        if (a.poisson) {
            R = T(1) + a.lap[e];                                       // Eq. 19
        } else {
            T g2 = a.U[0][e] * a.U[0][e] + a.U[1][e] * a.U[1][e];
            if (nd == 3) g2 += a.U[2][e] * a.U[2][e];
            gm = sqrt(g2);
            T ph = a.src[e];
            T php = ph > T(0) ? ph : T(0);
            if (a.equation == WD_HJ_STD) gam = T(a.eps) * php;         // Eq. 6
            else if (a.equation == WD_HJ_LAD) {                        // Eq. 7
                T g1 = T(a.eps) * php, g2l = a.lad[e];
                gam = g1 < g2l ? g1 : g2l;
            }
            const T a2 = a.adv ? a.adv[e] : g2;                       // U.grad(phi)
            if (a.curvature) {                                         // Eq. 25
                v = T(0.001) * (T(1) - gm) * (T(1) - gm);
                T corr = gm * a.kap[e];
                corr = corr > T(0) ? corr : T(0);
                R = T(1) + (gam + v) * (a.lap[e] - corr) - a2;
            } else {
                R = T(1) + gam * a.lap[e] - a2;                        // Eqs. 5, 18
            }
        }
        if (stage <= 0) {
            if (a.poisson) dtv = T(a.cfl) / T(a.sig2[e]);
            else {
                T am = gm > T(1) ? gm : T(1);
                dtv = T(a.cfl) / (T(a.sig1[e]) * am + (gam + v) * T(a.sig2[e]));
            }
            a.dt[e] = dtv;
        } else {
            dtv = a.dt[e];
        }
        if (stage < 0) {
            a.dst[e] = R;
            continue;
        }
        T n = a.phin[e];
        T out;
        if (stage == 0) {
            a.acc[e] = R * T(1.0 / 6.0);
            out = n + T(0.5) * dtv * R;
        } else if (stage == 1) {
            a.acc[e] += R * T(1.0 / 3.0);
            out = n + T(0.5) * dtv * R;
        } else if (stage == 2) {
            a.acc[e] += R * T(1.0 / 3.0);
            out = n + dtv * R;
        } else {
            out = n + dtv * (a.acc[e] + R * T(1.0 / 6.0));
        }
        a.dst[e] = out;
    }
}

template <typename T, typename M>
cudaError_t launch_stage(const Dims& D, const StageArgs<T, M>& a, int stage, cudaStream_t st)
{
    k_stage<T, M><<<pw_grid(D.total), 256, 0, st>>>(D, a, stage);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_spalding(Dims D, const T* __restrict__ U0, const T* __restrict__ U1,
                           const T* __restrict__ U2, const T* __restrict__ phip, T* phi)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        T g2 = U0[e] * U0[e] + U1[e] * U1[e];
        if (D.ndim == 3) g2 += U2[e] * U2[e];
        // Eq. 4 with the minus root, -g + sqrt(g^2 + 2 phi'), evaluated in the equivalent
        // form 2 phi' / (g + sqrt(g^2 + 2 phi')) that does not cancel when 2 phi' << g^2
        T g = sqrt(g2);
        T arg = g2 + T(2) * phip[e];
        T r = sqrt(arg > T(0) ? arg : T(0));
        phi[e] = (arg > T(0) && g + r > T(0)) ? T(2) * phip[e] / (g + r) : -g;
    }
}

template <typename T, typename M>
cudaError_t launch_spalding(const Dims& D, const T* const* U, const T* phip, T* phi,
                            cudaStream_t st)
{
    k_spalding<T><<<pw_grid(D.total), 256, 0, st>>>(D, U[0], U[1], U[2], phip, phi);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// boundary conditions
// ------------------------------------------------------------------------------------

// Both directions' far-field / Neumann faces of a single 2-D grid in one launch, with the
// result of the two direction passes followed by the Dirichlet reset of the face nodes
// (interior nodes must already hold their Dirichlet values).  Direction-1 face nodes at the
// corners re-evaluate the two direction-0 face values they extrapolate from; direction-0
// threads leave the rows that a direction-1 face overwrites.
template <typename T>
__device__ __forceinline__ T face_value(int kind, T v1, T v2, double r)
{
    return kind == WD_BC_NEUMANN ? v1 : v1 + T(r) * (v1 - v2);
}

template <typename T>
__global__ void k_bc_faces2d(Dims D, int klo0, int khi0, int klo1, int khi1, const double* __restrict__ r0lo,
                             const double* __restrict__ r0hi, const double* __restrict__ r1lo,
                             const double* __restrict__ r1hi, const uint8_t* __restrict__ mask,
                             const T* __restrict__ dval, int poisson, T* phi)
{
    const int n0 = D.n[0], n1 = D.n[1];
    const long long p1 = D.pitch;
    auto act = [](int k) { return k == WD_BC_FARFIELD || k == WD_BC_NEUMANN; };
    const bool f1lo = act(klo1), f1hi = act(khi1);
    // direction-0 face value at row j (side 0: i = 0, side 1: i = n0 - 1), from interior values
    auto v0 = [&](int side, int j) -> T {
        const int kind = side ? khi0 : klo0;
        const long long b = D.idx(side ? n0 - 1 : 0, j, 0);
        const long long s = side ? -1 : 1;
        return face_value<T>(kind, phi[b + s], phi[b + 2 * s], (side ? r0hi : r0lo)[j]);
    };
    const int nf0 = 2 * n1, nf1 = 2 * n0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nf0 + nf1; e += gridDim.x * blockDim.x) {
        if (e < nf0) {
            const int side = e / n1, j = e - side * n1;
            const int kind = side ? khi0 : klo0;
            if (!act(kind)) continue;
            if ((j == 0 && f1lo) || (j == n1 - 1 && f1hi)) continue;   // a direction-1 face wins
            const long long b = D.idx(side ? n0 - 1 : 0, j, 0);
            T v = v0(side, j);
            if (mask[b]) v = poisson ? T(0) : dval[b];
            phi[b] = v;
        } else {
            const int q = e - nf0, side = q / n0, i = q - side * n0;
            const int kind = side ? khi1 : klo1;
            if (!act(kind)) continue;
            const int j = side ? n1 - 1 : 0, js = side ? -1 : 1;
            const long long b = D.idx(i, j, 0);
            T w1, w2;
            if ((i == 0 && act(klo0)) || (i == n0 - 1 && act(khi0))) {
                const int s0 = i == 0 ? 0 : 1;
                w1 = v0(s0, j + js);
                w2 = v0(s0, j + 2 * js);
            } else {
                w1 = phi[b + js * p1];
                w2 = phi[b + 2 * js * p1];
            }
            T v = face_value<T>(kind, w1, w2, (side ? r1hi : r1lo)[i]);
            if (mask[b]) v = poisson ? T(0) : dval[b];
            phi[b] = v;
        }
    }
}

template <typename T>
cudaError_t launch_bc_faces2d(const Dims& D, const int* klo, const int* khi, const double* const* rlo,
                              const double* const* rhi, const uint8_t* mask, const T* dval, int poisson, T* phi,
                              cudaStream_t st)
{
    const int n = 2 * (D.n[0] + D.n[1]);
    k_bc_faces2d<T><<<(n + 255) / 256, 256, 0, st>>>(D, klo[0], khi[0], klo[1], khi[1], rlo[0], rhi[0], rlo[1],
                                                     rhi[1], mask, dval, poisson, phi);
    return cudaGetLastError();
}
template cudaError_t launch_bc_faces2d<float>(const Dims&, const int*, const int*, const double* const*,
                                              const double* const*, const uint8_t*, const float*, int, float*,
                                              cudaStream_t);
template cudaError_t launch_bc_faces2d<double>(const Dims&, const int*, const int*, const double* const*,
                                               const double* const*, const uint8_t*, const double*, int, double*,
                                               cudaStream_t);

template <typename T>
__global__ void k_bc_face(Dims D, int d, int klo, int khi, const double* __restrict__ rlo,
                          const double* __restrict__ rhi, T* phi)
{
    const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
    const int fsize = D.n[o1] * D.n[o2];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * fsize; e += gridDim.x * blockDim.x) {
        int side = e / fsize, fidx = e - side * fsize;
        int kind = side ? khi : klo;
        if (kind != WD_BC_FARFIELD && kind != WD_BC_NEUMANN) continue;
        int c[3];
        c[o1] = fidx % D.n[o1];
        c[o2] = fidx / D.n[o1];
        c[d] = side ? D.n[d] - 1 : 0;
        long long p = D.idx(c[0], c[1], c[2]);
        long long s = side ? -D.stride(d) : D.stride(d);
        if (kind == WD_BC_NEUMANN) phi[p] = phi[p + s];
        else {
            T r = T((side ? rhi : rlo)[fidx]);
            T a1 = phi[p + s], a2 = phi[p + 2 * s];
            phi[p] = a1 + r * (a1 - a2);
        }
    }
}

template <typename T>
cudaError_t launch_bc_face(const Dims& D, int dir, int kind_lo, int kind_hi, const double* rlo,
                           const double* rhi, T* phi, cudaStream_t st)
{
    int o1 = (dir + 1) % 3, o2 = (dir + 2) % 3;
    int n = 2 * D.n[o1] * D.n[o2];
    k_bc_face<T><<<(n + 255) / 256, 256, 0, st>>>(D, dir, kind_lo, kind_hi, rlo, rhi, phi);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_bc_mask(Dims D, const uint8_t* __restrict__ mask, const T* __restrict__ dval, T* phi)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        if (mask[e]) phi[e] = dval ? dval[e] : T(0);
    }
}

template <typename T>
cudaError_t launch_bc_mask(const Dims& D, const uint8_t* mask, const T* dval, T* phi, cudaStream_t st)
{
    k_bc_mask<T><<<pw_grid(D.total), 256, 0, st>>>(D, mask, dval, phi);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// change norms (double, deterministic: fixed partition, fixed final order)
// ------------------------------------------------------------------------------------

template <typename T>
__global__ void k_norms(Dims D, const T* __restrict__ newp, T* oldp, const uint8_t* __restrict__ mask,
                        double* partial, unsigned* counter, double* result)
{
    __shared__ double s_ss[32], s_mx[32];
    __shared__ int s_last;
    const long long tot = D.total;
    double ss = 0.0, mx = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        T a = newp[e], b = oldp[e];
        oldp[e] = a;
        if (mask[e]) continue;
        double d = double(a) - double(b);
        ss += d * d;
        mx = fmax(mx, fabs(d));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        s_ss[wid] = ss;
        s_mx[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0;
        for (int w = 0; w < nw; w++) {
            a += s_ss[w];
            m = fmax(m, s_mx[w]);
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = m;
        __threadfence();
        unsigned v = atomicAdd(counter, 1u);
        s_last = (v == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ss = 0.0;
    mx = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        ss += __ldcg(partial + 2 * b);
        mx = fmax(mx, __ldcg(partial + 2 * b + 1));
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
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0;
        for (int w = 0; w < nw; w++) {
            a += s_ss[w];
            m = fmax(m, s_mx[w]);
        }
        result[0] = a;
        result[1] = m;
        *counter = 0u;
    }
}

template <typename T>
cudaError_t launch_norms(const Dims& D, const T* newp, T* oldp, const uint8_t* mask, double* partial,
                         unsigned* counter, double* result, int nblocks, cudaStream_t st)
{
    k_norms<T><<<nblocks, 256, 0, st>>>(D, newp, oldp, mask, partial, counter, result);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_fill(T* p, long long n, T v)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        p[e] = v;
}

template <typename T>
cudaError_t launch_fill(T* p, long long n, T v, cudaStream_t st)
{
    k_fill<T><<<pw_grid(n), 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// metrics (Sec. 3.1), computed once per grid in double
// ------------------------------------------------------------------------------------

__global__ void k_unwrap(Dims D, int dir, const double* __restrict__ x, double shift, double* out)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % D.pitch);
        if (i >= D.n[0]) continue;
        long long r = e / D.pitch;
        int crd[3] = {i, (int)(r % D.n[1]), (int)(r / D.n[1])};
        out[e] = x[e] - shift * (double)crd[dir] / (double)D.n[dir];
    }
}

template <typename S, typename DT>
__global__ void k_convert(const S* __restrict__ in, DT* out, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = DT(in[e]);
}

template <typename S, typename DT>
cudaError_t launch_convert(const S* in, DT* out, long long n, cudaStream_t st)
{
    k_convert<S, DT><<<pw_grid(n), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, long long, cudaStream_t);

cudaError_t launch_unwrap(const Dims& D, int dir, const double* x, double shift, double* out,
                          cudaStream_t st)
{
    k_unwrap<<<pw_grid(D.total), 256, 0, st>>>(D, dir, x, shift, out);
    return cudaGetLastError();
}

__global__ void k_add_const(Dims D, double* p, double c)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < D.total;
         e += (long long)gridDim.x * blockDim.x)
        if ((int)(e % D.pitch) < D.n[0]) p[e] += c;
}

cudaError_t launch_add_const(const Dims& D, double* p, double c, cudaStream_t st)
{
    k_add_const<<<pw_grid(D.total), 256, 0, st>>>(D, p, c);
    return cudaGetLastError();
}

// A[(m*3+l)*total + e] = dx_m/dxi_l (the periodic shift already added back).
template <typename M>
__global__ void k_metric_finish(Dims D, const double* __restrict__ A, double* xi_d, double* J,
                                double* dx, M* xi_m, M* sig1, M* sig2)
{
    const long long tot = D.total;
    const int nd = D.ndim;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        double a[3][3];
        for (int m = 0; m < 3; m++)
            for (int l = 0; l < 3; l++)
                a[m][l] = (m < nd && l < nd) ? A[(long long)(m * 3 + l) * tot + e] : (m == l ? 1.0 : 0.0);
        // cofactor expansion: inv[l][m] = cof[m][l] / det
        double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
        double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
        double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
        double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
        double inv[3][3];
        inv[0][0] = c00 / det;
        inv[1][0] = c01 / det;
        inv[2][0] = c02 / det;
        inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
        inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
        inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
        inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
        inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
        inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
        J[e] = det;
        double s1 = 0.0, s2 = 0.0;
        for (int l = 0; l < 3; l++) {
            double q = 0.0, col = 0.0;
            for (int m = 0; m < 3; m++) {
                double x = (l < nd && m < nd) ? inv[l][m] : 0.0;
                xi_d[(long long)(l * 3 + m) * tot + e] = x;
                if (xi_m) xi_m[(long long)(l * 3 + m) * tot + e] = M(x);
                q += x * x;
                if (m < nd && l < nd) col += a[m][l] * a[m][l];
            }
            dx[(long long)l * tot + e] = l < nd ? sqrt(col) : 0.0;
            if (l < nd) s1 += sqrt(q);
        }
        // time-step bound of the second-order term: Gershgorin sum of the contravariant
        // metric tensor g^{lk} = grad(xi_l) . grad(xi_k), cross terms included
        for (int l = 0; l < nd; l++)
            for (int k = 0; k < nd; k++) {
                double q = 0.0;
                for (int m = 0; m < nd; m++) q += inv[l][m] * inv[k][m];
                s2 += fabs(q);
            }
        sig1[e] = M(s1);
        sig2[e] = M(s2);
    }
}

template <typename M>
cudaError_t launch_metric_finish(const Dims& D, const double* A, double* xi_d, double* J, double* dx,
                                 M* xi_m, M* sig1, M* sig2, cudaStream_t st)
{
    k_metric_finish<M><<<pw_grid(D.total), 256, 0, st>>>(D, A, xi_d, J, dx, xi_m, sig1, sig2);
    return cudaGetLastError();
}

// LAD scale s_l = (sum_m xi_{l,x_m}^2)^2 Delta x_l^ex of Eq. 7
template <typename M>
__global__ void k_lad_scale(Dims D, const double* __restrict__ xi_d, const double* __restrict__ dx,
                            double ex, M* lads)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        for (int l = 0; l < D.ndim; l++) {
            double q = 0.0;
            for (int m = 0; m < D.ndim; m++) {
                double x = xi_d[(long long)(l * 3 + m) * tot + e];
                q += x * x;
            }
            lads[(long long)l * tot + e] = M(q * q * pow(dx[(long long)l * tot + e], ex));
        }
    }
}

template <typename M>
cudaError_t launch_lad_scale(const Dims& D, const double* xi_d, const double* dx, double ex, M* lads,
                             cudaStream_t st)
{
    k_lad_scale<M><<<pw_grid(D.total), 256, 0, st>>>(D, xi_d, dx, ex, lads);
    return cudaGetLastError();
}

// spacing ratio |x_b - x_b1| / |x_b1 - x_b2| on the face nodes of both faces of every
// direction; ratio[(2d+side)*fmax + fidx]
__global__ void k_ff_ratio(Dims D, const double* __restrict__ xyz, double* ratio, long long fmax)
{
    for (int d = 0; d < D.ndim; d++) {
        const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
        const int fsize = D.n[o1] * D.n[o2];
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * fsize; e += gridDim.x * blockDim.x) {
            int side = e / fsize, fidx = e - side * fsize;
            int c[3];
            c[o1] = fidx % D.n[o1];
            c[o2] = fidx / D.n[o1];
            c[d] = side ? D.n[d] - 1 : 0;
            long long p = D.idx(c[0], c[1], c[2]);
            long long s = side ? -D.stride(d) : D.stride(d);
            double d1 = 0.0, d2 = 0.0;
            for (int m = 0; m < 3; m++) {
                const double* x = xyz + (long long)m * D.total;
                double a = x[p] - x[p + s], b = x[p + s] - x[p + 2 * s];
                d1 += a * a;
                d2 += b * b;
            }
            ratio[(long long)(2 * d + side) * fmax + fidx] = sqrt(d1) / sqrt(d2);
        }
    }
}

cudaError_t launch_ff_ratio(const Dims& D, const double* xyz, double* ratio, long long fmax,
                            cudaStream_t st)
{
    k_ff_ratio<<<(int)((2 * fmax + 255) / 256), 256, 0, st>>>(D, xyz, ratio, fmax);
    return cudaGetLastError();
}

// mask[e] = wall[e] | user (dense); dval[e] = wall ? 0 : user value (dense)
template <typename T>
__global__ void k_mask_merge(Dims D, const uint8_t* __restrict__ um, const T* __restrict__ uv,
                             uint8_t* mask, T* dval, const uint8_t* __restrict__ wall)
{
    const long long tot = D.total;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e % D.pitch);
        if (i >= D.n[0]) continue;
        long long r = e / D.pitch;
        long long q = i + (long long)D.n[0] * r;     // dense index
        uint8_t w = wall[e];
        uint8_t u = um ? (um[q] != 0) : 0;
        mask[e] = w | u;
        dval[e] = (!w && u && uv) ? uv[q] : T(0);
    }
}

template <typename T>
cudaError_t launch_mask_merge(const Dims& D, const uint8_t* src_dense, const T* val_dense,
                              uint8_t* mask, T* dval, const uint8_t* wallmask, cudaStream_t st)
{
    k_mask_merge<T><<<pw_grid(D.total), 256, 0, st>>>(D, src_dense, val_dense, mask, dval, wallmask);
    return cudaGetLastError();
}

__global__ void k_count(Dims D, const uint8_t* __restrict__ mask, unsigned long long* out)
{
    unsigned long long c = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < D.total;
         e += (long long)gridDim.x * blockDim.x) {
        if ((int)(e % D.pitch) >= D.n[0]) continue;
        if (!mask[e]) c++;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

cudaError_t launch_count(const Dims& D, const uint8_t* mask, unsigned long long* out, cudaStream_t st)
{
    k_count<<<pw_grid(D.total), 256, 0, st>>>(D, mask, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// explicit instantiations: (state, metric) = (double, double), (float, float)
// ------------------------------------------------------------------------------------

#define WD_INST_TM(T, M)                                                                          \
    template cudaError_t launch_line<T, M>(const Dims&, int, const HostLineTab&, const LineOp&,   \
                                           int, int, const Fields<T>&, const M*, int, int,        \
                                           cudaStream_t);                                         \
    template cudaError_t launch_grad<T, M>(const Dims&, const T* const*, const M*, T* const*,     \
                                           T* const*, double, cudaStream_t);                      \
    template cudaError_t launch_lad_raw<T, M>(const Dims&, const T*, const M*, double, T*,        \
                                              cudaStream_t);                                      \
    template cudaError_t launch_stage<T, M>(const Dims&, const StageArgs<T, M>&, int,             \
                                            cudaStream_t);                                        \
    template cudaError_t launch_spalding<T, M>(const Dims&, const T* const*, const T*, T*,        \
                                               cudaStream_t);

WD_INST_TM(double, double)
WD_INST_TM(float, float)

#define WD_INST_T(T)                                                                              \
    template cudaError_t launch_bc_face<T>(const Dims&, int, int, int, const double*,             \
                                           const double*, T*, cudaStream_t);                      \
    template cudaError_t launch_bc_mask<T>(const Dims&, const uint8_t*, const T*, T*,             \
                                           cudaStream_t);                                         \
    template cudaError_t launch_norms<T>(const Dims&, const T*, T*, const uint8_t*, double*,      \
                                         unsigned*, double*, int, cudaStream_t);                  \
    template cudaError_t launch_fill<T>(T*, long long, T, cudaStream_t);                          \
    template cudaError_t launch_mask_merge<T>(const Dims&, const uint8_t*, const T*, uint8_t*,    \
                                              T*, const uint8_t*, cudaStream_t);

WD_INST_T(double)
WD_INST_T(float)

template cudaError_t launch_metric_finish<double>(const Dims&, const double*, double*, double*,
                                                  double*, double*, double*, double*, cudaStream_t);
template cudaError_t launch_metric_finish<float>(const Dims&, const double*, double*, double*,
                                                 double*, float*, float*, float*, cudaStream_t);
template cudaError_t launch_lad_scale<double>(const Dims&, const double*, const double*, double,
                                              double*, cudaStream_t);
template cudaError_t launch_lad_scale<float>(const Dims&, const double*, const double*, double,
                                             float*, cudaStream_t);
template cudaError_t launch_fill<uint8_t>(uint8_t*, long long, uint8_t, cudaStream_t);

}  // namespace wd
