// wd_zfilter.cu -- the implicit filter of Eq. 21 along direction 2 of a 3-D grid, fused with
// the commit of the pseudo step (Dirichlet reset, phi^n <- new state, change norms of Eq. 20),
// streamed along z.
//
// Direction 2 is the slowest in memory: its lines' nodes lie a whole plane apart.  Instead of
// staging lines in shared memory, one thread takes one (i, j) column and walks its z-line
// while the threads of a block hold up to 256 neighbouring columns of a row, so every access
// of a warp is a 128-byte row segment and a block's accesses to a plane one contiguous run.
// The filter system a_t x_{t-1} + x_t + c_t x_{t+1} = d_t (delta form: d_t the right-hand
// side of second differences, x_t = fh_t - f_t) is solved by the Thomas algorithm with factors
// computed once on the host:
//   forward  (t = 0 .. N-1):  y_t = (d_t - a_t y_{t-1}) / m_t      -> scratch
//   backward (t = N-1 .. 0):  x_t = y_t - c'_t x_{t+1},  fh_t = f_t + x_t, then the commit.
// Each sweep loads its next chunk of planes (16 forward, 8 backward) while it computes the
// current one, so that loads stay in flight across the whole sweep.  (Four columns per thread
// with 16-byte accesses, and chunks twice as long, measured slower.)  The right-hand side and
// the epilogue are those of the line passes: the order-2hw member with hw = min(5, distance to
// the nearer end), end nodes unfiltered; Dirichlet nodes take their values (0 in the Poisson
// phase); the squared changes of the other nodes are summed per block in double (per thread
// over chunks of 8 nodes in the state precision), the blocks in a fixed order.
#include "wd_zfilter.h"

namespace wd {

// 256 threads per block over up to 256 consecutive columns of a row (a block's accesses to a
// plane are then one contiguous run), 8 rows of 32 on narrower grids
static dim3 zf_block(const Dims& D)
{
    const int bx = D.n[0] >= 256 ? 256 : (D.n[0] >= 128 ? 128 : (D.n[0] >= 64 ? 64 : 32));
    return dim3(bx, 256 / bx, 1);
}

static dim3 zf_grid(const Dims& D)
{
    const dim3 b = zf_block(D);
    return dim3((D.n[0] + b.x - 1) / b.x, (D.n[1] + b.y - 1) / b.y, 1);
}

bool zfilter_supported(const Dims& D, int max_partials)
{
    if (D.ndim != 3 || D.per[2] || D.n[2] < 6) return false;
    const dim3 g = zf_grid(D);
    return (long long)g.x * g.y <= max_partials;
}

void zfilter_factors(double alpha_f, int N, double* out)
{
    std::vector<double> a, c;
    int imp;
    filter_rows(alpha_f, N, 0, a, c, imp);
    double cp = 0.0;
    for (int t = 0; t < N; t++) {
        const double m = 1.0 - a[t] * cp;
        cp = c[t] / m;
        out[t] = a[t];
        out[N + t] = cp;
        out[2 * N + t] = 1.0 / m;
    }
}

namespace {

constexpr int ZF_FWD = 16;   // planes per chunk of the forward sweep
constexpr int ZF_BWD = 8;    // of the backward sweep

// right-hand side of row t from the window v[0..10] = f_{t-5} .. f_{t+5} (Sec. 3.4: the
// order drops to 2 hw near the ends, the end rows are not filtered)
template <typename T>
__device__ __forceinline__ T zf_rhs(const T* v, int t, int N, const T (*cf)[6])
{
    const int e = t < N - 1 - t ? t : N - 1 - t;
    const int hw = e < 5 ? e : 5;
    const T f0 = v[5];
    T s = T(0);
    if (hw == 5) {
#pragma unroll
        for (int m = 5; m >= 1; m--) s += cf[5][m] * ((v[5 + m] - f0) + (v[5 - m] - f0));
        return s;
    }
#pragma unroll
    for (int m = 5; m >= 1; m--)
        if (m <= hw) s += cf[hw][m] * ((v[5 + m] - f0) + (v[5 - m] - f0));
    return s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_zf_fwd(ZfArgs<T> a)
{
    __shared__ T cf[6][6];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid < 36) cf[tid / 6][tid % 6] = a.cf[tid / 6][tid % 6];
    __syncthreads();
    const Dims& D = a.D;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= D.n[0] || j >= D.n[1]) return;
    const int N = D.n[2];
    const long long st = (long long)D.pitch * D.n[1];
    const T* f = a.src + i + (long long)D.pitch * j;
    T* y = a.scratch + i + (long long)D.pitch * j;
    const T* ta = a.tab;
    const T* tim = a.tab + 2 * N;
    // window w[m] = f_{k0 - 5 + m}: 11 planes around the chunk's first row and the chunk's
    // ZF_FWD planes ahead; the next chunk's planes (nx) are loaded before the current chunk
    // is computed (double buffer)
    T w[11 + ZF_FWD], nx[ZF_FWD];
#pragma unroll
    for (int m = 0; m < 5; m++) w[m] = T(0);
#pragma unroll
    for (int m = 5; m < 11; m++) w[m] = m - 5 < N ? f[(m - 5) * st] : T(0);
    auto load = [&](int k0) {
#pragma unroll
        for (int m = 0; m < ZF_FWD; m++) {
            const int kk = k0 + 6 + m;
            nx[m] = kk < N ? f[kk * st] : T(0);
        }
    };
    load(0);
    T yp = T(0);
    for (int k0 = 0; k0 < N; k0 += ZF_FWD) {
#pragma unroll
        for (int m = 0; m < ZF_FWD; m++) w[11 + m] = nx[m];
        if (k0 + ZF_FWD < N) load(k0 + ZF_FWD);
#pragma unroll
        for (int m = 0; m < ZF_FWD; m++) {
            const int k = k0 + m;
            if (k < N) {
                const T d = zf_rhs<T>(w + m, k, N, cf);
                yp = (d - __ldg(ta + k) * yp) * __ldg(tim + k);
                y[k * st] = yp;
            }
        }
#pragma unroll
        for (int m = 0; m < 11; m++) w[m] = w[m + ZF_FWD];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_zf_bwd(ZfArgs<T> a)
{
    __shared__ double s_ss[8], s_mx[8];
    const Dims& D = a.D;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, w = tid >> 5;
    double ss = 0.0;
    T mx = T(0);
    if (i < D.n[0] && j < D.n[1]) {
        const int N = D.n[2];
        const long long st = (long long)D.pitch * D.n[1], e0 = i + (long long)D.pitch * j;
        const T* tcp = a.tab + N;
        T x = T(0);
        // chunk buffers: the next chunk's loads are issued before the current one is computed
        T yn[ZF_BWD], fn[ZF_BWD], on[ZF_BWD];
        uint8_t mn[ZF_BWD];
        auto load = [&](int k0) {
#pragma unroll
            for (int m = 0; m < ZF_BWD; m++) {
                const int k = k0 - m;
                if (k >= 0) {
                    const long long e = e0 + k * st;
                    yn[m] = a.scratch[e];
                    fn[m] = a.src[e];
                    on[m] = a.phin[e];
                    mn[m] = a.mask[e];
                }
            }
        };
        load(N - 1);
        for (int k0 = N - 1; k0 >= 0; k0 -= ZF_BWD) {
            T yv[ZF_BWD], fv[ZF_BWD], ov[ZF_BWD];
            uint8_t mk[ZF_BWD];
#pragma unroll
            for (int m = 0; m < ZF_BWD; m++) yv[m] = yn[m], fv[m] = fn[m], ov[m] = on[m], mk[m] = mn[m];
            if (k0 - ZF_BWD >= 0) load(k0 - ZF_BWD);
            T cs = T(0);
#pragma unroll
            for (int m = 0; m < ZF_BWD; m++) {
                const int k = k0 - m;
                if (k >= 0) {
                    const long long e = e0 + k * st;
                    x = yv[m] - __ldg(tcp + k) * x;
                    T nv = fv[m] + x;   // delta form: f + (fh - f)
                    if (mk[m]) nv = a.poisson ? T(0) : __ldg(a.dval + e);
                    a.phin_w[e] = nv;
                    if (!mk[m]) {
                        const T d = nv - ov[m];
                        cs += d * d;
                        mx = fmax(mx, fabs(d));
                    }
                }
            }
            ss += double(cs);
        }
    }
    double mxd = double(mx);
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mxd = fmax(mxd, __shfl_down_sync(0xffffffffu, mxd, o));
    }
    if (lane == 0) {
        s_ss[w] = ss;
        s_mx[w] = mxd;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0, mm = 0.0;
        for (int k = 0; k < 8; k++) {
            t += s_ss[k];
            mm = fmax(mm, s_mx[k]);
        }
        const int b = blockIdx.y * gridDim.x + blockIdx.x;
        a.partial[2 * b] = t;
        a.partial[2 * b + 1] = mm;
    }
}

// the block partials in a fixed order (one block)
__global__ void __launch_bounds__(1024) k_zf_reduce(const double* __restrict__ partial, int nb, double* result)
{
    __shared__ double s_ss[32], s_mx[32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    double t = 0.0, mm = 0.0;
    for (int b = tid; b < nb; b += 1024) {
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
    if (tid == 0) {
        double u = 0.0, v = 0.0;
        for (int k = 0; k < 32; k++) {
            u += s_ss[k];
            v = fmax(v, s_mx[k]);
        }
        result[0] = u;
        result[1] = v;
    }
}

}  // namespace

template <typename T>
cudaError_t zfilter_commit(const ZfArgs<T>& a, cudaStream_t st)
{
    if (!zfilter_supported(a.D, a.max_partials)) return cudaErrorNotSupported;
    const dim3 blk = zf_block(a.D), grd = zf_grid(a.D);
    k_zf_fwd<T><<<grd, blk, 0, st>>>(a);
    k_zf_bwd<T><<<grd, blk, 0, st>>>(a);
    k_zf_reduce<<<1, 1024, 0, st>>>(a.partial, (int)(grd.x * grd.y), a.result);
    return cudaGetLastError();
}

template cudaError_t zfilter_commit<float>(const ZfArgs<float>&, cudaStream_t);
template cudaError_t zfilter_commit<double>(const ZfArgs<double>&, cudaStream_t);

}  // namespace wd
