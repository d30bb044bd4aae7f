// wd_unsteady.cu -- receding-surface update (Sec. 5.5) and the length of a level set of a
// 2-D field (the burning perimeter).
#include "wd_api_internal.h"

namespace wd {

// surface receded by s: phi <- phi - s (the distance to the receded surface, and the warm
// start of the next solve); the burned set {phi <= 0} becomes Dirichlet with that value,
// floored at `floor`; every other node is released (dense arrays of n)
template <typename T>
__global__ void k_recede(T* __restrict__ phi, long long n, double s, double floor,
                         uint8_t* __restrict__ mask, T* __restrict__ dval)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const T v = phi[q] - T(s);
        phi[q] = v;
        const bool burned = v <= T(0);
        mask[q] = burned;
        dval[q] = burned ? (v < T(floor) ? T(floor) : v) : T(0);
    }
}

template <typename T>
cudaError_t launch_recede(T* phi, long long n, double s, double floor, uint8_t* mask, T* dval,
                          cudaStream_t st)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    k_recede<T><<<(int)(b < 1 ? 1 : b), 256, 0, st>>>(phi, n, s, floor, mask, dval);
    return cudaGetLastError();
}

// crossing of the zero level on the edge a-b of a cell (values va, vb of opposite sign)
__device__ __forceinline__ void cross(double va, double vb, double xa, double ya, double xb, double yb,
                                      double& x, double& y)
{
    const double t = va / (va - vb);
    x = xa + t * (xb - xa);
    y = ya + t * (yb - ya);
}

struct Period2 {
    double p[2][2];   // shift of (x, y) across the wrap of direction d
};

// marching squares over the cells of a 2-D grid: phi dense (n0 x n1, i fastest), xyz padded
// (pitch); a periodic direction adds the wrap cells (node n-1 to node 0, whose coordinates
// are shifted by the period); each block writes the FP64 sum of its cells' segment lengths
// to part[blockIdx.x]
template <typename T>
__global__ void __launch_bounds__(256) k_level_length(Dims D, const T* __restrict__ phi,
                                                      const double* __restrict__ xyz, Period2 per,
                                                      double level, double* part)
{
    const int n0 = D.n[0], n1 = D.n[1];
    const int c0 = n0 - !D.per[0], c1 = n1 - !D.per[1];
    const long long cells = (long long)c0 * c1;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % c0), j = (int)(c / c0);
        const int i1 = i + 1 == n0 ? 0 : i + 1, j1 = j + 1 == n1 ? 0 : j + 1;
        // corners 0 (i, j), 1 (i+1, j), 2 (i+1, j+1), 3 (i, j+1)
        const int ci[4] = {i, i1, i1, i};
        const int cj[4] = {j, j, j1, j1};
        const int wi[4] = {0, i1 < i, i1 < i, 0};
        const int wj[4] = {0, 0, j1 < j, j1 < j};
        double v[4], X[4], Y[4];
        int neg = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[k] = (double)phi[(long long)cj[k] * n0 + ci[k]] - level;
            const long long e = (long long)cj[k] * D.pitch + ci[k];
            X[k] = xyz[e] + wi[k] * per.p[0][0] + wj[k] * per.p[1][0];
            Y[k] = xyz[D.total + e] + wi[k] * per.p[0][1] + wj[k] * per.p[1][1];
            neg |= (v[k] < 0.0) << k;
        }
        if (neg == 0 || neg == 15) continue;
        // crossing points on edges k = (k, k+1)
        double px[4], py[4];
        int has[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int a = k, b = (k + 1) & 3;
            has[k] = ((neg >> a) & 1) != ((neg >> b) & 1);
            if (has[k]) cross(v[a], v[b], X[a], Y[a], X[b], Y[b], px[k], py[k]);
        }
        const int nc = has[0] + has[1] + has[2] + has[3];
        if (nc == 2) {
            int e0 = -1, e1 = -1;
            for (int k = 0; k < 4; k++)
                if (has[k]) {
                    if (e0 < 0) e0 = k;
                    else e1 = k;
                }
            acc += hypot(px[e1] - px[e0], py[e1] - py[e0]);
        } else {
            // saddle: the centre value (mean of the corners) decides which corners the
            // level set cuts off
            const double ctr = 0.25 * (v[0] + v[1] + v[2] + v[3]);
            if ((ctr < 0.0) == (v[0] < 0.0)) {
                // corners 1 and 3 are cut off: edges (0, 1) and (2, 3)
                acc += hypot(px[1] - px[0], py[1] - py[0]) + hypot(px[3] - px[2], py[3] - py[2]);
            } else {
                // corners 0 and 2 are cut off: edges (3, 0) and (1, 2)
                acc += hypot(px[0] - px[3], py[0] - py[3]) + hypot(px[2] - px[1], py[2] - py[1]);
            }
        }
    }
    // fixed-order block sum
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <typename T>
cudaError_t launch_level_length(const Dims& D, const T* phi, const double* xyz,
                                const double (*period)[3], double level, double* part, int nblocks,
                                cudaStream_t st)
{
    Period2 per;
    for (int d = 0; d < 2; d++)
        for (int m = 0; m < 2; m++) per.p[d][m] = D.per[d] ? period[d][m] : 0.0;
    k_level_length<T><<<nblocks, 256, 0, st>>>(D, phi, xyz, per, level, part);
    return cudaGetLastError();
}

template cudaError_t launch_recede<float>(float*, long long, double, double, uint8_t*, float*,
                                          cudaStream_t);
template cudaError_t launch_recede<double>(double*, long long, double, double, uint8_t*, double*,
                                           cudaStream_t);
template cudaError_t launch_level_length<float>(const Dims&, const float*, const double*,
                                                const double (*)[3], double, double*, int, cudaStream_t);
template cudaError_t launch_level_length<double>(const Dims&, const double*, const double*,
                                                 const double (*)[3], double, double*, int, cudaStream_t);

}  // namespace wd
