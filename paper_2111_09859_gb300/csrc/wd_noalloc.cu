// wd_noalloc.cu -- change norms of two state arrays without any device allocation.
//
// The same reduction as the solver's change-norm kernel (RMS and max of new - old over the
// nodes whose mask byte is 0, accumulated in double with a fixed block partition and a
// fixed final order), but its scratch (the per-block partial sums and the arrival
// counter) lives in the file-scope array below, so a call allocates nothing.  It serves
// callers that cannot allocate device memory: an application whose own memory pool has
// already taken the device memory, or a real-time loop that must not call the allocator
// (cudaMalloc / cudaFree can synchronise the device).  The paper has no counterpart.
//
// The array's device address is looked up once per device, on the first call with that
// device current, and kept for the process; a cudaDeviceReset invalidates it, so the entry
// point is not for use on a device after a reset.
#include <mutex>

#include "wd_api_internal.h"

namespace {

constexpr int NA_BLOCKS = 1024;          // at most this many blocks share the scratch
constexpr int NA_THREADS = 256;
constexpr long long NA_MAX_N = 1LL << 30;
// [0, 32): arrival counter (first 4 bytes); then 3 doubles per block (sum of squares,
// max |change|, count)
constexpr int NA_DOUBLES = 32 + 3 * NA_BLOCKS;

// One copy per GPU that loads the library, kept until the process exits (about 25 KB).
// Every call on a device shares it and finds the previous call's contents.
static __device__ __align__(256) double g_na_scratch[NA_DOUBLES];

std::mutex g_na_mutex;
double* g_na_ptr[64] = {};   // device address of g_na_scratch, per device

template <typename T>
__global__ void k_norms_noalloc(const T* __restrict__ a, const T* __restrict__ b,
                                const uint8_t* __restrict__ mask, long long n, double inv_scale,
                                double* scratch, double* out)
{
    __shared__ double s_ss[NA_THREADS / 32], s_mx[NA_THREADS / 32], s_ct[NA_THREADS / 32];
    __shared__ int s_last;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch);
    double* part = scratch + 32;
    double ss = 0.0, mx = 0.0, ct = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        if (mask && mask[e]) continue;
        const double d = double(a[e]) - double(b[e]);
        ss += d * d;
        mx = fmax(mx, fabs(d));
        ct += 1.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        ct += __shfl_down_sync(0xffffffffu, ct, o);
    }
    if (lane == 0) {
        s_ss[wid] = ss;
        s_mx[wid] = mx;
        s_ct[wid] = ct;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, m = 0.0, c = 0.0;
        for (int w = 0; w < nw; w++) {
            t += s_ss[w];
            m = fmax(m, s_mx[w]);
            c += s_ct[w];
        }
        part[3 * blockIdx.x] = t;
        part[3 * blockIdx.x + 1] = m;
        part[3 * blockIdx.x + 2] = c;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    double t = 0.0, m = 0.0, c = 0.0;
    for (int k = 0; k < (int)gridDim.x; k++) {
        t += __ldcg(part + 3 * k);
        m = fmax(m, __ldcg(part + 3 * k + 1));
        c += __ldcg(part + 3 * k + 2);
    }
    out[0] = c > 0.0 ? sqrt(t / c) * inv_scale : 0.0;
    out[1] = m * inv_scale;
    *counter = 0u;
}

// device address of the scratch array on the current device (set up once per device)
wd_status scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return wd::cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return wd::set_error(WD_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return wd::cuda_error(e, "cudaGetSymbolAddress(g_na_scratch)");
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
    return WD_OK;
}

}  // namespace

extern "C" wd_status wd_change_norms_noalloc(const void* new_dev, const void* old_dev,
                                             const uint8_t* mask_dev, long long n, int precision,
                                             double scale, double* norms_dev, void* cuda_stream)
{
    if (!new_dev || !old_dev || !norms_dev)
        return wd::set_error(WD_ERR_INVALID_ARG, "wd_change_norms_noalloc: NULL array");
    if (n < 1 || n > NA_MAX_N)
        return wd::set_error(WD_ERR_INVALID_ARG,
                             "wd_change_norms_noalloc: n must be in [1, 2^30] (the maximum size)");
    if (precision < WD_FP64 || precision > WD_FP32)
        return wd::set_error(WD_ERR_INVALID_ARG, "wd_change_norms_noalloc: bad precision");
    if (!(scale > 0.0)) return wd::set_error(WD_ERR_INVALID_ARG, "wd_change_norms_noalloc: scale must be > 0");
    double* scratch = nullptr;
    wd_status s = scratch_address(&scratch);
    if (s != WD_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the arrival counter must start at zero whatever the previous call left
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return wd::cuda_error(e, "wd_change_norms_noalloc: counter reset");
    long long nb = (n + NA_THREADS - 1) / NA_THREADS;
    int blocks = (int)(nb < NA_BLOCKS ? nb : NA_BLOCKS);
    if (precision == WD_FP64)
        k_norms_noalloc<double><<<blocks, NA_THREADS, 0, st>>>(
            (const double*)new_dev, (const double*)old_dev, mask_dev, n, 1.0 / scale, scratch, norms_dev);
    else
        k_norms_noalloc<float><<<blocks, NA_THREADS, 0, st>>>(
            (const float*)new_dev, (const float*)old_dev, mask_dev, n, 1.0 / scale, scratch, norms_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return wd::cuda_error(e, "wd_change_norms_noalloc: launch");
    return WD_OK;
}
