// wd_probe.cu -- arithmetic-rate probe: the FP64 and FP32 fused multiply-add throughput of
// the current GPU, measured with a kernel of independent FMA chains.  The solver's FP64 form
// is classed as ALU-bound or not against this rate, not against a data-sheet figure.
#include "wd_api_internal.h"

namespace {

constexpr int PROBE_CHAINS = 8;     // independent dependency chains per thread
constexpr int PROBE_THREADS = 256;

// Every thread runs PROBE_CHAINS chains x <- a x + b, iters steps each (2 flops per step);
// the chains contract towards b / (1 - a), so the values stay finite for any iters.  The
// sum of the chains is stored so that no chain can be removed.
template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(T* out, int iters, T a, T b)
{
    T x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) x[c] = T(threadIdx.x) * T(1e-3) + T(c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; c++) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) s += x[c];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
wd_status run_probe(int iters, double* tflops, double* ms_out)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return wd::cuda_error(e, "fma probe: device query");
    const int blocks = sms * 8;
    T* out = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * PROBE_THREADS * sizeof(T));
    if (e != cudaSuccess) return wd::cuda_error(e, "fma probe: buffer");
    cudaEvent_t ev[2] = {nullptr, nullptr};
    float ms = 0.f;
    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) {
        k_fma_probe<T><<<blocks, PROBE_THREADS>>>(out, iters, T(0.9999), T(1e-4));   // warm-up
        cudaEventRecord(ev[0]);
        k_fma_probe<T><<<blocks, PROBE_THREADS>>>(out, iters, T(0.9999), T(1e-4));
        cudaEventRecord(ev[1]);
        e = cudaEventSynchronize(ev[1]);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(out);
    if (e != cudaSuccess) return wd::cuda_error(e, "fma probe");
    const double flops = 2.0 * PROBE_CHAINS * (double)iters * blocks * PROBE_THREADS;
    if (tflops) *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    if (ms_out) *ms_out = ms;
    return WD_OK;
}

}  // namespace

extern "C" wd_status wd_fma_probe(int precision, int iters, double* tflops, double* ms)
{
    if (iters < 1 || iters > (1 << 24) || (precision != WD_FP64 && precision != WD_FP32))
        return wd::set_error(WD_ERR_INVALID_ARG, "wd_fma_probe: precision WD_FP64 or WD_FP32, 1 <= iters <= 2^24");
    return precision == WD_FP64 ? run_probe<double>(iters, tflops, ms) : run_probe<float>(iters, tflops, ms);
}
