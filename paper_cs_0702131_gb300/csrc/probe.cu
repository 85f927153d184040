// Measurement helper: the FMA rate of the device in FP32 or FP64, the
// denominator of the pair kernels' arithmetic rooflines.  Every thread runs
// eight independent multiply-add chains, so the FMA pipes, not latency,
// bound the launch.
#include <algorithm>

#include "aica_internal.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 8;
__device__ double g_probe_sink[4096];

template <class T>
__global__ void __launch_bounds__(kProbeThreads) fma_chains(int iters, T m, T c) {
    T v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = (T)(threadIdx.x + 8 * i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = fma(v[i], m, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += v[i];
    if (s == (T)-12345) g_probe_sink[blockIdx.x & 4095] = (double)s;   // keeps the chains live
}

}  // namespace

extern "C" aica_status aica_probe_fma_rate(int fp64, int64_t iters, double *flops_per_s, void *stream) {
    if (!flops_per_s) { aica::set_error("aica_probe_fma_rate: NULL output"); return AICA_ERR_INVALID_ARG; }
    if (iters < 1 || iters > (1ll << 30)) { aica::set_error("aica_probe_fma_rate: iters out of range"); return AICA_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    AICA_CUDA(cudaGetDevice(&dev));
    AICA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, sms) * kProbeBlocksPerSM;
    const int warm = (int)std::max<int64_t>(1, iters / 10);
    cudaEvent_t e0, e1;
    AICA_CUDA(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err != cudaSuccess) { cudaEventDestroy(e0); return aica::cuda_fail(err, "cudaEventCreate"); }
    auto launch = [&](int n) {
        if (fp64) fma_chains<double><<<grid, kProbeThreads, 0, st>>>(n, 0.9999999, 1e-9);
        else fma_chains<float><<<grid, kProbeThreads, 0, st>>>(n, 0.9999f, 1e-6f);
    };
    launch(warm);
    err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) launch((int)iters);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return aica::cuda_fail(err, "aica_probe_fma_rate");
    const double flops = 2.0 * 8.0 * (double)iters * (double)grid * (double)kProbeThreads;
    *flops_per_s = ms > 0.f ? flops / (ms * 1e-3) : 0.0;
    return AICA_OK;
}
