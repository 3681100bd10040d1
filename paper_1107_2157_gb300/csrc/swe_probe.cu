// swe_probe.cu -- arithmetic throughput probes: the measured peaks against
// which the library states the ALU fractions of its kernels (the stencil's
// FP32 lane operations, the FP64 path's FMAs).  Each probe runs independent
// FMA chains on every SM (enough warps and chains to hide the pipeline
// latency) and times itself with CUDA events; it changes no device setting.
#include "swe_device.cuh"

namespace swe {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;

// Written only if a chain ends on an exact sentinel value, which keeps the
// chains live without a store per thread.
static __device__ float g_probe_sink32;
static __device__ double g_probe_sink64;

// kind 0: scalar FP32 FMA; 1: packed f32x2 FMA (two lanes per instruction);
// 2: FP64 FMA.
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters)
{
    const float t = (float)(threadIdx.x & 7) * 1e-3f;
    if constexpr (KIND == 0) {
        float x[kProbeChains];
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = t + (float)k;
        const float a = 0.999f, b = 1e-4f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) x[k] = fmaf(x[k], a, b);
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) s += x[k];
        if (s == 12345.0f) g_probe_sink32 = s;
    } else if constexpr (KIND == 1) {
        F2 x[kProbeChains];
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = pack2(t + (float)k, t - (float)k);
        const F2 a = pack2(0.999f, 0.998f), b = pack2(1e-4f, 2e-4f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) x[k] = fma2(x[k], a, b);
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) s += lo2(x[k]) + hi2(x[k]);
        if (s == 12345.0f) g_probe_sink32 = s;
    } else {
        double x[kProbeChains];
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = (double)t + (double)k;
        const double a = 0.999, b = 1e-4;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], a, b);
        }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) s += x[k];
        if (s == 12345.0) g_probe_sink64 = s;
    }
}

}  // namespace swe

extern "C" swe_status swe_probe_rate(int kind, double *rate_out)
{
    using namespace swe;
    if (!rate_out || kind < 0 || kind > 2) return SWE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SWE_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SWE_ECUDA;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    swe_status st = SWE_ECUDA;
    const int blocks = sms * 8;                  // 64 warps per SM
    const int iters = kind == 2 ? 1024 : 65536;  // FP64 runs at a small fraction of the FP32 rate
    const double lanes = kind == 1 ? 2.0 : 1.0;  // FMAs per thread per instruction
    const double fmas = (double)blocks * kProbeThreads * kProbeChains * (double)iters * lanes;
    float ms = 0.0f;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SWE_ECUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    for (int rep = 0; rep < 3; ++rep) {  // the first launch warms up; the last is timed
        cudaEventRecord(e0, s);
        if (kind == 0) fma_probe_kernel<0><<<blocks, kProbeThreads, 0, s>>>(iters);
        else if (kind == 1) fma_probe_kernel<1><<<blocks, kProbeThreads, 0, s>>>(iters);
        else fma_probe_kernel<2><<<blocks, kProbeThreads, 0, s>>>(iters);
        cudaEventRecord(e1, s);
    }
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) goto done;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f)) goto done;
    *rate_out = fmas / ((double)ms * 1e-3);
    st = SWE_OK;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return st;
}
