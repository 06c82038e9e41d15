// Arithmetic peaks of the device, measured: the roofline denominators of
// the kernels bound by FP32 or FP64 arithmetic (the FP64 hopping sweeps of
// the reliable updates, the SAP block solve, the network's transport).  The
// paper has no counterpart; its method needs none of this.
//
// Every thread runs CH independent multiply-add chains x <- x a + b (a < 1,
// so x stays bounded) for `iters` rounds; 2048 threads per SM keep the
// pipes' latency covered.  Flops = 2 per multiply-add and lane.
#include <cuda_runtime.h>

#include "internal.h"

namespace lqcd {

enum { PEAK_CH = 8, PEAK_BLOCK = 256, PEAK_BLOCKS_PER_SM = 8 };

// Written only if a chain's sum takes an impossible value (they converge to
// 1 each): the condition keeps the chains live without a buffer to write.
__device__ double g_peak_sink;

template <int KIND>
__global__ void __launch_bounds__(PEAK_BLOCK) fma_peak_kernel(int iters, float a32, float b32, double a64,
                                                             double b64)
{
    double out = 0.0;
    if constexpr (KIND == 0) {
        float x[PEAK_CH];
#pragma unroll
        for (int k = 0; k < PEAK_CH; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < PEAK_CH; ++k) x[k] = fmaf(x[k], a32, b32);
#pragma unroll
        for (int k = 0; k < PEAK_CH; ++k) out += x[k];
    } else if constexpr (KIND == 1) {
        float2 x[PEAK_CH];
        const float2 a = make_float2(a32, a32), b = make_float2(b32, b32);
#pragma unroll
        for (int k = 0; k < PEAK_CH; ++k) x[k] = make_float2(1e-3f * (float)(threadIdx.x + k), 2e-3f * (float)k);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < PEAK_CH; ++k) x[k] = __ffma2_rn(x[k], a, b);
#pragma unroll
        for (int k = 0; k < PEAK_CH; ++k) out += x[k].x + x[k].y;
    } else {
        double x[PEAK_CH];
#pragma unroll
        for (int k = 0; k < PEAK_CH; ++k) x[k] = 1e-3 * (double)(threadIdx.x + k);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < PEAK_CH; ++k) x[k] = fma(x[k], a64, b64);
#pragma unroll
        for (int k = 0; k < PEAK_CH; ++k) out += x[k];
    }
    if (out == -1.0) g_peak_sink = out;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_fma_peak(int device, int kind, double* tflops)
{
    if (!tflops) return fail(LQCD_ERR_INVALID, "lqcd_fma_peak: null result");
    if (kind < 0 || kind > 2) return fail(LQCD_ERR_INVALID, "lqcd_fma_peak: kind must be 0, 1 or 2");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(device));
    int sms = 0;
    LQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = sms * PEAK_BLOCKS_PER_SM;
    const long threads = (long)blocks * PEAK_BLOCK;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lqcd_status st = LQCD_OK;
    auto run = [&](int iters, float& ms) -> cudaError_t {
        cudaError_t e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) return e;
        switch (kind) {
        case 0: fma_peak_kernel<0><<<blocks, PEAK_BLOCK, 0, s>>>(iters, 0.9999999f, 1e-7f, 0.0, 0.0); break;
        case 1: fma_peak_kernel<1><<<blocks, PEAK_BLOCK, 0, s>>>(iters, 0.9999999f, 1e-7f, 0.0, 0.0); break;
        default: fma_peak_kernel<2><<<blocks, PEAK_BLOCK, 0, s>>>(iters, 0.f, 0.f, 0.99999999, 1e-8); break;
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        return e;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // size the timed launch to ~20 ms from a short one (the short one also warms up)
    int iters = kind == 2 ? 256 : 4096;
    float ms = 0.f;
    if (e == cudaSuccess) e = run(iters, ms);
    if (e == cudaSuccess) {
        const double scale = ms > 0.f ? 20.0 / ms : 1.0;
        const double want = (double)iters * (scale < 1.0 ? 1.0 : scale);
        iters = (int)(want < 1e8 ? want : 1e8);
        e = run(iters, ms);
    }
    if (e == cudaSuccess && ms > 0.f) {
        const double lanes = kind == 1 ? 2.0 : 1.0;  // a packed pair is two multiply-adds
        *tflops = 2.0 * lanes * PEAK_CH * (double)iters * (double)threads / (ms * 1e-3) / 1e12;
    } else if (e == cudaSuccess) {
        e = cudaErrorUnknown;
    }
    if (e != cudaSuccess) st = fail(LQCD_ERR_CUDA, std::string("lqcd_fma_peak: ") + cudaGetErrorString(e));
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    return st;
}
