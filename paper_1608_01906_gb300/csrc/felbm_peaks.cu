// Arithmetic peaks of the current GPU, measured: every thread runs kChains
// independent FMA chains for a fixed number of iterations (no memory traffic
// inside the loop), one full-occupancy launch timed with CUDA events.  These
// are the ALU ceilings the step kernels are compared with; the step kernels
// do not use this file.
#include <cuda_runtime.h>

#include "felbm_internal.h"

namespace felbm {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, T b, T c, T *out) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == T(-1)) out[0] = s;  // never true for the arguments used; keeps the chains live
}

// Packed two-wide FP32 (FFMA2): each instruction is two FMAs.
__global__ void __launch_bounds__(kPeakThreads) k_ffma2_peak(int iters, float2 b, float2 c, float2 *out) {
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    if (s == -1.0f) out[0] = make_float2(s, s);
}

}  // namespace felbm

using namespace felbm;

extern "C" int felbm_alu_peak(int kind, double *flops_per_s) {
    if (!flops_per_s || kind < 0 || kind > 2) return FELBM_ERR_INVALID_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess) return cuda_status(e);
    const unsigned blocks = (unsigned)sms * (unsigned)(per_sm / kPeakThreads);
    // about 20 G FMA per launch in FP32, 1/16 of that in FP64 (a few ms each)
    const int iters = kind == 2 ? 512 : 8192;
    void *out = nullptr;
    e = cudaMalloc(&out, 16);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(t0, 0);
        if (kind == 0)
            k_fma_peak<float><<<blocks, kPeakThreads>>>(iters, 0.999999f, 1e-3f, (float *)out);
        else if (kind == 1)
            k_ffma2_peak<<<blocks, kPeakThreads>>>(iters / 2, make_float2(0.999999f, 0.999999f),
                                                   make_float2(1e-3f, 1e-3f), (float2 *)out);
        else
            k_fma_peak<double><<<blocks, kPeakThreads>>>(iters, 0.999999, 1e-3, (double *)out);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(t1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return cuda_status(e);
    // FFMA2 runs iters / 2 iterations of two FMAs per chain: the same count
    const double fmas = (double)blocks * kPeakThreads * kChains * (double)iters;
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
    return FELBM_OK;
}
