// Allocation-free variant of the FP64 mass / momentum reduction.
//
// felbm_totals_nalloc computes the same totals as felbm_moments_get
// (sum w rho, sum w rho ux, sum w rho uy with FP64 accumulation) over device
// arrays the caller owns.  It exists for callers whose device memory belongs
// to another allocator -- a framework's caching allocator, or an arena sized
// once at start-up -- and who therefore must not let this library call
// cudaMalloc.  Its scratch (the per-block partial sums) is a file-scope
// device array of fixed size that every GPU loading the library holds until
// the process exits.
#include <mutex>

#include "felbm_internal.h"

namespace {

constexpr int kNaBlocks = 1024;         // partial-sum slots (blocks of the first pass)
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

// Scratch shared by every call on a device: 3 partial sums per block.
static __device__ __align__(256) double g_na_partials[3 * kNaBlocks];

double *g_na_addr[kNaMaxDevices];
cudaError_t g_na_err[kNaMaxDevices];
std::once_flag g_na_once[kNaMaxDevices];

template <typename T>
__global__ void __launch_bounds__(kNaThreads) k_na_partial(int64_t n, const T *__restrict__ rho,
                                                           const T *__restrict__ ux,
                                                           const T *__restrict__ uy,
                                                           const double *__restrict__ w,
                                                           double *__restrict__ part) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double mr = (w ? w[i] : 1.0) * (double)rho[i];
        s0 += mr;
        s1 += mr * (double)ux[i];
        s2 += mr * (double)uy[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    __shared__ double sh[3][kNaThreads / 32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][wid] = s0;
        sh[1][wid] = s1;
        sh[2][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (int k = 0; k < kNaThreads / 32; ++k) {
            t0 += sh[0][k];
            t1 += sh[1][k];
            t2 += sh[2][k];
        }
        part[3 * blockIdx.x] = t0;
        part[3 * blockIdx.x + 1] = t1;
        part[3 * blockIdx.x + 2] = t2;
    }
}

__global__ void k_na_final(int nparts, const double *__restrict__ part, double *__restrict__ out) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = threadIdx.x; k < nparts; k += 32) {
        s0 += part[3 * k];
        s1 += part[3 * k + 1];
        s2 += part[3 * k + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (threadIdx.x == 0) {
        out[0] = s0;
        out[1] = s1;
        out[2] = s2;
    }
}

}  // namespace

extern "C" int felbm_totals_nalloc(const void *rho, const void *ux, const void *uy,
                                   const double *weight, int64_t n, int32_t precision,
                                   double *totals, void *stream) {
    if (!rho || !ux || !uy || !totals) return FELBM_ERR_INVALID_ARG;
    if (n < 1 || n > FELBM_NALLOC_MAX_NODES) return FELBM_ERR_INVALID_ARG;
    if (precision != FELBM_FP64 && precision != FELBM_FP32) return FELBM_ERR_INVALID_ARG;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return FELBM_ERR_CUDA;
    if (dev < 0 || dev >= kNaMaxDevices) return FELBM_ERR_UNSUPPORTED;
    // Once per device, with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in for it).
    std::call_once(g_na_once[dev], [dev]() {
        g_na_err[dev] = cudaGetSymbolAddress(reinterpret_cast<void **>(&g_na_addr[dev]),
                                             g_na_partials);
    });
    if (g_na_err[dev] != cudaSuccess || !g_na_addr[dev]) return FELBM_ERR_CUDA;
    double *part = g_na_addr[dev];
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t want = (n + kNaThreads - 1) / kNaThreads;
    const int blocks = (int)(want < kNaBlocks ? want : kNaBlocks);
    // every slot the final pass reads is written by the first pass of the
    // same call, so nothing needs clearing
    if (precision == FELBM_FP64)
        k_na_partial<double><<<blocks, kNaThreads, 0, st>>>(
            n, static_cast<const double *>(rho), static_cast<const double *>(ux),
            static_cast<const double *>(uy), weight, part);
    else
        k_na_partial<float><<<blocks, kNaThreads, 0, st>>>(
            n, static_cast<const float *>(rho), static_cast<const float *>(ux),
            static_cast<const float *>(uy), weight, part);
    k_na_final<<<1, 32, 0, st>>>(blocks, part, totals);
    e = cudaGetLastError();
    return e == cudaSuccess ? FELBM_OK : FELBM_ERR_CUDA;
}
