// dgk_peak.cu -- the arithmetic peak the FP64 form is measured against: a fused
// multiply-add throughput kernel in double (or float), timed with CUDA events.
//
// Each thread runs kChains independent FMA chains (enough independent work to cover the
// pipe latency), kIters times; the grid fills every SM several times over.  The chains'
// operands come from the kernel arguments and the results are stored, so nothing can be
// folded away.  Flops = 2 per FMA.
#include <cuda_runtime.h>

#include "dgk.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T a, T b, int iters, T *out)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(int device, int iters, double *flops_per_s)
{
    if (cudaSetDevice(device) != cudaSuccess) return DGK_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return DGK_ERR_CUDA;
    const int blocks = prop.multiProcessorCount * 8;
    T *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(T)) != cudaSuccess) return DGK_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a = 1 - 2^-20, b = 2^-20: the chains stay finite and away from denormals
    const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1048576.0);
    k_fma_peak<T><<<blocks, kThreads>>>(a, b, iters / 4 + 1, out);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        k_fma_peak<T><<<blocks, kThreads>>>(a, b, iters, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return DGK_ERR_CUDA;
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *flops_per_s = flops / (best * 1e-3);
    return DGK_OK;
}

}  // namespace

extern "C" int dgk_fma_peak(int device, int precision, double *flops_per_s)
{
    if (!flops_per_s || (precision != DGK_PREC_FP64 && precision != DGK_PREC_FP32BULK)) return DGK_ERR_ARG;
    // about 0.25 s (FP64) and 0.13 s (FP32) per timed launch on a GB300
    return precision == DGK_PREC_FP64 ? measure<double>(device, 64, flops_per_s)
                                      : measure<float>(device, 2048, flops_per_s);
}
