// peak.cu -- measured CUDA-core arithmetic peaks (FP32 FFMA, FP64 DFMA) of the current
// device, the denominators of the "alu" rooflines of the CUDA-core kernels (the plain
// level products, the leaves, the batched kernel, the FP64 path).
//
// Every thread runs 8 independent dependent chains x <- x * a + b (one fused multiply-add
// each, 2 flops); a and b are kernel arguments, so nothing folds at compile time, and
// the chains' sum is stored so nothing is dropped.  The grid holds `blocks_per_sm` CTAs
// of 512 threads per SM, enough warps to hide the FMA latency on every sub-partition.
// The launch is timed with CUDA events on a private stream after one warm-up launch.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace triinv {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T *out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
tri_status time_chain(int sms, int blocks_per_sm, int iters, double *tflops, double *ms_out) {
    const int blocks = sms * blocks_per_sm;
    T *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tri_status st = TRI_ERR_CUDA;
    float ms = 0.f;
    if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) return TRI_ERR_NOMEM;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        const T a = T(0.999999), b = T(1e-6);
        fma_chain_kernel<T><<<blocks, kThreads, 0, s>>>(out, iters / 8, a, b);   // warm-up
        cudaEventRecord(e0, s);
        fma_chain_kernel<T><<<blocks, kThreads, 0, s>>>(out, iters, a, b);
        cudaEventRecord(e1, s);
        if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
            const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
            *tflops = flops / (ms * 1e-3) / 1e12;
            if (ms_out) *ms_out = ms;
            st = TRI_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    return st;
}

}  // namespace
}  // namespace triinv

extern "C" tri_status tri_alu_peak(tri_dtype dtype, int iters, double *tflops, double *ms) {
    using namespace triinv;
    if (!tflops || iters < 8 || (dtype != TRI_F32 && dtype != TRI_F64)) return TRI_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TRI_ERR_CUDA;
    // FP32: 4 CTAs of 512 threads per SM (64 warps); FP64: 2 per SM, its pipe is narrow
    return dtype == TRI_F32 ? time_chain<float>(sms, 4, iters, tflops, ms)
                            : time_chain<double>(sms, 2, iters, tflops, ms);
}
