// Measured FMA-pipe ceilings of the current GPU, for the roofline of the recursion kernels (which are
// bound by FP32 or FP64 fused multiply-adds, not by memory).
//
// The probe kernel runs 8 independent FMA chains per thread at full occupancy on every SM; its FLOP
// count divided by its CUDA-event time is the attainable FMA rate at the clocks of the run.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdarg>

#include "sq_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kProbeBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeBlock) k_fma_chains(T a, T b, int iters, T *sink)
{
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int i = 0; i < kChains; i++) x[i] = fma(x[i], a, b);
        }
    }
    T s = (T)0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += x[i];
    // never true for the arguments the host passes; keeps the chains from being removed
    if (s == (T)-1.0) sink[blockIdx.x] = s;
}

template <typename T>
cudaError_t probe(int iters, int grid, cudaStream_t stream, float *ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    cudaEventRecord(e0, stream);
    k_fma_chains<T><<<grid, kProbeBlock, 0, stream>>>((T)0.999999, (T)1e-7, iters, nullptr);
    e = cudaGetLastError();
    cudaEventRecord(e1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

template <typename T>
sq_status run(double *tflops, double *ms_out, cudaStream_t stream)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SQ_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, kProbeBlock, 0) != cudaSuccess ||
        per_sm < 1)
        return SQ_ERR_CUDA;
    const int grid = sms * per_sm;
    float ms = 0.f;
    // calibrate on a short run, then time a run of about 100 ms (after one untimed warm-up)
    int iters = sizeof(T) == 4 ? 2000 : 50;
    if (probe<T>(iters, grid, stream, &ms) != cudaSuccess) return SQ_ERR_CUDA;
    if (ms > 0.f) {
        const double scale = 100.0 / ms;
        const double want = iters * (scale > 200.0 ? 200.0 : scale);
        iters = want < 1.0 ? 1 : (want > 2e8 ? 200000000 : (int)want);
    }
    if (probe<T>(iters, grid, stream, &ms) != cudaSuccess) return SQ_ERR_CUDA;
    if (probe<T>(iters, grid, stream, &ms) != cudaSuccess) return SQ_ERR_CUDA;
    const double flops = 2.0 * kChains * kUnroll * (double)iters * (double)grid * kProbeBlock;
    if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return SQ_OK;
}

}  // namespace

extern "C" sq_status sq_fma_throughput(int precision, double *tflops, double *ms, void *stream)
{
    if (precision != SQ_FP64 && precision != SQ_FP32) return SQ_ERR_ARG;
    sq::count_launches(3);
    return precision == SQ_FP64 ? run<double>(tflops, ms, (cudaStream_t)stream)
                                : run<float>(tflops, ms, (cudaStream_t)stream);
}
