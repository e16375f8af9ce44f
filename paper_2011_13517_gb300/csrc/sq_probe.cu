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

// Warp-level tensor-core MMA (mma.sync) chains: 8 independent accumulator tiles per warp, the inputs
// held in registers, at full occupancy on every SM.  kind 0: TF32 m16n8k8 (2048 FLOP per instruction),
// kind 1: BF16 m16n8k16 (4096 FLOP).  These are the warp-level tensor instructions a per-warp
// mode-product contraction of the projector term could use.
template <int KIND>
__global__ void __launch_bounds__(kProbeBlock) k_mma_chains(unsigned a0, unsigned b0, int iters, float *sink)
{
    float acc[8][4];
#pragma unroll
    for (int t = 0; t < 8; t++)
#pragma unroll
        for (int i = 0; i < 4; i++) acc[t][i] = 0.f;
    const unsigned a1 = a0 ^ threadIdx.x, a2 = a0 + 3u, a3 = a0 ^ 0x00010001u, b1 = b0 ^ 5u;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int t = 0; t < 8; t++) {
            if (KIND == 0)
                asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                             "{%0,%1,%2,%3};"
                             : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                             : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            else
                asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                             "{%8,%9}, {%0,%1,%2,%3};"
                             : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                             : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < 8; t++) s += acc[t][0] + acc[t][1] + acc[t][2] + acc[t][3];
    if (s == -1.0f) sink[blockIdx.x] = s;
}

template <int KIND>
sq_status run_mma(double *tflops, double *ms_out, cudaStream_t stream)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SQ_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mma_chains<KIND>, kProbeBlock, 0) != cudaSuccess ||
        per_sm < 1)
        return SQ_ERR_CUDA;
    const int grid = sms * per_sm;
    // small exponents: the TF32 / BF16 operands stay finite in every chain
    const unsigned a0 = KIND == 0 ? 0x3c000000u : 0x3c003c00u, b0 = KIND == 0 ? 0x3b800000u : 0x3b803b80u;
    auto timed = [&](int iters, float *ms) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return cudaErrorUnknown;
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return cudaErrorUnknown;
        }
        cudaEventRecord(e0, stream);
        k_mma_chains<KIND><<<grid, kProbeBlock, 0, stream>>>(a0, b0, iters, nullptr);
        cudaError_t e = cudaGetLastError();
        cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return e;
    };
    float ms = 0.f;
    int iters = 200;
    if (timed(iters, &ms) != cudaSuccess) return SQ_ERR_CUDA;
    if (ms > 0.f) {
        const double scale = 100.0 / ms;
        const double want = iters * (scale > 1000.0 ? 1000.0 : scale);
        iters = want < 1.0 ? 1 : (want > 2e8 ? 200000000 : (int)want);
    }
    if (timed(iters, &ms) != cudaSuccess) return SQ_ERR_CUDA;
    if (timed(iters, &ms) != cudaSuccess) return SQ_ERR_CUDA;
    const double per = KIND == 0 ? 2.0 * 16 * 8 * 8 : 2.0 * 16 * 8 * 16;
    const double flops = per * 8.0 * (double)iters * (double)grid * (kProbeBlock / 32);
    if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return SQ_OK;
}

}  // namespace

extern "C" sq_status sq_mma_throughput(int kind, double *tflops, double *ms, void *stream)
{
    if (kind != 0 && kind != 1) return SQ_ERR_ARG;
    sq::count_launches(3);
    return kind == 0 ? run_mma<0>(tflops, ms, (cudaStream_t)stream) : run_mma<1>(tflops, ms, (cudaStream_t)stream);
}

extern "C" sq_status sq_fma_throughput(int precision, double *tflops, double *ms, void *stream)
{
    if (precision != SQ_FP64 && precision != SQ_FP32) return SQ_ERR_ARG;
    sq::count_launches(3);
    return precision == SQ_FP64 ? run<double>(tflops, ms, (cudaStream_t)stream)
                                : run<float>(tflops, ms, (cudaStream_t)stream);
}
