// Gauss spectral quadrature (Sec. 2.2 "Spectral Gauss quadrature"): the Lanczos iteration of every
// column (Eq. Lanczos) and the Gauss nodes and weights from each column's Jacobi matrix.
//
//   lanczos_kernel   the generic column machinery of sq_column.cuh in its Lanczos mode: per column
//                    K operator applications with two CTA reductions each, writing a_1..a_K and
//                    b_1..b_K (FP64) of the scaled truncated operator;
//   k_gauss_rule     one thread per column: eigenvalues of the K x K Jacobi matrix and the squared
//                    first components of its normalised eigenvectors, by implicit symmetric QR
//                    sweeps with the Wilkinson shift that carry only the first row of the
//                    accumulated rotations (the weights need nothing else).  The nodes come back in
//                    the unscaled energy, lambda = tau lambda_hat + omega.
#include <cuda_runtime.h>

#include <cmath>

#include "sq_column.cuh"
#include "sq_gauss_rule.h"

namespace sq {
namespace {

template <typename T, int P, int BLOCK, bool VSMEM>
__global__ void __launch_bounds__(BLOCK, BLOCK == 256 ? 2 : 1) lanczos_kernel(const RecursionArgs<T> args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    column_range<T, P, BLOCK, VSMEM, false, true>(args, args.q0 + blockIdx.x, args.q1, gridDim.x, smem_raw,
                                                  VSMEM ? nullptr : args.scratch + (size_t)blockIdx.x * 2 * args.nc3);
}

template <typename T, int P, int BLOCK, bool VSMEM>
cudaError_t lanczos_cfg(const RecursionArgs<T> &args, int grid, size_t smem, cudaStream_t stream)
{
    auto kern = lanczos_kernel<T, P, BLOCK, VSMEM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, BLOCK, smem, stream>>>(args);
    return cudaGetLastError();
}

template <typename T, int P, int BLOCK, bool VSMEM>
int lanczos_blocks_cfg(size_t smem)
{
    auto kern = lanczos_kernel<T, P, BLOCK, VSMEM>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, BLOCK, smem) != cudaSuccess) return 0;
    return n;
}

template <typename T, int P>
cudaError_t lanczos_p(const RecursionArgs<T> &args, int grid, int block, size_t smem, cudaStream_t stream)
{
    if (args.vec_in_smem) return block == 512 ? lanczos_cfg<T, P, 512, true>(args, grid, smem, stream)
                                             : lanczos_cfg<T, P, 256, true>(args, grid, smem, stream);
    return lanczos_cfg<T, P, 256, false>(args, grid, smem, stream);
}

template <typename T, int P>
int lanczos_blocks_p(int block, size_t smem, int vec_in_smem)
{
    if (vec_in_smem)
        return block == 512 ? lanczos_blocks_cfg<T, P, 512, true>(smem) : lanczos_blocks_cfg<T, P, 256, true>(smem);
    return lanczos_blocks_cfg<T, P, 256, false>(smem);
}

// Per column: Jacobi matrix from ab, Gauss rule, nodes and weights in the [K][N_d] layout.  The
// eigensolve works on local copies (K <= kGaussMaxK).
__global__ void k_gauss_rule(const double *ab, long long N_d, long long q0, long long q1, int K, double omega,
                             double tau, double *nodes, double *weights, int *bad)
{
    double d[kGaussMaxK], e[kGaussMaxK], z[kGaussMaxK];
    for (long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; q < q1;
         q += (long long)gridDim.x * blockDim.x) {
        for (int k = 0; k < K; k++) {
            d[k] = ab[(size_t)k * N_d + q];
            e[k] = ab[(size_t)(K + k) * N_d + q];
        }
        const int n = gauss_rule_inplace(d, e, z, K);
        if (n < 0) atomicExch(bad, 1);
        const int nn = n < 0 ? -n : n;
        for (int k = 0; k < K; k++) {
            nodes[(size_t)k * N_d + q] = k < nn ? tau * d[k] + omega : omega;
            weights[(size_t)k * N_d + q] = k < nn ? z[k] * z[k] : 0.0;
        }
    }
}

}  // namespace

#define SQ_DISPATCH_P(FN, ...)                         \
    switch (fd_half) {                                 \
    case 1: return FN<T, 1>(__VA_ARGS__);              \
    case 2: return FN<T, 2>(__VA_ARGS__);              \
    case 3: return FN<T, 3>(__VA_ARGS__);              \
    case 4: return FN<T, 4>(__VA_ARGS__);              \
    case 5: return FN<T, 5>(__VA_ARGS__);              \
    case 6: return FN<T, 6>(__VA_ARGS__);              \
    case 7: return FN<T, 7>(__VA_ARGS__);              \
    case 8: return FN<T, 8>(__VA_ARGS__);              \
    default: break;                                    \
    }

template <typename T>
cudaError_t launch_lanczos(const RecursionArgs<T> &args, int fd_half, int grid, int block, size_t smem,
                           cudaStream_t stream)
{
    SQ_DISPATCH_P(lanczos_p, args, grid, block, smem, stream)
    return cudaErrorInvalidValue;
}

template <typename T>
int lanczos_blocks_per_sm(int fd_half, int block, size_t smem, int vec_in_smem)
{
    SQ_DISPATCH_P(lanczos_blocks_p, block, smem, vec_in_smem)
    return 0;
}

template cudaError_t launch_lanczos<double>(const RecursionArgs<double> &, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_lanczos<float>(const RecursionArgs<float> &, int, int, int, size_t, cudaStream_t);
template int lanczos_blocks_per_sm<double>(int, int, size_t, int);
template int lanczos_blocks_per_sm<float>(int, int, size_t, int);

cudaError_t launch_gauss_rule(const double *ab, long long N_d, long long q0, long long q1, int K, double omega,
                              double tau, double *nodes, double *weights, int *bad, int num_sms, cudaStream_t stream)
{
    if (K < 1 || K > kGaussMaxK) return cudaErrorInvalidValue;
    const long long n = q1 - q0;
    long long grid = (n + 127) / 128;
    if (grid > (long long)num_sms * 16) grid = (long long)num_sms * 16;
    if (grid < 1) grid = 1;
    k_gauss_rule<<<(int)grid, 128, 0, stream>>>(ab, N_d, q0, q1, K, omega, tau, nodes, weights, bad);
    return cudaGetLastError();
}

}  // namespace sq
