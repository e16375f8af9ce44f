// Per-grid-point Chebyshev recursion of the truncated Kohn-Sham Hamiltonian (the SQ hot loop).
//
// For every grid point q (a "column"), with the cube C_q of half-width m around q and the scaled
// restricted operator Hhat_q = P_q (H - omega)/tau P_q (Sec. 3 "Hamiltonian at each grid point",
// Sec. 2.2 scale and shift), the kernel runs the three-term recursion of Eq. Chebyshev,
//     v_0 = e_q,  v_1 = Hhat_q v_0,  v_{k+1} = 2 Hhat_q v_k - v_{k-1},
// and records mu_k^q = v_k(q).  With force moments requested it also accumulates
//     A_k^{J,lm,d} += chi_Jlm(x_q) (d_d chi_Jlm)^T v_k        (Eq. NLforceSQ),
// for the atoms whose projectors are nonzero at x_q.
//
// Mapping: one CTA owns one column at a time (persistent loop over columns).  Each recursion step
// has two phases separated by CTA barriers:
//   phase 1  warp-per-atom projector contractions chi^T v_k.  The projectors are separable, so each
//            lane sums one x-row of the atom's support box against the 1D x factors and weights the
//            row with the y and z factors; a warp shuffle reduction gives the 4 s/p dots (and the
//            12 force dots for atoms that touch x_q).
//   phase 2  thread-per-x-segment update: the segment and its x halo are held in registers, the y
//            and z neighbours are read from the vector, the KB term is gathered from the atoms whose
//            support covers the row, and w = a Hhat v_k - b v_{k-1} overwrites v_{k-1} in place.
// The two cube vectors live in shared memory when they fit, else in a per-CTA global scratch slot.
#include <cuda_runtime.h>

#include "sq_internal.h"

#include "sq_column.cuh"

namespace sq {
namespace {

template <typename T, int P, int BLOCK, bool VSMEM>
__global__ void __launch_bounds__(BLOCK, BLOCK == 256 ? 2 : 1) recursion_kernel(const RecursionArgs<T> args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    column_range<T, P, BLOCK, VSMEM>(args, args.q0 + blockIdx.x, args.q1, gridDim.x, smem_raw,
                                     VSMEM ? nullptr : args.scratch + (size_t)blockIdx.x * 2 * args.nc3);
}

// Reverse-mode (vector-Jacobian) pass over all columns: vectors in per-CTA global scratch of
// 2 + 2 nseg + kc + 1 + 3 cube vectors.
template <typename T, int P>
__global__ void __launch_bounds__(256, 2) adjoint_kernel(const RecursionArgs<T> args, long long scratch_stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    column_range<T, P, 256, false, true>(args, args.q0 + blockIdx.x, args.q1, gridDim.x, smem_raw,
                                         args.scratch + (size_t)blockIdx.x * scratch_stride);
}

// Many cells in one persistent launch: each CTA takes (cell, column range) work items from a queue
// (one atomicAdd per item; no CTA ever waits on another) until the queue is empty.
template <typename T, int P, int BLOCK, bool VSMEM>
__global__ void __launch_bounds__(BLOCK, BLOCK == 256 ? 2 : 1)
    batch_kernel(const RecursionArgs<T> *cells, const BatchItem *items, int nitems, unsigned *counter, T *scratch,
                 long long scratch_stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = item_s;
        __syncthreads();
        if (it >= nitems) break;
        const BatchItem w = items[it];
        const RecursionArgs<T> a = cells[w.cell];
        column_range<T, P, BLOCK, VSMEM>(a, w.begin, w.end < a.N_d ? w.end : a.N_d, 1, smem_raw,
                                         VSMEM ? nullptr : scratch + (size_t)blockIdx.x * scratch_stride);
    }
}

template <typename T, int P, int BLOCK, bool VSMEM>
cudaError_t launch_cfg(const RecursionArgs<T> &args, int grid, size_t smem, cudaStream_t stream)
{
    auto kern = recursion_kernel<T, P, BLOCK, VSMEM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, BLOCK, smem, stream>>>(args);
    return cudaGetLastError();
}

template <typename T, int P, int BLOCK, bool VSMEM>
int blocks_cfg(size_t smem)
{
    auto kern = recursion_kernel<T, P, BLOCK, VSMEM>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, BLOCK, smem) != cudaSuccess) return 0;
    return n;
}

// block 256 with vectors in global scratch, or block 512 with vectors in shared memory
template <typename T, int P>
cudaError_t launch_p(const RecursionArgs<T> &args, int grid, int block, size_t smem, cudaStream_t stream)
{
    if (args.vec_in_smem) return block == 512 ? launch_cfg<T, P, 512, true>(args, grid, smem, stream)
                                             : launch_cfg<T, P, 256, true>(args, grid, smem, stream);
    return launch_cfg<T, P, 256, false>(args, grid, smem, stream);
}

template <typename T, int P>
int blocks_p(int block, size_t smem, int vec_in_smem)
{
    if (vec_in_smem) return block == 512 ? blocks_cfg<T, P, 512, true>(smem) : blocks_cfg<T, P, 256, true>(smem);
    return blocks_cfg<T, P, 256, false>(smem);
}

template <typename T, int P, int BLOCK, bool VSMEM>
cudaError_t launch_batch_cfg(const BatchLaunch<T> &b, cudaStream_t stream)
{
    auto kern = batch_kernel<T, P, BLOCK, VSMEM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem);
    if (e != cudaSuccess) return e;
    kern<<<b.grid, BLOCK, b.smem, stream>>>(b.cells, b.items, b.nitems, b.counter, b.scratch, b.scratch_stride);
    return cudaGetLastError();
}

template <typename T, int P, int BLOCK, bool VSMEM>
int batch_blocks_cfg(size_t smem)
{
    auto kern = batch_kernel<T, P, BLOCK, VSMEM>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, BLOCK, smem) != cudaSuccess) return 0;
    return n;
}

template <typename T, int P>
cudaError_t launch_batch_p(const BatchLaunch<T> &b, cudaStream_t stream)
{
    if (b.vec_in_smem) return b.block == 512 ? launch_batch_cfg<T, P, 512, true>(b, stream)
                                             : launch_batch_cfg<T, P, 256, true>(b, stream);
    return launch_batch_cfg<T, P, 256, false>(b, stream);
}

template <typename T, int P>
int batch_blocks_p(int block, size_t smem, int vec_in_smem)
{
    if (vec_in_smem) return block == 512 ? batch_blocks_cfg<T, P, 512, true>(smem)
                                         : batch_blocks_cfg<T, P, 256, true>(smem);
    return batch_blocks_cfg<T, P, 256, false>(smem);
}

}  // namespace

template <typename T>
size_t recursion_smem_bytes(int natom, const int nc[3], int vec_in_smem)
{
    const size_t nc3 = (size_t)nc[0] * nc[1] * nc[2];
    const int nsx = (nc[0] + kSeg - 1) / kSeg;
    const int maskw = (natom + 31) / 32;
    size_t s = sizeof(AtomRec) * (size_t)natom;
    s += sizeof(T) * (4 * (size_t)natom + 1);
    s = (s + 15) & ~size_t(15);
    s += sizeof(double) * 4 * (size_t)natom;
    s += sizeof(int) * 40;
    s += sizeof(unsigned) * (size_t)(nc[1] + nc[2] + nsx) * maskw;
    s = (s + 15) & ~size_t(15);
    if (vec_in_smem) s += sizeof(T) * 2 * nc3;
    return s + 32;
}

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
cudaError_t launch_recursion(const RecursionArgs<T> &args, int fd_half, int grid, int block, size_t smem,
                             cudaStream_t stream)
{
    SQ_DISPATCH_P(launch_p, args, grid, block, smem, stream)
    return cudaErrorInvalidValue;
}

template <typename T>
int recursion_blocks_per_sm(int fd_half, int block, size_t smem, int vec_in_smem)
{
    SQ_DISPATCH_P(blocks_p, block, smem, vec_in_smem)
    return 0;
}

template <typename T, int P>
cudaError_t launch_adjoint_p(const RecursionArgs<T> &args, long long stride, int grid, size_t smem, cudaStream_t stream)
{
    auto kern = adjoint_kernel<T, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 256, smem, stream>>>(args, stride);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint(const RecursionArgs<T> &args, int fd_half, long long stride, int grid, size_t smem,
                           cudaStream_t stream)
{
    SQ_DISPATCH_P(launch_adjoint_p, args, stride, grid, smem, stream)
    return cudaErrorInvalidValue;
}

template cudaError_t launch_adjoint<double>(const RecursionArgs<double> &, int, long long, int, size_t, cudaStream_t);
template cudaError_t launch_adjoint<float>(const RecursionArgs<float> &, int, long long, int, size_t, cudaStream_t);

template <typename T>
cudaError_t launch_batch(const BatchLaunch<T> &b, int fd_half, cudaStream_t stream)
{
    SQ_DISPATCH_P(launch_batch_p, b, stream)
    return cudaErrorInvalidValue;
}

template <typename T>
int batch_blocks_per_sm(int fd_half, int block, size_t smem, int vec_in_smem)
{
    SQ_DISPATCH_P(batch_blocks_p, block, smem, vec_in_smem)
    return 0;
}

template cudaError_t launch_batch<double>(const BatchLaunch<double> &, int, cudaStream_t);
template cudaError_t launch_batch<float>(const BatchLaunch<float> &, int, cudaStream_t);
template int batch_blocks_per_sm<double>(int, int, size_t, int);
template int batch_blocks_per_sm<float>(int, int, size_t, int);
template cudaError_t launch_recursion<double>(const RecursionArgs<double> &, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_recursion<float>(const RecursionArgs<float> &, int, int, int, size_t, cudaStream_t);
template size_t recursion_smem_bytes<double>(int, const int *, int);
template size_t recursion_smem_bytes<float>(int, const int *, int);
template int recursion_blocks_per_sm<double>(int, int, size_t, int);
template int recursion_blocks_per_sm<float>(int, int, size_t, int);

}  // namespace sq
