// Device helpers shared by the FP32 slab kernels (one CTA per column) and the cluster kernels (a
// cluster of CTAs per column): atom records, periodic window ranges, warp reductions and the ordered
// block-wide compaction.  Internal to libsq.
#pragma once

#include <cuda_runtime.h>

namespace sq {
namespace slabdev {

struct SlabRec {
    int J;          // atom index
    int fidx;       // force slot or -1
    short lo[3];    // bounding local range of the support inside the cube, per axis
    short hi[3];
};

__device__ __forceinline__ int smod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Support range of atom J's projector inside the cube window [wstart, wstart + nc) on one axis,
// as a bounding local interval; false when they do not meet.  (Same rule as recursion_kernel.)
__device__ __forceinline__ bool window_range(int st, int len, int na, int nca, int wstart, short &lo, short &hi)
{
    if (len >= na) {
        lo = 0;
        hi = (short)(nca - 1);
        return true;
    }
    const bool first_in = smod(wstart - st, na) < len;
    const int d = smod(st - wstart, na);
    const bool starts_in = d < nca;
    if (!first_in && !starts_in) return false;
    const bool last_in = smod(wstart + nca - 1 - st, na) < len;
    lo = (short)(first_in ? 0 : d);
    hi = (last_in || (first_in && starts_in && d > 0)) ? (short)(nca - 1) : (short)smod(st + len - 1 - wstart, na);
    return true;
}

// Transposed butterfly: on entry every lane holds v[0..7]; on exit the lane holds the warp-wide sum
// of v[idx] with idx = 4 bit4(lane) + 2 bit3(lane) + bit2(lane) (9 shuffles instead of 40).
__device__ __forceinline__ float reduce8(const float v[8], int lane)
{
    float a[4], b[2];
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float send = h16 ? v[i] : v[i + 4];
        const float keep = h16 ? v[i + 4] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float send = h8 ? a[i] : a[i + 2];
        const float keep = h8 ? a[i + 2] : a[i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c = (h4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h4 ? b[0] : b[1], 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// Transposed butterfly for four values: the lane ends with the warp-wide sum of v[2 bit4 + bit3].
__device__ __forceinline__ float reduce4(const float v[4], int lane)
{
    float a[2];
    const bool h16 = lane & 16, h8 = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float send = h16 ? v[i] : v[i + 2];
        const float keep = h16 ? v[i + 2] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float c = (h8 ? a[1] : a[0]) + __shfl_xor_sync(0xffffffffu, h8 ? a[0] : a[1], 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// Ordered block-wide compaction (see recursion_kernel).
__device__ inline int compact(bool flag, int *scan, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) scan[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < nwarp; w++) {
            const int c = scan[w];
            scan[w] = acc;
            acc += c;
        }
        scan[32] = acc;
    }
    __syncthreads();
    const int slot = flag ? scan[warp] + __popc(bal & ((1u << lane) - 1u)) : -1;
    *total = scan[32];
    __syncthreads();
    return slot;
}

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace slabdev
}  // namespace sq
