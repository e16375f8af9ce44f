// FP32 per-column Chebyshev recursion for cubic 29^3 truncation cubes with the 12th-order stencil:
// the "cluster" kernel, a thread-block cluster of two CTAs (on two SMs) per column.
//
// Same mathematics as recursion_kernel and slab_kernel (Eq. Chebyshev on the truncated scaled
// Hamiltonian, with the Kleinman-Bylander term and the force moments of Eq. NLforceSQ).  A 29^3
// cube does not fit the one-CTA slab mapping: its two FP32 vectors alone take 190 KB of shared
// memory, and 29 warps leave 64 registers per thread for two 29-point pencils.  Here the cube's
// y-slabs are split between the two CTAs of a cluster (rank 0: slabs 0..14, rank 1: 15..28):
//   - warp w of rank r owns y-slab b = 15 r + w; lane l holds x position a = l (lanes 29..31 are
//     zero), and the z-pencil of v_k stays in registers (128 registers per thread: one 480-thread
//     CTA per SM);
//   - each CTA keeps in shared memory its own slabs of v_k plus the 6 slabs next to the split that
//     belong to the partner (the y reach of the stencil); after every step each CTA writes its 6
//     boundary slabs of v_{k+1} straight into the partner's buffer (distributed shared memory);
//   - v_{k-1} lives in registers; x neighbours come from predicated warp shuffles, y neighbours
//     from the shared buffer, z neighbours from registers;
//   - projector contractions chi^T v as in the slab kernel (two atoms per pass, z-half classes,
//     transposed butterflies, per-slab slots, fixed-order sums); each CTA sums its own slabs and
//     writes its partial into both CTAs, and both form the same total in the same order;
//   - force moments: each CTA adds its slabs' partial sums to A with FP64 atomics;
//   - two cluster barriers per step: X after the partial dots are exchanged (it also publishes
//     the halo slabs written in the previous step), and Y between the last read of v_k's buffer
//     (the local stencil) and the first write of v_{k+1}, split into arrive/wait around the
//     KB update so its latency overlaps that work.
// The barriers are hardware cluster barriers reached the same number of times by both CTAs (both
// take identical control flow: the column sequence, atom lists and K are shared), so no wait is open
// ended.  No TMA multicast is used.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <utility>

#include "sq_internal.h"
#include "sq_slab_common.cuh"

namespace cg = cooperative_groups;

namespace sq {
namespace {

using namespace slabdev;

template <int NC, int P>
struct CGeo {
    static constexpr int NB0 = (NC + 1) / 2;              // y-slabs of rank 0 (rank 1 owns NC - NB0)
    static constexpr int NW = NB0;                        // warps per CTA
    static constexpr int NR = NB0 + P;                    // rows of the shared vector buffer
    static constexpr int HB = NB0 - P;                    // slab held in row 0 of rank 1's buffer
    static constexpr int NZ = (NC + 1) & ~1;              // z-table entries per atom (even)
    static constexpr int HALF = ((NC - 1) / 2) & ~1;      // even split point of the z range
    static_assert(NC <= 32 && NC - NB0 + P <= NR, "layout");
};

struct CSmem {
    float *U;          // [NC z][NR rows][NC x]: own slabs of v_k plus the partner's P boundary slabs
    float2 *tx;        // [amax][NC]   (g, hp) along x
    float2 *ty;        // [amax][NB0]  (g, hp) along y, own slabs
    float4 *tz;        // [amax][NZ/2] (g[c], hp[c], g[c+1], hp[c+1]) along z
    float2 *fx;        // [fmax][NC]   (g', hp') of force atoms
    float2 *fy;        // [fmax][NB0]
    float4 *fz;        // [fmax][NZ/2]
    float *slot;       // [NB0][amax][4]
    float *fslot;      // [NB0][fmax][12]
    float *part;       // [2][amax][4]: partial dots of rank 0 and rank 1 (each written by its rank)
    float *sd;         // [amax][4]: total dots
    SlabRec *rec;      // [amax]
    double *chiq;      // [fmax][4]
    int *ftl;          // [fmax]
    unsigned *ymask;   // [NB0][W] own slabs
    unsigned *fbits;   // [W]
    unsigned *zlo;     // [W]
    unsigned *zhi;     // [W]
    float4 *zero;      // [NZ/2]
    int *scan;         // [40]
};

__host__ __device__ inline size_t c_align16(size_t x) { return (x + 15) & ~size_t(15); }

template <int NC, int P>
__host__ __device__ inline size_t cluster_layout(unsigned char *base, int amax, int fmax, CSmem *s)
{
    using G = CGeo<NC, P>;
    const int W = (amax + 31) / 32;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = c_align16(off + bytes);
        return base ? base + o : nullptr;
    };
    unsigned char *p;
    p = take(sizeof(float) * (size_t)NC * G::NR * NC);         if (s) s->U = (float *)p;
    p = take(sizeof(float2) * (size_t)amax * NC);              if (s) s->tx = (float2 *)p;
    p = take(sizeof(float2) * (size_t)amax * G::NB0);          if (s) s->ty = (float2 *)p;
    p = take(sizeof(float2) * (size_t)amax * G::NZ);           if (s) s->tz = (float4 *)p;
    p = take(sizeof(float2) * (size_t)fmax * NC);              if (s) s->fx = (float2 *)p;
    p = take(sizeof(float2) * (size_t)fmax * G::NB0);          if (s) s->fy = (float2 *)p;
    p = take(sizeof(float2) * (size_t)fmax * G::NZ);           if (s) s->fz = (float4 *)p;
    p = take(sizeof(float) * (size_t)G::NB0 * amax * 4);       if (s) s->slot = (float *)p;
    p = take(sizeof(float) * (size_t)G::NB0 * fmax * 12);      if (s) s->fslot = (float *)p;
    p = take(sizeof(float) * (size_t)2 * amax * 4);            if (s) s->part = (float *)p;
    p = take(sizeof(float) * (size_t)amax * 4);                if (s) s->sd = (float *)p;
    p = take(sizeof(SlabRec) * (size_t)amax);                  if (s) s->rec = (SlabRec *)p;
    p = take(sizeof(double) * (size_t)fmax * 4);               if (s) s->chiq = (double *)p;
    p = take(sizeof(int) * (size_t)fmax);                      if (s) s->ftl = (int *)p;
    p = take(sizeof(unsigned) * (size_t)G::NB0 * W);           if (s) s->ymask = (unsigned *)p;
    p = take(sizeof(unsigned) * (size_t)W);                    if (s) s->fbits = (unsigned *)p;
    p = take(sizeof(unsigned) * (size_t)W);                    if (s) s->zlo = (unsigned *)p;
    p = take(sizeof(unsigned) * (size_t)W);                    if (s) s->zhi = (unsigned *)p;
    p = take(sizeof(float4) * (size_t)(G::NZ / 2));            if (s) s->zero = (float4 *)p;
    p = take(sizeof(int) * 40);                                if (s) s->scan = (int *)p;
    return off;
}

// Per-thread geometry of the cluster mapping.
template <int NC, int P>
struct CThread {
    int lane, w, rank;
    int b;            // global y-slab of this warp (NC for rank 1's spare warp when NC is odd)
    int a;            // x position (= lane)
    bool slab;        // the warp owns a slab
    bool live;        // the thread holds a cube pencil
    bool centre_xy;   // (a, b) is the column's own (x, y)
    int row;          // buffer row of slab b
    int prow;         // row of slab b in the partner's buffer, or -1 when the partner does not hold it
    unsigned yvalid;  // bit 2j-2: slab b+j exists, bit 2j-1: slab b-j exists
    __device__ CThread(int rank_)
    {
        using G = CGeo<NC, P>;
        rank = rank_;
        lane = threadIdx.x & 31;
        w = threadIdx.x >> 5;
        b = rank * G::NB0 + w;
        a = lane;
        slab = b < NC;
        live = slab && a < NC;
        centre_xy = live && a == (NC - 1) / 2 && b == (NC - 1) / 2;
        row = b - (rank ? G::HB : 0);
        if (rank == 0) prow = (b >= G::NB0 - P && slab) ? b - G::HB : -1;
        else prow = (b < G::NB0 + P && slab) ? b : -1;
        yvalid = 0u;
#pragma unroll
        for (int j = 1; j <= P; j++) {
            if (slab && b + j < NC) yvalid |= 1u << (2 * j - 2);
            if (slab && b - j >= 0) yvalid |= 1u << (2 * j - 1);
        }
    }
};

// t += wgt * (x of lane + j) when that lane exists, and t += wgt * (x of lane - j) likewise
// (predicated FMAs on the shuffle's in-range predicate; lanes past the cube hold zeros).
__device__ __forceinline__ float xpair(float t, float x, int j, float wgt)
{
    asm("{\n\t.reg .pred pu, pd;\n\t.reg .f32 ru, rd;\n\t"
        "shfl.sync.down.b32 rd|pd, %1, %2, 0x1f, 0xffffffff;\n\t"
        "shfl.sync.up.b32 ru|pu, %1, %2, 0x0, 0xffffffff;\n\t"
        "@pd fma.rn.f32 %0, %3, rd, %0;\n\t"
        "@pu fma.rn.f32 %0, %3, ru, %0;\n\t}"
        : "+f"(t)
        : "f"(x), "r"(j), "f"(wgt));
    return t;
}

// Per-column set-up (same rules as slab_setup): ordered active atoms, window tables (y tables and
// masks for this CTA's slabs), force atoms and their tables.  Both CTAs compute the same lists.
template <int NC, int P>
__device__ int cluster_setup(const RecursionArgs<float> &args, const CSmem &S, long long q, int amax, int fmax,
                             int *err, int qa[3], int *nfrc_out, int rank)
{
    using G = CGeo<NC, P>;
    constexpr int NZ = G::NZ, NB0 = G::NB0, kHalf = G::HALF;
    const int NTH = blockDim.x;
    const int W = (amax + 31) / 32;
    const int natom = args.natom;
    const int bfirst = rank * NB0;
    qa[0] = (int)(q % args.n[0]);
    qa[1] = (int)((q / args.n[0]) % args.n[1]);
    qa[2] = (int)(q / ((long long)args.n[0] * args.n[1]));
    int wstart[3];
#pragma unroll
    for (int ax = 0; ax < 3; ax++) wstart[ax] = smod(qa[ax] - args.m[ax], args.n[ax]);
    int nact = 0;
    for (int base = 0; base < natom; base += NTH) {
        const int J = base + (int)threadIdx.x;
        bool on = J < natom;
        short lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int ax = 0; ax < 3 && on; ax++)
            on = window_range(args.sup_start[J * 3 + ax], args.sup_len[J * 3 + ax], args.n[ax], NC, wstart[ax],
                              lo[ax], hi[ax]);
        int total;
        const int slot = compact(on, S.scan, &total);
        if (slot >= 0 && nact + slot < amax) {
            SlabRec r;
            r.J = J;
            r.fidx = -1;
            for (int ax = 0; ax < 3; ax++) {
                r.lo[ax] = lo[ax];
                r.hi[ax] = hi[ax];
            }
            S.rec[nact + slot] = r;
        }
        nact += total;
    }
    if (nact > amax) {
        if (threadIdx.x == 0 && rank == 0) atomicExch(err, 1);
        return -1;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < nact * NC; it += NTH) {
        const int o = it % NC, t = it / NC;
        const float *f0 = args.fac + (size_t)S.rec[t].J * args.fac_stride + args.fac_off[0] + wstart[0] + o;
        S.tx[it] = make_float2(f0[0], f0[2 * args.n[0]]);
    }
    for (int it = threadIdx.x; it < nact * NB0; it += NTH) {
        const int o = it % NB0, t = it / NB0;
        float2 v = make_float2(0.f, 0.f);
        if (bfirst + o < NC) {
            const float *f1 = args.fac + (size_t)S.rec[t].J * args.fac_stride + args.fac_off[1] + wstart[1] + bfirst + o;
            v = make_float2(f1[0], f1[2 * args.n[1]]);
        }
        S.ty[it] = v;
    }
    for (int it = threadIdx.x; it < nact * NZ; it += NTH) {
        const int o = it % NZ, t = it / NZ;
        float2 v = make_float2(0.f, 0.f);
        if (o < NC) {
            const float *f2 = args.fac + (size_t)S.rec[t].J * args.fac_stride + args.fac_off[2] + wstart[2] + o;
            v = make_float2(f2[0], f2[2 * args.n[2]]);
        }
        reinterpret_cast<float2 *>(S.tz)[it] = v;
    }
    int nfrc = 0;
    if (args.want_force) {
        for (int base = 0; base < nact; base += NTH) {
            const int t = base + (int)threadIdx.x;
            bool on = false;
            const double *f = nullptr;
            if (t < nact) {
                f = args.fac64 + (size_t)S.rec[t].J * args.fac64_stride;
                on = f[args.fac64_off[0] + qa[0]] != 0.0 && f[args.fac64_off[1] + qa[1]] != 0.0 &&
                     f[args.fac64_off[2] + qa[2]] != 0.0;
            }
            int total;
            const int slot = compact(on, S.scan, &total);
            if (slot >= 0 && nfrc + slot < fmax) {
                const int fi = nfrc + slot;
                S.rec[t].fidx = fi;
                S.ftl[fi] = t;
                const double gx = f[args.fac64_off[0] + qa[0]], hx = f[args.fac64_off[0] + args.n[0] + qa[0]];
                const double gy = f[args.fac64_off[1] + qa[1]], hy = f[args.fac64_off[1] + args.n[1] + qa[1]];
                const double gz = f[args.fac64_off[2] + qa[2]], hz = f[args.fac64_off[2] + args.n[2] + qa[2]];
                S.chiq[4 * fi + 0] = args.Nnorm * gx * gy * gz;
                S.chiq[4 * fi + 1] = args.Nnorm * hx * gy * gz;
                S.chiq[4 * fi + 2] = args.Nnorm * gx * hy * gz;
                S.chiq[4 * fi + 3] = args.Nnorm * gx * gy * hz;
            }
            nfrc += total;
        }
        if (nfrc > fmax) {
            if (threadIdx.x == 0 && rank == 0) atomicExch(err, 2);
            return -1;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < nfrc * NC; it += NTH) {
            const int o = it % NC, fi = it / NC;
            const float *f0 = args.fac + (size_t)S.rec[S.ftl[fi]].J * args.fac_stride + args.fac_off[0] + wstart[0] + o;
            S.fx[it] = make_float2(f0[4 * args.n[0]], f0[6 * args.n[0]]);
        }
        for (int it = threadIdx.x; it < nfrc * NB0; it += NTH) {
            const int o = it % NB0, fi = it / NB0;
            float2 v = make_float2(0.f, 0.f);
            if (bfirst + o < NC) {
                const float *f1 = args.fac + (size_t)S.rec[S.ftl[fi]].J * args.fac_stride + args.fac_off[1] +
                                  wstart[1] + bfirst + o;
                v = make_float2(f1[4 * args.n[1]], f1[6 * args.n[1]]);
            }
            S.fy[it] = v;
        }
        for (int it = threadIdx.x; it < nfrc * NZ; it += NTH) {
            const int o = it % NZ, fi = it / NZ;
            float2 v = make_float2(0.f, 0.f);
            if (o < NC) {
                const float *f2 = args.fac + (size_t)S.rec[S.ftl[fi]].J * args.fac_stride + args.fac_off[2] +
                                  wstart[2] + o;
                v = make_float2(f2[4 * args.n[2]], f2[6 * args.n[2]]);
            }
            reinterpret_cast<float2 *>(S.fz)[it] = v;
        }
    }
    for (int it = threadIdx.x; it < NB0 * W; it += NTH) {
        const int wd = it % W, bl = it / W;
        const int bb = bfirst + bl;
        unsigned msk = 0u;
        if (bb < NC)
            for (int t = 32 * wd; t < min(nact, 32 * wd + 32); t++)
                if (bb >= S.rec[t].lo[1] && bb <= S.rec[t].hi[1]) msk |= 1u << (t - 32 * wd);
        S.ymask[it] = msk;
    }
    for (int wd = threadIdx.x; wd < W; wd += NTH) {
        unsigned fb = 0u, zl = 0u, zh = 0u;
        for (int t = 32 * wd; t < min(nact, 32 * wd + 32); t++) {
            const unsigned bit = 1u << (t - 32 * wd);
            if (S.rec[t].fidx >= 0) fb |= bit;
            if (S.rec[t].hi[2] <= kHalf) zl |= bit;
            else if (S.rec[t].lo[2] >= kHalf) zh |= bit;
        }
        S.fbits[wd] = fb;
        S.zlo[wd] = zl;
        S.zhi[wd] = zh;
    }
    __syncthreads();   // tables and masks complete before any warp reads them
    *nfrc_out = nfrc;
    return nact;
}

// Projector contractions of two atoms per pass over z in [C0, C1), into this warp's slab slots.
template <int NC, int P, int C0, int C1>
__device__ __forceinline__ void cl_dots_pairs(unsigned msk, int wd, const CSmem &S, const float (&vz)[NC], int bl,
                                              int a, bool live, int lane, int amax)
{
    constexpr int NZ = CGeo<NC, P>::NZ, NB0 = CGeo<NC, P>::NB0;
    while (msk) {
        const int t0 = 32 * wd + __ffs(msk) - 1;
        msk &= msk - 1u;
        const bool two = msk != 0u;
        const int t1 = two ? 32 * wd + __ffs(msk) - 1 : t0;
        msk &= msk - 1u;
        const float4 *z0 = S.tz + t0 * (NZ / 2);
        const float4 *z1 = two ? S.tz + t1 * (NZ / 2) : S.zero;
        float G0a = 0.f, H0a = 0.f, G0b = 0.f, H0b = 0.f;
        float G1a = 0.f, H1a = 0.f, G1b = 0.f, H1b = 0.f;
#pragma unroll
        for (int c = C0; c < C1; c += 2) {
            const float4 p0 = z0[c >> 1], p1 = z1[c >> 1];
            G0a += p0.x * vz[c];
            H0a += p0.y * vz[c];
            G1a += p1.x * vz[c];
            H1a += p1.y * vz[c];
            if (c + 1 < NC) {
                G0b += p0.z * vz[c + 1];
                H0b += p0.w * vz[c + 1];
                G1b += p1.z * vz[c + 1];
                H1b += p1.w * vz[c + 1];
            }
        }
        const float G0 = G0a + G0b, H0 = H0a + H0b, G1 = G1a + G1b, H1 = H1a + H1b;
        const float2 x0 = live ? S.tx[t0 * NC + a] : make_float2(0.f, 0.f);
        const float2 x1 = live ? S.tx[t1 * NC + a] : make_float2(0.f, 0.f);
        const float v8[8] = {x0.x * G0, x0.y * G0, x0.x * H0, x0.x * G0, x1.x * G1, x1.y * G1, x1.x * H1, x1.x * G1};
        const float red = reduce8(v8, lane);
        const int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if ((lane & 3) == 0 && (idx < 4 || two)) {
            const int t = idx < 4 ? t0 : t1;
            const int comp = idx & 3;
            const float2 yv = S.ty[t * NB0 + bl];
            S.slot[((size_t)bl * amax + t) * 4 + (comp == 2 ? 3 : comp == 3 ? 2 : comp)] = (comp == 3 ? yv.y : yv.x) * red;
        }
    }
}

// KB update of two atoms per pass over z in [C0, C1): w += kappa_l chi (chi^T v) from the total dots.
template <int NC, int P, int C0, int C1>
__device__ __forceinline__ void cl_update_pairs(unsigned msk, int wd, const CSmem &S, float (&w)[NC], int bl, int a,
                                                bool live, float kap0, float kap1)
{
    constexpr int NZ = CGeo<NC, P>::NZ, NB0 = CGeo<NC, P>::NB0;
    while (msk) {
        const int t0 = 32 * wd + __ffs(msk) - 1;
        msk &= msk - 1u;
        const bool two = msk != 0u;
        const int t1 = two ? 32 * wd + __ffs(msk) - 1 : t0;
        msk &= msk - 1u;
        float A1[2], A2[2];
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int t = i ? t1 : t0;
            const float4 s = *reinterpret_cast<const float4 *>(S.sd + 4 * t);
            const float2 yv = S.ty[t * NB0 + bl];
            const float2 xv = live ? S.tx[t * NC + a] : make_float2(0.f, 0.f);
            const float Pv = kap0 * s.x * yv.x + kap1 * s.z * yv.y;
            const float Qv = kap1 * s.w * yv.x;
            const float Rv = kap1 * s.y * yv.x;
            A1[i] = xv.x * Pv + xv.y * Rv;
            A2[i] = xv.x * Qv;
        }
        const float4 *z0 = S.tz + t0 * (NZ / 2);
        const float4 *z1 = two ? S.tz + t1 * (NZ / 2) : S.zero;
#pragma unroll
        for (int c = C0; c < C1; c += 2) {
            const float4 p0 = z0[c >> 1], p1 = z1[c >> 1];
            w[c] += p0.x * A1[0] + p0.y * A2[0] + p1.x * A1[1] + p1.y * A2[1];
            if (c + 1 < NC) w[c + 1] += p0.z * A1[0] + p0.w * A2[0] + p1.z * A1[1] + p1.w * A2[1];
        }
    }
}

// Contraction phase of step k: this CTA's slots, then its slab sums -> partial dots written into both
// CTAs' part[rank] (and force moments added to A).  Ends before the cluster barrier X.
template <int NC, int P>
__device__ __forceinline__ void cluster_contract(const RecursionArgs<float> &args, const CSmem &S, float *part_remote,
                                                 const CThread<NC, P> &th, const float (&vz)[NC], int k,
                                                 bool need_dots, int nact, int nfrc, int amax, int fmax)
{
    using G = CGeo<NC, P>;
    constexpr int NZ = G::NZ, NB0 = G::NB0, kHalf = G::HALF;
    const int W = (amax + 31) / 32;
    const int bl = th.w, a = th.a, lane = th.lane;
    const bool live = th.live;
    const int NTH = blockDim.x;
    if (th.slab && (need_dots || args.want_force)) {
        for (int wd = 0; wd < W; wd++) {
            const unsigned all = S.ymask[bl * W + wd];
            const unsigned fb = S.fbits[wd];
            if (need_dots) {
                const unsigned nf = all & ~fb, zl = S.zlo[wd], zh = S.zhi[wd];
                cl_dots_pairs<NC, P, 0, kHalf + 1>(nf & zl, wd, S, vz, bl, a, live, lane, amax);
                cl_dots_pairs<NC, P, kHalf, NC>(nf & zh, wd, S, vz, bl, a, live, lane, amax);
                cl_dots_pairs<NC, P, 0, NC>(nf & ~(zl | zh), wd, S, vz, bl, a, live, lane, amax);
            }
            unsigned msk = args.want_force ? (all & fb) : 0u;
            while (msk) {
                const int t = 32 * wd + __ffs(msk) - 1;
                msk &= msk - 1u;
                const int fidx = S.rec[t].fidx;
                const float4 *tz = S.tz + t * (NZ / 2);
                const float4 *fz = S.fz + fidx * (NZ / 2);
                float Ga = 0.f, Ha = 0.f, Gda = 0.f, Hda = 0.f, Gb = 0.f, Hb = 0.f, Gdb = 0.f, Hdb = 0.f;
#pragma unroll
                for (int c = 0; c < NC; c += 2) {
                    const float4 z = tz[c >> 1], zd = fz[c >> 1];
                    Ga += z.x * vz[c];
                    Ha += z.y * vz[c];
                    Gda += zd.x * vz[c];
                    Hda += zd.y * vz[c];
                    if (c + 1 < NC) {
                        Gb += z.z * vz[c + 1];
                        Hb += z.w * vz[c + 1];
                        Gdb += zd.z * vz[c + 1];
                        Hdb += zd.w * vz[c + 1];
                    }
                }
                const float Gs = Ga + Gb, Hs = Ha + Hb, Gd = Gda + Gdb, Hd = Hda + Hdb;
                const float2 xv = live ? S.tx[t * NC + a] : make_float2(0.f, 0.f);
                const float2 yv = S.ty[t * NB0 + bl];
                float *sl = S.slot + ((size_t)bl * amax + t) * 4;
                const float2 xd = live ? S.fx[fidx * NC + a] : make_float2(0.f, 0.f);
                const float2 yd = S.fy[fidx * NB0 + bl];
                const float v8[8] = {xv.x * Gs, xv.y * Gs, xv.x * Hs, xd.x * Gs, xv.x * Gd, xd.y * Gs, xv.y * Gd, xd.x * Hs};
                const float red = reduce8(v8, lane);
                const float v9 = wsum(xv.x * Hd);
                const int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                float *fs = S.fslot + ((size_t)bl * fmax + fidx) * 12;
                if ((lane & 3) == 0) {
                    switch (idx) {
                    case 0: if (need_dots) { sl[0] = yv.x * red; sl[2] = yv.y * red; }
                            fs[1] = yd.x * red; fs[7] = yd.y * red; break;
                    case 1: if (need_dots) sl[1] = yv.x * red;
                            fs[4] = yd.x * red; break;
                    case 2: if (need_dots) sl[3] = yv.x * red;
                            fs[10] = yd.x * red; break;
                    case 3: fs[0] = yv.x * red; fs[6] = yv.y * red; break;
                    case 4: fs[2] = yv.x * red; fs[8] = yv.y * red; break;
                    case 5: fs[3] = yv.x * red; break;
                    case 6: fs[5] = yv.x * red; break;
                    default: fs[9] = yv.x * red; break;
                    }
                }
                if (lane == 0) fs[11] = yv.x * v9;
            }
        }
    }
    __syncthreads();
    // fixed-order sums over this CTA's slabs
    if (need_dots) {
        float *mine = S.part + (size_t)th.rank * amax * 4;
        float *theirs = part_remote + (size_t)th.rank * amax * 4;
        for (int it = threadIdx.x; it < nact * 4; it += NTH) {
            const int t = it >> 2, comp = it & 3;
            float s = 0.f;
            for (int bb = 0; bb < NB0; bb++)
                if ((S.ymask[bb * W + (t >> 5)] >> (t & 31)) & 1u) s += S.slot[((size_t)bb * amax + t) * 4 + comp];
            mine[it] = s;
            theirs[it] = s;
        }
    }
    if (args.want_force) {
        const int nproj = args.nproj, natom = args.natom;
        const int nf = nproj > 1 ? 12 : 3;
        for (int it = threadIdx.x; it < nfrc * nf; it += NTH) {
            const int fi = it / nf, i = it % nf;
            const int t = S.ftl[fi];
            double s = 0.0;
            bool any = false;
            for (int bb = 0; bb < NB0; bb++)
                if ((S.ymask[bb * W + (t >> 5)] >> (t & 31)) & 1u) {
                    s += (double)S.fslot[((size_t)bb * fmax + fi) * 12 + i];
                    any = true;
                }
            const int lm = i / 3, d = i % 3;
            if (any)
                atomicAdd(args.A + ((((size_t)k * natom + S.rec[t].J) * nproj + lm) * 3 + d),
                          S.chiq[4 * fi + lm] * args.Nnorm * s);
        }
    }
}

template <int NC, int P>
__global__ void __launch_bounds__(CGeo<NC, P>::NW * 32, 1) cluster_kernel(const RecursionArgs<float> args, int amax,
                                                                         int fmax, int *err)
{
    using G = CGeo<NC, P>;
    constexpr int NZ = G::NZ, NR = G::NR, kHalf = G::HALF;
    static_assert(P <= 6, "x shuffles assume a half-width of at most 6");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int partner = rank ^ 1;
    CSmem S;
    cluster_layout<NC, P>(smem_raw, amax, fmax, &S);
    float *U_remote = cluster.map_shared_rank(S.U, partner);
    float *part_remote = cluster.map_shared_rank(S.part, partner);
    const CThread<NC, P> th(rank);
    const int m = (NC - 1) / 2;
    const long long N_d = args.N_d;
    const size_t plane_p = (size_t)args.pn[0] * args.pn[1];
    const long long ncl = gridDim.x / 2;
    const long long cid = blockIdx.x / 2;
    const float kap0 = args.kappa[0], kap1 = args.kappa[1];
    const int W = (amax + 31) / 32;

    for (int i = threadIdx.x; i < NZ / 2; i += blockDim.x) S.zero[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    cluster.sync();   // both CTAs are running before any write into the partner's shared memory

    for (long long q = args.q0 + cid; q < args.q1; q += ncl) {
        int qa[3], nfrc = 0;
        const int nact = cluster_setup<NC, P>(args, S, q, amax, fmax, err, qa, &nfrc, rank);
        if (nact < 0) continue;   // both CTAs see the same count
        // ---- v_0 = e_q (registers, own rows, the partner's halo rows), v_{-1} = 0 ----
        float vz[NC], vp[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) {
            vz[c] = (th.centre_xy && c == m) ? 1.0f : 0.0f;
            vp[c] = 0.f;
            if (th.live) {
                S.U[((size_t)c * NR + th.row) * NC + th.a] = vz[c];
                if (th.prow >= 0) U_remote[((size_t)c * NR + th.prow) * NC + th.a] = vz[c];
            }
        }
        if (th.centre_xy) args.mu[q] = 1.0f;
        const float *drow = args.dpad + (size_t)qa[2] * plane_p + (size_t)(qa[1] + (th.slab ? th.b : 0)) * args.pn[0] +
                            qa[0] + (th.live ? th.a : 0);

        for (int k = 0; k <= args.K; k++) {
            const bool need_dots = k < args.K;
            cluster_contract<NC, P>(args, S, part_remote, th, vz, k, need_dots, nact, nfrc, amax, fmax);
            cluster.sync();   // X: partial dots of both CTAs, and the halo rows of v_k, are visible
            if (!need_dots) break;
            for (int it = threadIdx.x; it < nact * 4; it += blockDim.x) S.sd[it] = S.part[it] + S.part[amax * 4 + it];
            __syncthreads();
            const float ca = k == 0 ? 1.f : 2.f, cb = k == 0 ? 0.f : 1.f;
            // ---- local part of Hhat v_k: stencil and diagonal ----
            float w[NC];
#pragma unroll
            for (int c = 0; c < NC; c++) {
                const float x = vz[c];
                float t = 0.f;
#pragma unroll
                for (int j = 1; j <= P; j++) {
                    const float zp = (c + j < NC) ? vz[c + j] : 0.f;
                    const float zm = (c - j >= 0) ? vz[c - j] : 0.f;
                    t += args.w[2][j - 1] * (zp + zm);
                }
#pragma unroll
                for (int j = 1; j <= P; j++) t = xpair(t, x, j, args.w[0][j - 1]);
                if (th.live) {
                    const float *row = S.U + ((size_t)c * NR + th.row) * NC + th.a;
#pragma unroll
                    for (int j = 1; j <= P; j++) {
                        const float yp = (th.yvalid >> (2 * j - 2)) & 1u ? row[j * NC] : 0.f;
                        const float ym = (th.yvalid >> (2 * j - 1)) & 1u ? row[-j * NC] : 0.f;
                        t += args.w[1][j - 1] * (yp + ym);
                    }
                    w[c] = t + drow[(size_t)c * plane_p] * x;
                } else {
                    w[c] = 0.f;
                }
            }
            // Y (arrive): this CTA's reads of v_k's buffer are done
            __syncwarp();
            auto y_token = cluster.barrier_arrive();
            // ---- KB term ----
            if (th.slab) {
                for (int wd = 0; wd < W; wd++) {
                    const unsigned all = S.ymask[th.w * W + wd], zl = S.zlo[wd], zh = S.zhi[wd];
                    cl_update_pairs<NC, P, 0, kHalf + 1>(all & zl, wd, S, w, th.w, th.a, th.live, kap0, kap1);
                    cl_update_pairs<NC, P, kHalf, NC>(all & zh, wd, S, w, th.w, th.a, th.live, kap0, kap1);
                    cl_update_pairs<NC, P, 0, NC>(all & ~(zl | zh), wd, S, w, th.w, th.a, th.live, kap0, kap1);
                }
            }
            // Y (wait): both CTAs are done reading v_k's buffers
            __syncwarp();
            cluster.barrier_wait(std::move(y_token));
            // ---- v_{k+1} = ca Hhat v_k - cb v_{k-1}; v_k becomes v_{k-1} ----
#pragma unroll
            for (int c = 0; c < NC; c++) {
                if (th.live) {
                    // v_k comes back from the own row it still occupies, so its registers are free
                    // during the KB update
                    float *own = S.U + ((size_t)c * NR + th.row) * NC + th.a;
                    const float nv = ca * w[c] - cb * vp[c];
                    vp[c] = *own;
                    vz[c] = nv;
                    *own = nv;
                    if (th.prow >= 0) U_remote[((size_t)c * NR + th.prow) * NC + th.a] = nv;
                } else {
                    vp[c] = 0.f;
                    vz[c] = 0.f;
                }
            }
            if (th.centre_xy) args.mu[(size_t)(k + 1) * N_d + q] = vz[m];
        }
    }
    cluster.sync();   // no CTA leaves while its partner may still write into its shared memory
}

template <int NC, int P>
cudaError_t cluster_config(int amax, int fmax, size_t *smem, int *max_clusters)
{
    using G = CGeo<NC, P>;
    const size_t sm = cluster_layout<NC, P>(nullptr, amax, fmax, nullptr);
    *smem = sm;
    auto kern = cluster_kernel<NC, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(G::NW * 32, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, kern, &cfg);
}

template <int NC, int P>
cudaError_t cluster_launch(const RecursionArgs<float> &args, int amax, int fmax, int nclusters, size_t smem, int *err,
                           cudaStream_t stream)
{
    using G = CGeo<NC, P>;
    auto kern = cluster_kernel<NC, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * nclusters, 1, 1);
    cfg.blockDim = dim3(G::NW * 32, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, args, amax, fmax, err);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

bool cluster_supported(const int nc[3], int fd_half)
{
    return nc[0] == nc[1] && nc[1] == nc[2] && nc[0] == 29 && fd_half == 6;
}

cudaError_t cluster_prepare(int nc, int amax, int fmax, size_t *smem, int *max_clusters)
{
    if (nc != 29) return cudaErrorInvalidValue;
    return cluster_config<29, 6>(amax, fmax, smem, max_clusters);
}

cudaError_t launch_cluster(const RecursionArgs<float> &args, int amax, int fmax, int nclusters, size_t smem, int *err,
                           cudaStream_t stream)
{
    if (args.nc[0] != 29) return cudaErrorInvalidValue;
    return cluster_launch<29, 6>(args, amax, fmax, nclusters, smem, err, stream);
}

}  // namespace sq
