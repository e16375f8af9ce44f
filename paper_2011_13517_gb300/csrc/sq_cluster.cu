// FP32 per-column Chebyshev recursion for cubic 29^3 truncation cubes with the 12th-order stencil:
// the "cluster" kernel, a thread-block cluster of two CTAs (on two SMs) per column.
//
// Same mathematics as recursion_kernel and slab_kernel (Eq. Chebyshev on the truncated scaled
// Hamiltonian, with the Kleinman-Bylander term and the force moments of Eq. NLforceSQ).  A 29^3
// cube does not fit the one-CTA slab mapping: its two FP32 vectors alone take 190 KB of shared
// memory, and 29 warps leave 64 registers per thread for two 29-point pencils.  Here the cube's
// y-slabs are split between the two CTAs of a cluster (rank 0: slabs 0..14, rank 1: 15..28), and
// each slab's z range between two warps of its CTA (z 0..14 and z 15..28):
//   - warp 2s + h of rank r owns y-slab b = 15 r + s and z-half h; lane l holds x position a = l
//     (lanes 29..31 are zero), and the warp's 15-point z-pencil of v_k stays in registers (30 warps,
//     64 registers per thread, one 960-thread CTA per SM); v_{k-1} waits in per-CTA global scratch
//     (L2-resident), read and written once per step;
//   - each CTA keeps in shared memory its own slabs of v_k (all z) plus the 6 slabs next to the split
//     that belong to the partner (the y reach of the stencil); after every step each CTA writes its
//     boundary slabs of v_{k+1} straight into the partner's buffer (distributed shared memory);
//   - x neighbours come from predicated warp shuffles, y neighbours from the shared buffer, z
//     neighbours from registers, or from the shared buffer across the z split;
//   - projector contractions chi^T v as in the slab kernel (two atoms per pass, transposed
//     butterflies, per-(slab, z-half) slots, fixed-order sums) over each warp's z half, skipping the
//     atoms whose support lies in the other half; each CTA sums its own slots and writes its partial
//     into both CTAs, and both form the same total in the same order;
//   - force moments: each CTA adds its slots' partial sums to A with FP64 atomics;
//   - two cluster barriers per step: X after the partial dots are exchanged (it also publishes
//     the halo slabs and the other z half written in the previous step), and Y between the last
//     read of v_k's buffer (the local stencil) and the first write of v_{k+1}, split into
//     arrive/wait around the KB update so its latency overlaps that work.
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
    static constexpr int NW = 2 * NB0;                    // warps per CTA: two z halves per slab
    static constexpr int NR = NB0 + P;                    // rows of the shared vector buffer
    static constexpr int HB = NB0 - P;                    // slab held in row 0 of rank 1's buffer
    static constexpr int ZS = (NC + 1) / 2;               // z split: half 0 holds z < ZS, half 1 the rest
    static constexpr int ZL = ZS;                         // pencil registers per thread
    static constexpr int NZP = (ZL + 1) / 2;              // float4 z-table entries per atom and half
    static constexpr int SCR = NC * NB0 * 32;             // floats of v_{k-1} scratch per CTA
    static_assert(NC <= 32 && NC - NB0 + P <= NR && 2 * ZS >= NC, "layout");
};
template <int NC, int P, int H>
struct ZHalf {
    static constexpr int Z0 = H * CGeo<NC, P>::ZS;                         // first z of the half
    static constexpr int LEN = H ? NC - CGeo<NC, P>::ZS : CGeo<NC, P>::ZS;  // z points of the half
};

struct CSmem {
    float *U;          // [NC z][NR rows][NC x]: own slabs of v_k plus the partner's P boundary slabs
    float2 *tx;        // [amax][NC]   (g, hp) along x
    float2 *ty;        // [amax][NB0]  (g, hp) along y, own slabs
    float4 *tz;        // [2][amax][NZP] per z half: (g[z], hp[z], g[z+1], hp[z+1]) from the half's first z
    float2 *fx;        // [fmax][NC]   (g', hp') of force atoms
    float2 *fy;        // [fmax][NB0]
    float4 *fz;        // [2][fmax][NZP]
    float *slot;       // [NB0][2][amax][4] per (slab, z half)
    float *fslot;      // [NB0][2][fmax][12]
    float *part;       // [2][amax][4]: partial dots of rank 0 and rank 1 (each written by its rank)
    float *sd;         // [amax][4]: total dots
    SlabRec *rec;      // [amax]
    double *chiq;      // [fmax][4]
    int *ftl;          // [fmax]
    unsigned *ymask;   // [NB0][W] own slabs
    unsigned *zmask;   // [2][W]: atoms whose z support meets half h
    unsigned *fbits;   // [W]
    float4 *zero;      // [NZP]
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
    p = take(sizeof(float4) * (size_t)2 * amax * G::NZP);      if (s) s->tz = (float4 *)p;
    p = take(sizeof(float2) * (size_t)fmax * NC);              if (s) s->fx = (float2 *)p;
    p = take(sizeof(float2) * (size_t)fmax * G::NB0);          if (s) s->fy = (float2 *)p;
    p = take(sizeof(float4) * (size_t)2 * fmax * G::NZP);      if (s) s->fz = (float4 *)p;
    p = take(sizeof(float) * (size_t)G::NB0 * 2 * amax * 4);   if (s) s->slot = (float *)p;
    p = take(sizeof(float) * (size_t)G::NB0 * 2 * fmax * 12);  if (s) s->fslot = (float *)p;
    p = take(sizeof(float) * (size_t)2 * amax * 4);            if (s) s->part = (float *)p;
    p = take(sizeof(float) * (size_t)amax * 4);                if (s) s->sd = (float *)p;
    p = take(sizeof(SlabRec) * (size_t)amax);                  if (s) s->rec = (SlabRec *)p;
    p = take(sizeof(double) * (size_t)fmax * 4);               if (s) s->chiq = (double *)p;
    p = take(sizeof(int) * (size_t)fmax);                      if (s) s->ftl = (int *)p;
    p = take(sizeof(unsigned) * (size_t)G::NB0 * W);           if (s) s->ymask = (unsigned *)p;
    p = take(sizeof(unsigned) * (size_t)2 * W);                if (s) s->zmask = (unsigned *)p;
    p = take(sizeof(unsigned) * (size_t)W);                    if (s) s->fbits = (unsigned *)p;
    p = take(sizeof(float4) * (size_t)G::NZP);                 if (s) s->zero = (float4 *)p;
    p = take(sizeof(int) * 40);                                if (s) s->scan = (int *)p;
    return off;
}

// Per-thread geometry of the cluster mapping.
template <int NC, int P>
struct CThread {
    int lane, w, rank;
    int bl;           // local y-slab of this warp (0 .. NB0-1)
    int zh;           // z half of this warp
    int b;            // global y-slab (NC for rank 1's spare slab when NC is odd)
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
        bl = w >> 1;
        zh = w & 1;
        b = rank * G::NB0 + bl;
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
// masks for this CTA's slabs, z tables per z half), force atoms and their tables.  Both CTAs compute
// the same lists.  Ends with a CTA barrier: the tables and masks are complete when it returns.
template <int NC, int P>
__device__ int cluster_setup(const RecursionArgs<float> &args, const CSmem &S, long long q, int amax, int fmax,
                             int *err, int qa[3], int *nfrc_out, int rank)
{
    using G = CGeo<NC, P>;
    constexpr int NB0 = G::NB0, NZP = G::NZP, ZS = G::ZS;
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
    // z factor (g, hp) of atom J at cube z, or zeros outside the cube
    auto zfac = [&](int J, int z, int f0) {
        if (z >= NC) return make_float2(0.f, 0.f);
        const float *f2 = args.fac + (size_t)J * args.fac_stride + args.fac_off[2] + wstart[2] + z;
        return make_float2(f2[f0 * args.n[2]], f2[(f0 + 2) * args.n[2]]);
    };
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
    for (int it = threadIdx.x; it < 2 * nact * NZP; it += NTH) {
        const int i = it % NZP, t = (it / NZP) % nact, h = it / (NZP * nact);
        const int z = h * ZS + 2 * i;
        const int zend = h ? NC : ZS;
        const float2 u = z < zend ? zfac(S.rec[t].J, z, 0) : make_float2(0.f, 0.f);
        const float2 v = z + 1 < zend ? zfac(S.rec[t].J, z + 1, 0) : make_float2(0.f, 0.f);
        S.tz[((size_t)h * amax + t) * NZP + i] = make_float4(u.x, u.y, v.x, v.y);
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
        for (int it = threadIdx.x; it < 2 * nfrc * NZP; it += NTH) {
            const int i = it % NZP, fi = (it / NZP) % nfrc, h = it / (NZP * nfrc);
            const int z = h * ZS + 2 * i;
            const int zend = h ? NC : ZS;
            const int J = S.rec[S.ftl[fi]].J;
            const float2 u = z < zend ? zfac(J, z, 4) : make_float2(0.f, 0.f);
            const float2 v = z + 1 < zend ? zfac(J, z + 1, 4) : make_float2(0.f, 0.f);
            S.fz[((size_t)h * fmax + fi) * NZP + i] = make_float4(u.x, u.y, v.x, v.y);
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
        unsigned fb = 0u, z0 = 0u, z1 = 0u;
        for (int t = 32 * wd; t < min(nact, 32 * wd + 32); t++) {
            const unsigned bit = 1u << (t - 32 * wd);
            if (S.rec[t].fidx >= 0) fb |= bit;
            if (S.rec[t].lo[2] < ZS) z0 |= bit;
            if (S.rec[t].hi[2] >= ZS) z1 |= bit;
        }
        S.fbits[wd] = fb;
        S.zmask[wd] = z0;
        S.zmask[W + wd] = z1;
    }
    __syncthreads();   // tables and masks complete before any warp reads them
    *nfrc_out = nfrc;
    return nact;
}

// Projector contractions of two atoms per pass over the warp's z half, into its (slab, half) slots.
template <int NC, int P, int H>
__device__ __forceinline__ void cl_dots_pairs(unsigned msk, int wd, const CSmem &S, const float (&vz)[CGeo<NC, P>::ZL],
                                              int bl, int a, bool live, int lane, int amax)
{
    constexpr int NZP = CGeo<NC, P>::NZP, NB0 = CGeo<NC, P>::NB0, LEN = ZHalf<NC, P, H>::LEN;
    const float4 *tzh = S.tz + (size_t)H * amax * NZP;
    float *slot = S.slot + ((size_t)bl * 2 + H) * amax * 4;
    while (msk) {
        const int t0 = 32 * wd + __ffs(msk) - 1;
        msk &= msk - 1u;
        const bool two = msk != 0u;
        const int t1 = two ? 32 * wd + __ffs(msk) - 1 : t0;
        msk &= msk - 1u;
        const float4 *z0 = tzh + t0 * NZP;
        const float4 *z1 = two ? tzh + t1 * NZP : S.zero;
        float G0a = 0.f, H0a = 0.f, G0b = 0.f, H0b = 0.f;
        float G1a = 0.f, H1a = 0.f, G1b = 0.f, H1b = 0.f;
#pragma unroll
        for (int c = 0; c < LEN; c += 2) {
            const float4 p0 = z0[c >> 1], p1 = z1[c >> 1];
            G0a += p0.x * vz[c];
            H0a += p0.y * vz[c];
            G1a += p1.x * vz[c];
            H1a += p1.y * vz[c];
            if (c + 1 < LEN) {
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
            slot[t * 4 + (comp == 2 ? 3 : comp == 3 ? 2 : comp)] = (comp == 3 ? yv.y : yv.x) * red;
        }
    }
}

// KB update of two atoms per pass over the warp's z half: w += kappa_l chi (chi^T v) from the total dots.
template <int NC, int P, int H>
__device__ __forceinline__ void cl_update_pairs(unsigned msk, int wd, const CSmem &S, float (&w)[CGeo<NC, P>::ZL],
                                                int bl, int a, bool live, float kap0, float kap1, int amax)
{
    constexpr int NZP = CGeo<NC, P>::NZP, NB0 = CGeo<NC, P>::NB0, LEN = ZHalf<NC, P, H>::LEN;
    const float4 *tzh = S.tz + (size_t)H * amax * NZP;
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
        const float4 *z0 = tzh + t0 * NZP;
        const float4 *z1 = two ? tzh + t1 * NZP : S.zero;
#pragma unroll
        for (int c = 0; c < LEN; c += 2) {
            const float4 p0 = z0[c >> 1], p1 = z1[c >> 1];
            w[c] += p0.x * A1[0] + p0.y * A2[0] + p1.x * A1[1] + p1.y * A2[1];
            if (c + 1 < LEN) w[c + 1] += p0.z * A1[0] + p0.w * A2[0] + p1.z * A1[1] + p1.w * A2[1];
        }
    }
}

// Warp part of the contraction phase of step k for z half H: projector dots (need_dots) and force
// moments of the warp's (slab, half) into its slots.
template <int NC, int P, int H>
__device__ __forceinline__ void cluster_dots(const RecursionArgs<float> &args, const CSmem &S, const CThread<NC, P> &th,
                                             const float (&vz)[CGeo<NC, P>::ZL], bool need_dots, int amax, int fmax)
{
    using G = CGeo<NC, P>;
    constexpr int NZP = G::NZP, NB0 = G::NB0, LEN = ZHalf<NC, P, H>::LEN;
    const int W = (amax + 31) / 32;
    const int bl = th.bl, a = th.a, lane = th.lane;
    const bool live = th.live;
    if (!th.slab || !(need_dots || args.want_force)) return;
    const float4 *tzh = S.tz + (size_t)H * amax * NZP;
    const float4 *fzh = S.fz + (size_t)H * fmax * NZP;
    float *slot = S.slot + ((size_t)bl * 2 + H) * amax * 4;
    float *fslot = S.fslot + ((size_t)bl * 2 + H) * fmax * 12;
    for (int wd = 0; wd < W; wd++) {
        const unsigned all = S.ymask[bl * W + wd] & S.zmask[H * W + wd];
        const unsigned fb = S.fbits[wd];
        if (need_dots) cl_dots_pairs<NC, P, H>(all & ~fb, wd, S, vz, bl, a, live, lane, amax);
        unsigned msk = args.want_force ? (all & fb) : 0u;
        while (msk) {
            const int t = 32 * wd + __ffs(msk) - 1;
            msk &= msk - 1u;
            const int fidx = S.rec[t].fidx;
            const float4 *tz = tzh + t * NZP;
            const float4 *fz = fzh + fidx * NZP;
            float Ga = 0.f, Ha = 0.f, Gda = 0.f, Hda = 0.f, Gb = 0.f, Hb = 0.f, Gdb = 0.f, Hdb = 0.f;
#pragma unroll
            for (int c = 0; c < LEN; c += 2) {
                const float4 z = tz[c >> 1], zd = fz[c >> 1];
                Ga += z.x * vz[c];
                Ha += z.y * vz[c];
                Gda += zd.x * vz[c];
                Hda += zd.y * vz[c];
                if (c + 1 < LEN) {
                    Gb += z.z * vz[c + 1];
                    Hb += z.w * vz[c + 1];
                    Gdb += zd.z * vz[c + 1];
                    Hdb += zd.w * vz[c + 1];
                }
            }
            const float Gs = Ga + Gb, Hs = Ha + Hb, Gd = Gda + Gdb, Hd = Hda + Hdb;
            const float2 xv = live ? S.tx[t * NC + a] : make_float2(0.f, 0.f);
            const float2 yv = S.ty[t * NB0 + bl];
            float *sl = slot + t * 4;
            const float2 xd = live ? S.fx[fidx * NC + a] : make_float2(0.f, 0.f);
            const float2 yd = S.fy[fidx * NB0 + bl];
            const float v8[8] = {xv.x * Gs, xv.y * Gs, xv.x * Hs, xd.x * Gs, xv.x * Gd, xd.y * Gs, xv.y * Gd, xd.x * Hs};
            const float red = reduce8(v8, lane);
            const float v9 = wsum(xv.x * Hd);
            const int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
            float *fs = fslot + fidx * 12;
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

// CTA part of the contraction phase: fixed-order sums of this CTA's (slab, half) slots -> partial dots
// written into both CTAs' part[rank], and force moments added to A.  Ends before the cluster barrier X.
template <int NC, int P>
__device__ __forceinline__ void cluster_slot_sums(const RecursionArgs<float> &args, const CSmem &S, float *part_remote,
                                                  int rank, int k, bool need_dots, int nact, int nfrc, int amax,
                                                  int fmax)
{
    constexpr int NB0 = CGeo<NC, P>::NB0;
    const int W = (amax + 31) / 32;
    const int NTH = blockDim.x;
    if (need_dots) {
        float *mine = S.part + (size_t)rank * amax * 4;
        float *theirs = part_remote + (size_t)rank * amax * 4;
        for (int it = threadIdx.x; it < nact * 4; it += NTH) {
            const int t = it >> 2, comp = it & 3;
            const int wd = t >> 5;
            const unsigned bit = 1u << (t & 31);
            const bool in0 = S.zmask[wd] & bit, in1 = S.zmask[W + wd] & bit;
            float s = 0.f;
            for (int bb = 0; bb < NB0; bb++)
                if (S.ymask[bb * W + wd] & bit) {
                    if (in0) s += S.slot[(((size_t)bb * 2 + 0) * amax + t) * 4 + comp];
                    if (in1) s += S.slot[(((size_t)bb * 2 + 1) * amax + t) * 4 + comp];
                }
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
            const int wd = t >> 5;
            const unsigned bit = 1u << (t & 31);
            const bool in0 = S.zmask[wd] & bit, in1 = S.zmask[W + wd] & bit;
            double s = 0.0;
            bool any = false;
            for (int bb = 0; bb < NB0; bb++)
                if (S.ymask[bb * W + wd] & bit) {
                    if (in0) s += (double)S.fslot[(((size_t)bb * 2 + 0) * fmax + fi) * 12 + i];
                    if (in1) s += (double)S.fslot[(((size_t)bb * 2 + 1) * fmax + fi) * 12 + i];
                    any = true;
                }
            const int lm = i / 3, d = i % 3;
            if (any)
                atomicAdd(args.A + ((((size_t)k * natom + S.rec[t].J) * nproj + lm) * 3 + d),
                          S.chiq[4 * fi + lm] * args.Nnorm * s);
        }
    }
}

// Local part of Hhat v_k for z half H: stencil and diagonal into w (z neighbours from registers within
// the half, from the shared buffer across the split).
template <int NC, int P, int H>
__device__ __forceinline__ void cluster_local(const RecursionArgs<float> &args, const CSmem &S, const CThread<NC, P> &th,
                                              const float (&vz)[CGeo<NC, P>::ZL], float (&w)[CGeo<NC, P>::ZL],
                                              const float *drow, int plane_p)
{
    using G = CGeo<NC, P>;
    constexpr int NR = G::NR, ZL = G::ZL, Z0 = ZHalf<NC, P, H>::Z0, LEN = ZHalf<NC, P, H>::LEN;
    const float *col = S.U + (size_t)th.row * NC + th.a;   // (z = 0, this row, this x)
#pragma unroll
    for (int c = 0; c < ZL; c++) {
        const int zg = Z0 + c;
        const float x = vz[c];
        float t = 0.f;
#pragma unroll
        for (int j = 1; j <= P; j++) {
            float zp = 0.f, zm = 0.f;
            if (c + j < LEN) zp = vz[c + j];
            else if (zg + j < NC && c < LEN) zp = th.live ? col[(size_t)(zg + j) * NR * NC] : 0.f;
            if (c - j >= 0) zm = vz[c - j];
            else if (zg - j >= 0 && c < LEN) zm = th.live ? col[(size_t)(zg - j) * NR * NC] : 0.f;
            t += args.w[2][j - 1] * (zp + zm);
        }
#pragma unroll
        for (int j = 1; j <= P; j++) t = xpair(t, x, j, args.w[0][j - 1]);
        if (th.live && c < LEN) {
            const float *row = col + (size_t)zg * NR * NC;
#pragma unroll
            for (int j = 1; j <= P; j++) {
                const float yp = (th.yvalid >> (2 * j - 2)) & 1u ? row[j * NC] : 0.f;
                const float ym = (th.yvalid >> (2 * j - 1)) & 1u ? row[-j * NC] : 0.f;
                t += args.w[1][j - 1] * (yp + ym);
            }
            w[c] = t + drow[zg * plane_p] * x;
        } else {
            w[c] = 0.f;
        }
        // keep the loads of one z point from being hoisted into the next ones (register pressure)
        asm volatile("" ::: "memory");
    }
}

// KB term of Hhat v_k for z half H, added into w.
template <int NC, int P, int H>
__device__ __forceinline__ void cluster_kb(const CSmem &S, const CThread<NC, P> &th, float (&w)[CGeo<NC, P>::ZL],
                                           float kap0, float kap1, int amax)
{
    const int W = (amax + 31) / 32;
    if (!th.slab) return;
    for (int wd = 0; wd < W; wd++) {
        const unsigned all = S.ymask[th.bl * W + wd] & S.zmask[H * W + wd];
        cl_update_pairs<NC, P, H>(all, wd, S, w, th.bl, th.a, th.live, kap0, kap1, amax);
    }
}

// v_{k+1} = ca Hhat v_k - cb v_{k-1} for z half H: v_{k-1} from the CTA's scratch, v_k from the own
// rows (it moves into the scratch), v_{k+1} into the own rows, the partner's halo rows and vz.
// own, rem and pv point at z = 0 of this thread's own row, its row in the partner's buffer (when
// prow >= 0) and its scratch pencil; the z planes are reached by constant offsets.
template <int NC, int P, int H>
__device__ __forceinline__ void cluster_finish(const CThread<NC, P> &th, const float (&w)[CGeo<NC, P>::ZL],
                                               float (&vz)[CGeo<NC, P>::ZL], float *own, float *rem, float *pv,
                                               float ca, float cb, bool first)
{
    using G = CGeo<NC, P>;
    constexpr int NR = G::NR, NB0 = G::NB0, ZL = G::ZL, Z0 = ZHalf<NC, P, H>::Z0, LEN = ZHalf<NC, P, H>::LEN;
#pragma unroll
    for (int c = 0; c < ZL; c++) {
        if (th.live && c < LEN) {
            const int zg = Z0 + c;
            const float vkm1 = first ? 0.f : pv[zg * NB0 * 32];
            const float nv = ca * w[c] - cb * vkm1;
            pv[zg * NB0 * 32] = own[zg * NR * NC];
            own[zg * NR * NC] = nv;
            vz[c] = nv;
            if (th.prow >= 0) rem[zg * NR * NC] = nv;
        } else {
            vz[c] = 0.f;
        }
    }
}

template <int NC, int P>
__global__ void __launch_bounds__(CGeo<NC, P>::NW * 32, 1) cluster_kernel(const RecursionArgs<float> args, int amax,
                                                                         int fmax, int *err)
{
    using G = CGeo<NC, P>;
    constexpr int NZP = G::NZP, NR = G::NR, ZL = G::ZL;
    static_assert(P <= 6, "x shuffles assume a half-width of at most 6");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int partner = rank ^ 1;
    CSmem S;
    cluster_layout<NC, P>(smem_raw, amax, fmax, &S);
    float *U_remote = cluster.map_shared_rank(S.U, partner);
    float *part_remote = cluster.map_shared_rank(S.part, partner);
    float *vprev = args.scratch + (size_t)blockIdx.x * G::SCR;
    const CThread<NC, P> th(rank);
    const long long N_d = args.N_d;
    const size_t plane_p = (size_t)args.pn[0] * args.pn[1];
    const long long ncl = gridDim.x / 2;
    const long long cid = blockIdx.x / 2;
    const float kap0 = args.kappa[0], kap1 = args.kappa[1];
    float *own = S.U + (size_t)th.row * NC + th.a;
    float *rem = U_remote + (size_t)(th.prow >= 0 ? th.prow : 0) * NC + th.a;
    float *pv = vprev + (size_t)th.bl * 32 + th.lane;
    // the centre point (m, m, m) lies in z half mh, pencil index mc
    constexpr int m = (NC - 1) / 2;
    constexpr int mh = m < G::ZS ? 0 : 1, mc = m - mh * G::ZS;

    for (int i = threadIdx.x; i < NZP; i += blockDim.x) S.zero[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    cluster.sync();   // both CTAs are running before any write into the partner's shared memory

    for (long long q = args.q0 + cid; q < args.q1; q += ncl) {
        int qa[3], nfrc = 0;
        const int nact = cluster_setup<NC, P>(args, S, q, amax, fmax, err, qa, &nfrc, rank);
        if (nact < 0) continue;   // both CTAs see the same count
        // ---- v_0 = e_q (registers, own rows, the partner's halo rows) ----
        float vz[ZL];
        const int z0 = th.zh * G::ZS, len = th.zh ? NC - G::ZS : G::ZS;
#pragma unroll
        for (int c = 0; c < ZL; c++) {
            vz[c] = (th.centre_xy && th.zh == mh && c == mc) ? 1.0f : 0.0f;
            if (th.live && c < len) {
                S.U[((size_t)(z0 + c) * NR + th.row) * NC + th.a] = vz[c];
                if (th.prow >= 0) U_remote[((size_t)(z0 + c) * NR + th.prow) * NC + th.a] = vz[c];
            }
        }
        if (th.centre_xy && th.zh == mh) args.mu[q] = 1.0f;
        const float *drow = args.dpad + (size_t)qa[2] * plane_p + (size_t)(qa[1] + (th.slab ? th.b : 0)) * args.pn[0] +
                            qa[0] + (th.live ? th.a : 0);

        for (int k = 0; k <= args.K; k++) {
            const bool need_dots = k < args.K;
            if (th.zh == 0) cluster_dots<NC, P, 0>(args, S, th, vz, need_dots, amax, fmax);
            else cluster_dots<NC, P, 1>(args, S, th, vz, need_dots, amax, fmax);
            __syncthreads();
            cluster_slot_sums<NC, P>(args, S, part_remote, rank, k, need_dots, nact, nfrc, amax, fmax);
            cluster.sync();   // X: partial dots of both CTAs, the halo rows and the other z half are visible
            if (!need_dots) break;
            for (int it = threadIdx.x; it < nact * 4; it += blockDim.x) S.sd[it] = S.part[it] + S.part[amax * 4 + it];
            __syncthreads();
            const float ca = k == 0 ? 1.f : 2.f, cb = k == 0 ? 0.f : 1.f;
            float w[ZL];
            if (th.zh == 0) cluster_local<NC, P, 0>(args, S, th, vz, w, drow, (int)plane_p);
            else cluster_local<NC, P, 1>(args, S, th, vz, w, drow, (int)plane_p);
            // Y (arrive): this CTA's reads of v_k's buffer are done
            __syncwarp();
            auto y_token = cluster.barrier_arrive();
            if (th.zh == 0) cluster_kb<NC, P, 0>(S, th, w, kap0, kap1, amax);
            else cluster_kb<NC, P, 1>(S, th, w, kap0, kap1, amax);
            // Y (wait): both CTAs are done reading v_k's buffers
            __syncwarp();
            cluster.barrier_wait(std::move(y_token));
            if (th.zh == 0) cluster_finish<NC, P, 0>(th, w, vz, own, rem, pv, ca, cb, k == 0);
            else cluster_finish<NC, P, 1>(th, w, vz, own, rem, pv, ca, cb, k == 0);
            if (th.centre_xy && th.zh == mh) args.mu[(size_t)(k + 1) * N_d + q] = vz[mc];
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

long long cluster_scratch_floats(int nc)
{
    return nc == 29 ? (long long)CGeo<29, 6>::SCR : 0;
}

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
