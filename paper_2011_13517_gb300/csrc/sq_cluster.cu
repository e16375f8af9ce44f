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

// Row stride (floats) of the x factor rows: 32 x positions (zero past the cube) and 4 of padding, so
// the tensor-core fragment loads of one warp spread over the shared-memory banks.
constexpr int FAS = 36;

template <int NC, int P>
struct CGeo {
    static constexpr int NB0 = (NC + 1) / 2;              // y-slabs of rank 0 (rank 1 owns NC - NB0)
    static constexpr int NW = 2 * NB0;                    // warps per CTA: two z halves per slab
    static constexpr int NR = NB0 + P;                    // rows of the shared vector buffer
    static constexpr int HB = NB0 - P;                    // slab held in row 0 of rank 1's buffer
    static constexpr int ZS = (NC + 1) / 2;               // z split: half 0 holds z < ZS, half 1 the rest
    static constexpr int ZL = ZS;                         // pencil registers per thread
    static constexpr int NZP = 8;                         // float4 z-table entries per atom and half (16 z,
                                                          // the tensor-core path's two n-tiles)
    static constexpr int SCR = NC * NB0 * 32;             // floats of v_{k-1} scratch per CTA
    // z-plane stride of the shared vector buffer: at least NR rows plus a 32-wide read past the last row,
    // and 4 mod 32, so the tensor-core fragment accesses (8 z planes x 4 x, or 8 x by 4 z pairs) fall
    // in distinct banks
    static constexpr int PS = (NR * NC + 32 - NC - 4 + 31) / 32 * 32 + 4;
    // z planes of the buffer: the cube plus zero planes that the tensor-core path's whole 16-z tiles
    // of the upper half reach
    static constexpr int NZU = NC > ZS + 16 ? NC : ZS + 16;
    // the tensor-core fragment loads read x up to 31 in the last row of a plane and z up to ZS + 15
    static_assert(PS >= NR * NC && PS >= (NR - 1) * NC + 32 && PS % 32 == 4 && NZU >= ZS + 16, "buffer padding");
    static_assert(NC <= 32 && NC - NB0 + P <= NR && 2 * ZS >= NC && ZL <= 2 * NZP, "layout");
};
template <int NC, int P, int H>
struct ZHalf {
    static constexpr int Z0 = H * CGeo<NC, P>::ZS;                         // first z of the half
    static constexpr int LEN = H ? NC - CGeo<NC, P>::ZS : CGeo<NC, P>::ZS;  // z points of the half
};

struct CSmem {
    float *U;          // [NZU z][PS]: plane z holds [NR rows][NC x], own slabs of v_k plus the partner's P
                       // boundary slabs; zero outside them
    float *fa;         // [2 amax][FAS] x factor rows: row 2t = g, row 2t+1 = hp of active atom t, zero past NC
    float2 *ty;        // [amax+1][NB0]  (g, hp) along y, own slabs
    float4 *tz;        // [2][amax+1][NZP] per z half: (g[z], hp[z], g[z+1], hp[z+1]) from the half's first z
    float *fd;         // [2 (fmax+1)][FAS] x derivative rows (g', hp') of force slot fi, zero past NC; the
                       // rows of slot fmax stay zero
    float2 *fy;        // [fmax][NB0]
    float4 *fz;        // [2][fmax+1][NZP] (g', hp') pairs along z per half; entry fmax stays zero
    float *slot;       // [NB0][2][amax][4] per (slab, z half)
    float *fslot;      // [NB0][2][fmax][12]
    float *part;       // [2][amax][4]: partial dots of rank 0 and rank 1 (each written by its rank)
    float *sd;         // [amax+1][4]: total dots
    SlabRec *rec;      // [amax]
    double *chiq;      // [fmax][4]
    int *ftl;          // [fmax]
    unsigned *ymask;   // [NB0][W] own slabs
    unsigned *zmask;   // [2][W]: atoms whose z support meets half h
    unsigned *fbits;   // [W]
    float4 *zero;      // [NZP]
    int *scan;         // [40]
};

// x factors (g, hp) of active atom t at cube x position a (zeros for lanes past the cube)
__device__ __forceinline__ float2 xfac(const CSmem &S, int t, int a, bool live)
{
    return live ? make_float2(S.fa[2 * t * FAS + a], S.fa[(2 * t + 1) * FAS + a]) : make_float2(0.f, 0.f);
}

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
    // the atom tables have one more entry, index amax, which stays zero (padding of the tensor-core tiles)
    p = take(sizeof(float) * (size_t)G::NZU * G::PS);          if (s) s->U = (float *)p;
    p = take(sizeof(float) * (size_t)2 * (amax + 1) * FAS);    if (s) s->fa = (float *)p;
    p = take(sizeof(float2) * (size_t)(amax + 1) * G::NB0);    if (s) s->ty = (float2 *)p;
    p = take(sizeof(float4) * (size_t)2 * (amax + 1) * G::NZP); if (s) s->tz = (float4 *)p;
    p = take(sizeof(float) * (size_t)2 * (fmax + 1) * FAS);    if (s) s->fd = (float *)p;
    p = take(sizeof(float2) * (size_t)fmax * G::NB0);          if (s) s->fy = (float2 *)p;
    p = take(sizeof(float4) * (size_t)2 * (fmax + 1) * G::NZP); if (s) s->fz = (float4 *)p;
    p = take(sizeof(float) * (size_t)G::NB0 * 2 * amax * 4);   if (s) s->slot = (float *)p;
    p = take(sizeof(float) * (size_t)G::NB0 * 2 * fmax * 12);  if (s) s->fslot = (float *)p;
    p = take(sizeof(float) * (size_t)2 * amax * 4);            if (s) s->part = (float *)p;
    p = take(sizeof(float) * (size_t)(amax + 1) * 4);          if (s) s->sd = (float *)p;
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
    for (int it = threadIdx.x; it < nact * 2 * FAS; it += NTH) {
        const int o = it % FAS, row = it / FAS;
        float v = 0.f;
        if (o < NC)
            v = args.fac[(size_t)S.rec[row >> 1].J * args.fac_stride + args.fac_off[0] + wstart[0] + o +
                         (row & 1) * 2 * args.n[0]];
        S.fa[it] = v;
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
        S.tz[((size_t)h * (amax + 1) + t) * NZP + i] = make_float4(u.x, u.y, v.x, v.y);
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
        for (int it = threadIdx.x; it < nfrc * 2 * FAS; it += NTH) {
            const int o = it % FAS, row = it / FAS;
            float v = 0.f;
            if (o < NC)
                v = args.fac[(size_t)S.rec[S.ftl[row >> 1]].J * args.fac_stride + args.fac_off[0] + wstart[0] + o +
                             (4 + 2 * (row & 1)) * args.n[0]];
            S.fd[it] = v;
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
            S.fz[((size_t)h * (fmax + 1) + fi) * NZP + i] = make_float4(u.x, u.y, v.x, v.y);
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
    const float4 *tzh = S.tz + (size_t)H * (amax + 1) * NZP;
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
        const float2 x0 = xfac(S, t0, a, live), x1 = xfac(S, t1, a, live);
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
    const float4 *tzh = S.tz + (size_t)H * (amax + 1) * NZP;
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
            const float2 xv = xfac(S, t, a, live);
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

// ---- projector term on the tensor cores ----------------------------------------------------------
//
// Per warp (slab b, z half) the projector term is two small dense products over the separable
// factors of the atoms L whose support meets the warp's slab and half (two rows per atom: its x
// factors g and hp):
//   dots    C[f][z] = sum_x FA[f][x] v(x, b, z)          (16-row tiles of f, k = x, n = z),
//           then per atom the z factors and the y factor of slab b (CUDA cores);
//   update  W[x][z] = sum_f FA[f][x] Q_b[f][z]           (m = x, k = f, n = z), with
//           Q_b[2t][z] = (kappa_0 s_t g_y + kappa_1 py_t hp_y) g_z + kappa_1 pz_t g_y hp_z and
//           Q_b[2t+1][z] = kappa_1 px_t g_y g_z from the dots (s, px, py, pz) of atom t.
// Both run as m16n8k8 TF32 warp MMAs with FP32 accumulation, each operand split into a TF32 head and
// a TF32 tail (x = hi + lo, |x - hi - lo| <= 2^-22 |x|) and the product taken as lo*hi + hi*lo +
// hi*hi ("3xTF32"), so the products keep about FP32 accuracy.  Fragment layouts of m16n8k8 .tf32
// (g = lane / 4, t = lane % 4): A a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4); B b0 (k t, n g),
// b1 (k t+4, n g); C c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1).

__device__ __forceinline__ unsigned to_tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo)
{
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d += (ah + al)(bh + bl) without the al bl term, small terms first
__device__ __forceinline__ void mma3(float (&d)[4], const unsigned (&ah)[4], const unsigned (&al)[4],
                                     const unsigned (&bh)[2], const unsigned (&bl)[2])
{
    mma_tf32(d, al, bh);
    mma_tf32(d, ah, bl);
    mma_tf32(d, ah, bh);
}

// Largest atom list of one warp that the tensor-core path takes (two registers of list entries); a
// longer list sets error 3, and the host redoes the launch with the CUDA-core projector term.
constexpr int kMmaMaxList = 64;

// The warp's ordered list of atoms whose support meets slab bl and z half H: lane j holds entry j in
// l0 and entry 32 + j in l1 (-1 past the end).  Returns the list length (the same in every lane).
template <int H>
__device__ __forceinline__ int warp_atom_list(const CSmem &S, int bl, int W, int lane, int &l0, int &l1)
{
    int n = 0;
    l0 = -1;
    l1 = -1;
    for (int wd = 0; wd < W; wd++) {
        const unsigned msk = S.ymask[bl * W + wd] & S.zmask[H * W + wd];
        const int c = __popc(msk);
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int r = lane + 32 * e - n;
            if (r >= 0 && r < c) {
                unsigned mm = msk;
                for (int i = 0; i < r; i++) mm &= mm - 1u;
                const int v = 32 * wd + __ffs(mm) - 1;
                if (e == 0) l0 = v;
                else l1 = v;
            }
        }
        n += c;
    }
    return n;
}

// The force atoms (projectors nonzero at the column's centre) among the warp's list: lane j holds the
// atom index of entry j (-1 past the end).  Returns the count; a count above 32 is cut to 32 with
// error 3 (the host then redoes the launch on the CUDA-core path).
template <int H>
__device__ __forceinline__ int warp_force_list(const CSmem &S, int bl, int W, int lane, int &lf, int *err)
{
    int n = 0;
    lf = -1;
    for (int wd = 0; wd < W; wd++) {
        const unsigned msk = S.ymask[bl * W + wd] & S.zmask[H * W + wd] & S.fbits[wd];
        const int c = __popc(msk);
        const int r = lane - n;
        if (r >= 0 && r < c) {
            unsigned mm = msk;
            for (int i = 0; i < r; i++) mm &= mm - 1u;
            lf = 32 * wd + __ffs(mm) - 1;
        }
        n += c;
    }
    if (n > 32) {
        if (lane == 0) atomicExch(err, 3);
        n = 32;
    }
    return n;
}

// Projector dots of every atom in the warp's list (nL <= kMmaMaxList) into the warp's slots, from v_k
// in the warp's own rows of U.  With want_force also the force moments of the force atoms in the list
// (lf, nF): the rows g and hp of a force atom take two more z sums (with g'_z and hp'_z), and extra
// 16-row tiles carry the x derivative rows g' and hp' of the force atoms, so every one of the twelve
// contractions (d_d chi_lm)^T v of a force atom comes out of the same MMAs.
template <int NC, int P, int H>
__device__ __forceinline__ void cl_dots_mma(const CSmem &S, const CThread<NC, P> &th, int l0, int l1, int nL, int lf,
                                            int nF, int amax, int fmax, bool want_force, bool write_dots)
{
    using G = CGeo<NC, P>;
    constexpr int NR = G::NR, NZP = G::NZP, NB0 = G::NB0, Z0 = ZHalf<NC, P, H>::Z0, LEN = ZHalf<NC, P, H>::LEN;
    const int g = th.lane >> 2, t = th.lane & 3;
    const float4 *tzh = S.tz + (size_t)H * (amax + 1) * NZP;
    const float4 *fzh = S.fz + (size_t)H * (fmax + 1) * NZP;
    float *slot = S.slot + ((size_t)th.bl * 2 + H) * amax * 4;
    float *fslot = S.fslot + ((size_t)th.bl * 2 + H) * fmax * 12;
    const float *urow = S.U + (size_t)th.row * NC;   // (z 0, own row, x 0)
    for (int mt = 0; 8 * mt < nL; mt++) {
        const int src = mt < 4 ? l0 : l1;
        const int iA = 8 * mt + (g >> 1), iB = iA + 4;
        // entries past the list take the zero atom (index amax)
        const bool okA = iA < nL, okB = iB < nL;
        const int sA = __shfl_sync(0xffffffffu, src, iA & 31), sB = __shfl_sync(0xffffffffu, src, iB & 31);
        const int tA = okA ? sA : amax, tB = okB ? sB : amax;
        const float *rA = S.fa + (size_t)(2 * tA + (g & 1)) * FAS;
        const float *rB = S.fa + (size_t)(2 * tB + (g & 1)) * FAS;
        float acc[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ks++) {
            const int x0 = 8 * ks + t, x1 = x0 + 4;
            unsigned ah[4], al[4];
            split_tf32(rA[x0], ah[0], al[0]);
            split_tf32(rB[x0], ah[1], al[1]);
            split_tf32(rA[x1], ah[2], al[2]);
            split_tf32(rB[x1], ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
                // v at x = 8 ks + t (+4), z = Z0 + 8 nt + g: past the cube in x the loads reach the next
                // row and past the half in z the other half or the zero planes, all finite; their
                // products meet zero x factors (FA) or zero z factors (tz) below
                const float *col = urow + (size_t)(Z0 + 8 * nt + g) * CGeo<NC, P>::PS;
                unsigned bh[2], bo[2];
                split_tf32(col[x0], bh[0], bo[0]);
                split_tf32(col[x1], bh[1], bo[1]);
                mma3(acc[nt], ah, al, bh, bo);
            }
        }
        // z factors of the lane's two rows (z = 8 nt + 2t and 8 nt + 2t + 1 of the half): sums with g_z
        // and hp_z, and for force atoms with g'_z and hp'_z (slot fmax: zeros)
        const int fA = want_force && okA ? S.rec[tA].fidx : -1, fB = want_force && okB ? S.rec[tB].fidx : -1;
        const int zA = fA >= 0 ? fA : fmax, zB = fB >= 0 ? fB : fmax;
        float sA1 = 0.f, sA2 = 0.f, sB1 = 0.f, sB2 = 0.f, sA3 = 0.f, sA4 = 0.f, sB3 = 0.f, sB4 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
            const float4 pa = tzh[tA * NZP + 4 * nt + t], pb = tzh[tB * NZP + 4 * nt + t];
            sA1 += pa.x * acc[nt][0] + pa.z * acc[nt][1];
            sA2 += pa.y * acc[nt][0] + pa.w * acc[nt][1];
            sB1 += pb.x * acc[nt][2] + pb.z * acc[nt][3];
            sB2 += pb.y * acc[nt][2] + pb.w * acc[nt][3];
            if (want_force) {
                const float4 qa = fzh[zA * NZP + 4 * nt + t], qb = fzh[zB * NZP + 4 * nt + t];
                sA3 += qa.x * acc[nt][0] + qa.z * acc[nt][1];
                sA4 += qa.y * acc[nt][0] + qa.w * acc[nt][1];
                sB3 += qb.x * acc[nt][2] + qb.z * acc[nt][3];
                sB4 += qb.y * acc[nt][2] + qb.w * acc[nt][3];
            }
        }
        // sum over the four lanes of a row pair (they hold different z)
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            sA1 += __shfl_xor_sync(0xffffffffu, sA1, o);
            sA2 += __shfl_xor_sync(0xffffffffu, sA2, o);
            sB1 += __shfl_xor_sync(0xffffffffu, sB1, o);
            sB2 += __shfl_xor_sync(0xffffffffu, sB2, o);
            if (want_force) {
                sA3 += __shfl_xor_sync(0xffffffffu, sA3, o);
                sA4 += __shfl_xor_sync(0xffffffffu, sA4, o);
                sB3 += __shfl_xor_sync(0xffffffffu, sB3, o);
                sB4 += __shfl_xor_sync(0xffffffffu, sB4, o);
            }
        }
        // row g: x factor g (g even) or hp (g odd) of atom A; row g + 8 likewise of atom B
        if (t < 2 && (t == 0 ? okA : okB)) {
            const int at = t == 0 ? tA : tB, fi = t == 0 ? fA : fB;
            const float s1 = t == 0 ? sA1 : sB1, s2 = t == 0 ? sA2 : sB2;
            const float s3 = t == 0 ? sA3 : sB3, s4 = t == 0 ? sA4 : sB4;
            const float2 yv = S.ty[at * NB0 + th.bl];
            float *sl = slot + at * 4;
            if ((g & 1) == 0) {
                if (write_dots) {
                    sl[0] = yv.x * s1;   // s
                    sl[2] = yv.y * s1;   // p_y
                    sl[3] = yv.x * s2;   // p_z
                }
                if (fi >= 0) {
                    const float2 yd = S.fy[fi * NB0 + th.bl];
                    float *fs = fslot + fi * 12;
                    fs[1] = yd.x * s1;    // s d/dy
                    fs[7] = yd.y * s1;    // p_y d/dy
                    fs[10] = yd.x * s2;   // p_z d/dy
                    fs[2] = yv.x * s3;    // s d/dz
                    fs[8] = yv.y * s3;    // p_y d/dz
                    fs[11] = yv.x * s4;   // p_z d/dz
                }
            } else {
                if (write_dots) sl[1] = yv.x * s1;   // p_x
                if (fi >= 0) {
                    const float2 yd = S.fy[fi * NB0 + th.bl];
                    float *fs = fslot + fi * 12;
                    fs[4] = yd.x * s1;    // p_x d/dy
                    fs[5] = yv.x * s3;    // p_x d/dz
                }
            }
        }
    }
    if (!want_force) return;
    // x derivative rows of the force atoms: row g of a tile is g' (g even) or hp' (g odd) of force atom
    // 8 mt + g/2, row g + 8 of force atom 8 mt + 4 + g/2
    for (int mt = 0; 8 * mt < nF; mt++) {
        const int iA = 8 * mt + (g >> 1), iB = iA + 4;
        const bool okA = iA < nF, okB = iB < nF;
        const int sA = __shfl_sync(0xffffffffu, lf, iA & 31), sB = __shfl_sync(0xffffffffu, lf, iB & 31);
        const int tA = okA ? sA : amax, tB = okB ? sB : amax;
        const int fA = okA ? S.rec[sA].fidx : fmax, fB = okB ? S.rec[sB].fidx : fmax;
        const float *rA = S.fd + (size_t)(2 * fA + (g & 1)) * FAS;
        const float *rB = S.fd + (size_t)(2 * fB + (g & 1)) * FAS;
        float acc[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ks++) {
            const int x0 = 8 * ks + t, x1 = x0 + 4;
            unsigned ah[4], al[4];
            split_tf32(rA[x0], ah[0], al[0]);
            split_tf32(rB[x0], ah[1], al[1]);
            split_tf32(rA[x1], ah[2], al[2]);
            split_tf32(rB[x1], ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
                const float *col = urow + (size_t)(Z0 + 8 * nt + g) * CGeo<NC, P>::PS;
                unsigned bh[2], bo[2];
                split_tf32(col[x0], bh[0], bo[0]);
                split_tf32(col[x1], bh[1], bo[1]);
                mma3(acc[nt], ah, al, bh, bo);
            }
        }
        float sA1 = 0.f, sA2 = 0.f, sB1 = 0.f, sB2 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
            const float4 pa = tzh[tA * NZP + 4 * nt + t], pb = tzh[tB * NZP + 4 * nt + t];
            sA1 += pa.x * acc[nt][0] + pa.z * acc[nt][1];
            sA2 += pa.y * acc[nt][0] + pa.w * acc[nt][1];
            sB1 += pb.x * acc[nt][2] + pb.z * acc[nt][3];
            sB2 += pb.y * acc[nt][2] + pb.w * acc[nt][3];
        }
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            sA1 += __shfl_xor_sync(0xffffffffu, sA1, o);
            sA2 += __shfl_xor_sync(0xffffffffu, sA2, o);
            sB1 += __shfl_xor_sync(0xffffffffu, sB1, o);
            sB2 += __shfl_xor_sync(0xffffffffu, sB2, o);
        }
        if (t < 2 && (t == 0 ? okA : okB)) {
            const int at = t == 0 ? tA : tB, fi = t == 0 ? fA : fB;
            const float s1 = t == 0 ? sA1 : sB1, s2 = t == 0 ? sA2 : sB2;
            const float2 yv = S.ty[at * NB0 + th.bl];
            float *fs = fslot + fi * 12;
            if ((g & 1) == 0) {
                fs[0] = yv.x * s1;   // s d/dx
                fs[6] = yv.y * s1;   // p_y d/dx
                fs[9] = yv.x * s2;   // p_z d/dx
            } else {
                fs[3] = yv.x * s1;   // p_x d/dx
            }
        }
    }
}

// Projector term of Hhat v_k over the warp's (slab, half) block on the tensor cores: acc[mt][nt]
// holds W[x][z] for x = 16 mt + (g, g+8) and z = 8 nt + (2t, 2t+1) of the half.
template <int NC, int P, int H>
__device__ __forceinline__ void cl_kb_mma(const CSmem &S, const CThread<NC, P> &th, int l0, int l1, int nL,
                                          float kap0, float kap1, int amax, float (&acc)[2][2][4])
{
    using G = CGeo<NC, P>;
    constexpr int NZP = G::NZP, NB0 = G::NB0;
    const int g = th.lane >> 2, t = th.lane & 3, fac = t & 1;
    const float2 *tzh = reinterpret_cast<const float2 *>(S.tz + (size_t)H * (amax + 1) * NZP);
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[mt][nt][i] = 0.f;
    for (int ks = 0; 4 * ks < nL; ks++) {
        // rows 8 ks + j of FA / Q: atom 4 ks + j/2, factor j % 2; this lane holds j = t and t + 4
        const int src = ks < 8 ? l0 : l1;
        const int i0 = 4 * ks + (t >> 1), i1 = i0 + 2;
        // entries past the list take the zero atom (index amax)
        const int s0 = __shfl_sync(0xffffffffu, src, i0 & 31), s1 = __shfl_sync(0xffffffffu, src, i1 & 31);
        const int t0 = i0 < nL ? s0 : amax, t1 = i1 < nL ? s1 : amax;
        // Q rows of the two atoms: Q(z) = c1 g_z(z) + c2 hp_z(z)
        float c1[2], c2[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int at = r ? t1 : t0;
            const float4 sv = *reinterpret_cast<const float4 *>(S.sd + 4 * at);
            const float2 yv = S.ty[at * NB0 + th.bl];
            if (fac == 0) {
                c1[r] = kap0 * sv.x * yv.x + kap1 * sv.z * yv.y;
                c2[r] = kap1 * sv.w * yv.x;
            } else {
                c1[r] = kap1 * sv.y * yv.x;
                c2[r] = 0.f;
            }
        }
        unsigned bh[2][2], bo[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
            const int zl = 8 * nt + g;   // < 2 NZP: the half's z table covers it (zeros past the half)
            const float2 p0 = tzh[t0 * 2 * NZP + zl], p1 = tzh[t1 * 2 * NZP + zl];
            split_tf32(c1[0] * p0.x + c2[0] * p0.y, bh[nt][0], bo[nt][0]);
            split_tf32(c1[1] * p1.x + c2[1] * p1.y, bh[nt][1], bo[nt][1]);
        }
        const float *r0 = S.fa + (size_t)(2 * t0 + fac) * FAS;
        const float *r1 = S.fa + (size_t)(2 * t1 + fac) * FAS;
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            const int x = 16 * mt + g;
            unsigned ah[4], al[4];
            split_tf32(r0[x], ah[0], al[0]);
            split_tf32(r0[x + 8], ah[1], al[1]);
            split_tf32(r1[x], ah[2], al[2]);
            split_tf32(r1[x + 8], ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < 2; nt++) mma3(acc[mt][nt], ah, al, bh[nt], bo[nt]);
        }
    }
}

// Warp part of the contraction phase of step k for z half H: projector dots (need_dots) and force
// moments of the warp's (slab, half) into its slots.  With dots_fma false the dots of every atom come
// from the tensor-core pass (cl_dots_mma) and this pass adds only the force moments.
template <int NC, int P, int H>
__device__ __forceinline__ void cluster_dots(const RecursionArgs<float> &args, const CSmem &S, const CThread<NC, P> &th,
                                             const float (&vz)[CGeo<NC, P>::ZL], bool need_dots, bool dots_fma,
                                             int amax, int fmax)
{
    using G = CGeo<NC, P>;
    constexpr int NZP = G::NZP, NB0 = G::NB0, LEN = ZHalf<NC, P, H>::LEN;
    const int W = (amax + 31) / 32;
    const int bl = th.bl, a = th.a, lane = th.lane;
    const bool live = th.live;
    if (!th.slab || !(need_dots || args.want_force)) return;
    const float4 *tzh = S.tz + (size_t)H * (amax + 1) * NZP;
    const float4 *fzh = S.fz + (size_t)H * (fmax + 1) * NZP;
    float *slot = S.slot + ((size_t)bl * 2 + H) * amax * 4;
    float *fslot = S.fslot + ((size_t)bl * 2 + H) * fmax * 12;
    for (int wd = 0; wd < W; wd++) {
        const unsigned all = S.ymask[bl * W + wd] & S.zmask[H * W + wd];
        const unsigned fb = S.fbits[wd];
        const bool sl_on = need_dots && dots_fma;
        if (sl_on) cl_dots_pairs<NC, P, H>(all & ~fb, wd, S, vz, bl, a, live, lane, amax);
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
            const float2 xv = xfac(S, t, a, live);
            const float2 yv = S.ty[t * NB0 + bl];
            float *sl = slot + t * 4;
            const float2 xd = live ? make_float2(S.fd[2 * fidx * FAS + a], S.fd[(2 * fidx + 1) * FAS + a])
                                   : make_float2(0.f, 0.f);
            const float2 yd = S.fy[fidx * NB0 + bl];
            const float v8[8] = {xv.x * Gs, xv.y * Gs, xv.x * Hs, xd.x * Gs, xv.x * Gd, xd.y * Gs, xv.y * Gd, xd.x * Hs};
            const float red = reduce8(v8, lane);
            const float v9 = wsum(xv.x * Hd);
            const int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
            float *fs = fslot + fidx * 12;
            if ((lane & 3) == 0) {
                switch (idx) {
                case 0: if (sl_on) { sl[0] = yv.x * red; sl[2] = yv.y * red; }
                        fs[1] = yd.x * red; fs[7] = yd.y * red; break;
                case 1: if (sl_on) sl[1] = yv.x * red;
                        fs[4] = yd.x * red; break;
                case 2: if (sl_on) sl[3] = yv.x * red;
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
            else if (zg + j < NC && c < LEN) zp = th.live ? col[(size_t)(zg + j) * CGeo<NC, P>::PS] : 0.f;
            if (c - j >= 0) zm = vz[c - j];
            else if (zg - j >= 0 && c < LEN) zm = th.live ? col[(size_t)(zg - j) * CGeo<NC, P>::PS] : 0.f;
            t += args.w[2][j - 1] * (zp + zm);
        }
#pragma unroll
        for (int j = 1; j <= P; j++) t = xpair(t, x, j, args.w[0][j - 1]);
        if (th.live && c < LEN) {
            const float *row = col + (size_t)zg * CGeo<NC, P>::PS;
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
            pv[zg * NB0 * 32] = own[zg * CGeo<NC, P>::PS];
            own[zg * CGeo<NC, P>::PS] = nv;
            vz[c] = nv;
            if (th.prow >= 0) rem[zg * CGeo<NC, P>::PS] = nv;
        } else {
            vz[c] = 0.f;
        }
    }
}

// Tensor-core path, first half of v_{k+1} = ca Hhat v_k - cb v_{k-1} for z half H: w (the local part)
// becomes ca w - cb v_{k-1}, and v_k moves from the registers into the scratch in place of v_{k-1}.
template <int NC, int P, int H>
__device__ __forceinline__ void cluster_prefinish(const CThread<NC, P> &th, float (&w)[CGeo<NC, P>::ZL],
                                                  const float (&vz)[CGeo<NC, P>::ZL], float *pv, float ca, float cb,
                                                  bool first)
{
    using G = CGeo<NC, P>;
    constexpr int NB0 = G::NB0, ZL = G::ZL, Z0 = ZHalf<NC, P, H>::Z0, LEN = ZHalf<NC, P, H>::LEN;
#pragma unroll
    for (int c = 0; c < ZL; c++) {
        if (th.live && c < LEN) {
            const int zg = Z0 + c;
            const float vkm1 = first ? 0.f : pv[zg * NB0 * 32];
            pv[zg * NB0 * 32] = vz[c];
            w[c] = ca * w[c] - cb * vkm1;
        }
    }
}

// The warp's pencil of v_k from its own rows (zeros past the cube).
template <int NC, int P>
__device__ __forceinline__ void load_pencil(const CThread<NC, P> &th, const float *own, float (&v)[CGeo<NC, P>::ZL])
{
    using G = CGeo<NC, P>;
    constexpr int NR = G::NR, ZL = G::ZL;
    const int z0 = th.zh * G::ZS, len = th.zh ? NC - G::ZS : G::ZS;
#pragma unroll
    for (int c = 0; c < ZL; c++) v[c] = (th.live && c < len) ? own[(z0 + c) * CGeo<NC, P>::PS] : 0.f;
}

// Tensor-core path, second half (after the cluster barrier Y): the own rows receive w, then ca times
// the projector term at the MMA fragment positions; the finished pencils go to the partner's halo rows
// and, for the thread at the column's centre, mu_{k+1} to muk.
template <int NC, int P, int H>
__device__ __forceinline__ void cluster_finish_mma(const CSmem &S, const CThread<NC, P> &th,
                                                   const float (&w)[CGeo<NC, P>::ZL], const float (&acc)[2][2][4],
                                                   float *own, float *rem, float ca, float *muk, int mc)
{
    using G = CGeo<NC, P>;
    constexpr int NR = G::NR, ZL = G::ZL, Z0 = ZHalf<NC, P, H>::Z0, LEN = ZHalf<NC, P, H>::LEN;
#pragma unroll
    for (int c = 0; c < ZL; c++)
        if (th.live && c < LEN) own[(Z0 + c) * CGeo<NC, P>::PS] = w[c];
    __syncwarp();
    if (th.slab) {
        const int g = th.lane >> 2, t = th.lane & 3;
        float *base = S.U + (size_t)th.row * NC;
#pragma unroll
        for (int mt = 0; mt < 2; mt++)
#pragma unroll
            for (int nt = 0; nt < 2; nt++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int x = 16 * mt + g + ((i & 2) ? 8 : 0), zl = 8 * nt + 2 * t + (i & 1);
                    if (x < NC && zl < LEN) base[(size_t)(Z0 + zl) * CGeo<NC, P>::PS + x] += ca * acc[mt][nt][i];
                }
    }
    __syncwarp();
    if (th.live && (th.prow >= 0 || muk)) {
#pragma unroll
        for (int c = 0; c < ZL; c++) {
            if (c < LEN) {
                const float nv = own[(Z0 + c) * CGeo<NC, P>::PS];
                if (th.prow >= 0) rem[(Z0 + c) * CGeo<NC, P>::PS] = nv;
                if (muk && c == mc) *muk = nv;
            }
        }
    }
}

template <int NC, int P, bool MMA>
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
    // zero the vector buffer (rows and planes that no slab fills stay zero) and the zero atom's entries
    for (int i = threadIdx.x; i < G::NZU * G::PS; i += blockDim.x) S.U[i] = 0.f;
    for (int i = threadIdx.x; i < 2 * FAS; i += blockDim.x) S.fa[2 * amax * FAS + i] = 0.f;
    for (int i = threadIdx.x; i < G::NB0; i += blockDim.x) S.ty[(size_t)amax * G::NB0 + i] = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < 2 * NZP; i += blockDim.x)
        S.tz[((size_t)(i / NZP) * (amax + 1) + amax) * NZP + i % NZP] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i < 4; i += blockDim.x) S.sd[4 * amax + i] = 0.f;
    for (int i = threadIdx.x; i < 2 * FAS; i += blockDim.x) S.fd[2 * fmax * FAS + i] = 0.f;
    for (int i = threadIdx.x; i < 2 * NZP; i += blockDim.x)
        S.fz[((size_t)(i / NZP) * (fmax + 1) + fmax) * NZP + i % NZP] = make_float4(0.f, 0.f, 0.f, 0.f);
    cluster.sync();   // both CTAs are running before any write into the partner's shared memory

    for (long long q = args.q0 + cid; q < args.q1; q += ncl) {
        int qa[3], nfrc = 0;
        const int nact = cluster_setup<NC, P>(args, S, q, amax, fmax, err, qa, &nfrc, rank);
        if (nact < 0) continue;   // both CTAs see the same count
        // ---- v_0 = e_q (own rows, the partner's halo rows; registers on the CUDA-core path) ----
        float vz[ZL];
        const int z0 = th.zh * G::ZS, len = th.zh ? NC - G::ZS : G::ZS;
#pragma unroll
        for (int c = 0; c < ZL; c++) {
            vz[c] = (th.centre_xy && th.zh == mh && c == mc) ? 1.0f : 0.0f;
            if (th.live && c < len) {
                S.U[(size_t)(z0 + c) * G::PS + th.row * NC + th.a] = vz[c];
                if (th.prow >= 0) U_remote[(size_t)(z0 + c) * G::PS + th.prow * NC + th.a] = vz[c];
            }
        }
        if (th.centre_xy && th.zh == mh) args.mu[q] = 1.0f;
        __syncwarp();   // the tensor-core dots read the warp's own rows of v_0
        const float *drow = args.dpad + (size_t)qa[2] * plane_p + (size_t)(qa[1] + (th.slab ? th.b : 0)) * args.pn[0] +
                            qa[0] + (th.live ? th.a : 0);
        float *mu_out = (th.centre_xy && th.zh == mh) ? args.mu + q : nullptr;

        if constexpr (MMA) {
            // the warp's atom list; a longer one than the path takes is reported (the host then redoes the
            // launch on the CUDA-core path) and cut, so every index stays in range
            int l0 = -1, l1 = -1, nL = 0, lf = -1, nF = 0;
            if (th.slab) {
                const int W = (amax + 31) / 32;
                nL = th.zh == 0 ? warp_atom_list<0>(S, th.bl, W, th.lane, l0, l1)
                                : warp_atom_list<1>(S, th.bl, W, th.lane, l0, l1);
                if (nL > kMmaMaxList) {
                    if (th.lane == 0) atomicExch(err, 3);
                    nL = kMmaMaxList;
                }
                if (args.want_force)
                    nF = th.zh == 0 ? warp_force_list<0>(S, th.bl, W, th.lane, lf, err)
                                    : warp_force_list<1>(S, th.bl, W, th.lane, lf, err);
            }
            for (int k = 0; k <= args.K; k++) {
                const bool need_dots = k < args.K;
                if (need_dots || args.want_force) {
                    const bool wf = args.want_force != 0;
                    if (th.zh == 0) cl_dots_mma<NC, P, 0>(S, th, l0, l1, nL, lf, nF, amax, fmax, wf, need_dots);
                    else cl_dots_mma<NC, P, 1>(S, th, l0, l1, nL, lf, nF, amax, fmax, wf, need_dots);
                }
                __syncthreads();
                cluster_slot_sums<NC, P>(args, S, part_remote, rank, k, need_dots, nact, nfrc, amax, fmax);
                cluster.sync();   // X: partial dots of both CTAs, the halo rows and the other z half are visible
                if (!need_dots) break;
                for (int it = threadIdx.x; it < nact * 4; it += blockDim.x) S.sd[it] = S.part[it] + S.part[amax * 4 + it];
                __syncthreads();
                const float ca = k == 0 ? 1.f : 2.f, cb = k == 0 ? 0.f : 1.f;
                float w[ZL];
                {
                    float vk[ZL];
                    load_pencil<NC, P>(th, own, vk);
                    if (th.zh == 0) {
                        cluster_local<NC, P, 0>(args, S, th, vk, w, drow, (int)plane_p);
                        cluster_prefinish<NC, P, 0>(th, w, vk, pv, ca, cb, k == 0);
                    } else {
                        cluster_local<NC, P, 1>(args, S, th, vk, w, drow, (int)plane_p);
                        cluster_prefinish<NC, P, 1>(th, w, vk, pv, ca, cb, k == 0);
                    }
                }
                // Y (arrive): this CTA's reads of v_k's buffer are done
                __syncwarp();
                auto y_token = cluster.barrier_arrive();
                float acc[2][2][4];
                if (th.zh == 0) cl_kb_mma<NC, P, 0>(S, th, l0, l1, nL, kap0, kap1, amax, acc);
                else cl_kb_mma<NC, P, 1>(S, th, l0, l1, nL, kap0, kap1, amax, acc);
                // Y (wait): both CTAs are done reading v_k's buffers
                __syncwarp();
                cluster.barrier_wait(std::move(y_token));
                float *muk = mu_out ? mu_out + (size_t)(k + 1) * N_d : nullptr;
                if (th.zh == 0) cluster_finish_mma<NC, P, 0>(S, th, w, acc, own, rem, ca, muk, mc);
                else cluster_finish_mma<NC, P, 1>(S, th, w, acc, own, rem, ca, muk, mc);
            }
        } else {
            for (int k = 0; k <= args.K; k++) {
                const bool need_dots = k < args.K;
                if (th.zh == 0) cluster_dots<NC, P, 0>(args, S, th, vz, need_dots, true, amax, fmax);
                else cluster_dots<NC, P, 1>(args, S, th, vz, need_dots, true, amax, fmax);
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
                if (mu_out) mu_out[(size_t)(k + 1) * N_d] = vz[mc];
            }
        }
    }
    cluster.sync();   // no CTA leaves while its partner may still write into its shared memory
}

template <int NC, int P, bool MMA>
cudaError_t cluster_config(int amax, int fmax, size_t *smem, int *max_clusters)
{
    using G = CGeo<NC, P>;
    const size_t sm = cluster_layout<NC, P>(nullptr, amax, fmax, nullptr);
    *smem = sm;
    auto kern = cluster_kernel<NC, P, MMA>;
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

template <int NC, int P, bool MMA>
cudaError_t cluster_launch(const RecursionArgs<float> &args, int amax, int fmax, int nclusters, size_t smem, int *err,
                           cudaStream_t stream)
{
    using G = CGeo<NC, P>;
    auto kern = cluster_kernel<NC, P, MMA>;
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
    switch (nc) {
    case 25: return (long long)CGeo<25, 6>::SCR;
    case 29: return (long long)CGeo<29, 6>::SCR;
    default: return 0;
    }
}

// Cube sizes that take the cluster kernel (the 21^3 and 25^3 cubes run on the one-CTA slab kernel).
static bool cluster_cube(int nc) { return nc == 29; }

bool cluster_supported(const int nc[3], int fd_half)
{
    return nc[0] == nc[1] && nc[1] == nc[2] && cluster_cube(nc[0]) && fd_half == 6;
}

cudaError_t cluster_prepare(int nc, int amax, int fmax, int kb_fma, size_t *smem, int *max_clusters)
{
    switch (nc) {
    case 25: return kb_fma ? cluster_config<25, 6, false>(amax, fmax, smem, max_clusters)
                           : cluster_config<25, 6, true>(amax, fmax, smem, max_clusters);
    case 29: return kb_fma ? cluster_config<29, 6, false>(amax, fmax, smem, max_clusters)
                           : cluster_config<29, 6, true>(amax, fmax, smem, max_clusters);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cluster(const RecursionArgs<float> &args, int amax, int fmax, int nclusters, size_t smem, int *err,
                           cudaStream_t stream)
{
    switch (args.nc[0]) {
    case 25: return args.kb_fma ? cluster_launch<25, 6, false>(args, amax, fmax, nclusters, smem, err, stream)
                                : cluster_launch<25, 6, true>(args, amax, fmax, nclusters, smem, err, stream);
    case 29: return args.kb_fma ? cluster_launch<29, 6, false>(args, amax, fmax, nclusters, smem, err, stream)
                                : cluster_launch<29, 6, true>(args, amax, fmax, nclusters, smem, err, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sq
