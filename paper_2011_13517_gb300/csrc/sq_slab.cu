// FP32 per-column Chebyshev recursion for cubic truncation cubes of 21 or 25 points per axis with the
// 12th-order stencil: the "slab" kernel.
//
// Same mathematics as recursion_kernel (Eq. Chebyshev on the truncated scaled Hamiltonian, with the
// Kleinman-Bylander term and the force moments of Eq. NLforceSQ), mapped for the FP32 pipes:
//   - one CTA per column, NC warps: warp b owns the y-slab b of the cube; lane l holds the x position
//     a = l - 6 (lanes 0..5 and those past the cube hold zeros), and its z-pencil v(a, b, 0..NC-1)
//     stays in registers for the whole step;
//   - local part first: z neighbours from registers, x neighbours by warp shuffles (the zero lanes on
//     both sides make the cube boundary free of selects), y neighbours from the shared-memory copy of
//     v_k; the result goes to the accumulator pencil w and the registers of v_k are free again;
//   - KB term added into w two atoms per pass: for each atom whose support covers slab b, the y
//     factor folds into two per-lane scalars, and each 128-bit broadcast of a z-factor table feeds 4
//     FMAs; the z loops have no range branches: atoms whose support in the cube lies in the lower
//     or the upper half of the z range are paired among themselves and loop over that half only,
//     the others over the whole zero-padded table;
//   - projector contractions chi^T v: per-lane z sums (two atoms per pass, grouped by z half as
//     above; atoms with force moments in a pass of their own), a transposed butterfly reduction of
//     the x-weighted sums, per-slab slots in shared memory, then a fixed-order sum over slabs
//     (deterministic);
//   - two barriers per step: after the slab slots are written and after their sums are formed.  The
//     buffer written by step k is next read, and the buffer read by step k next written, behind the
//     two barriers of step k+1.
#include <cuda_runtime.h>

#include "sq_internal.h"
#include "sq_slab_common.cuh"

namespace sq {
namespace {

using namespace slabdev;

constexpr int kOff = 6;   // lane of x position 0

template <int NC>
struct Geo {
    static constexpr int NW = NC;                  // warps: one per y-slab
    static constexpr int NZ = (NC + 1) & ~1;       // z-table entries per atom (even: 128-bit pairs)
    static constexpr int HALF = ((NC - 1) / 2) & ~1;  // even split point of the z range
};

struct SlabSmem {
    float *va, *vb;
    float2 *tx, *ty;   // [amax][NC] (g, hp) window tables along x and y
    float4 *tz;        // [amax][NZ/2] (g[c], hp[c], g[c+1], hp[c+1]) along z
    float2 *fx, *fy;   // [fmax][NC] (g', hp') of force atoms along x and y
    float4 *fz;        // [fmax][NZ/2] (g', hp') pairs along z
    float *slot;       // [NC][amax][4]
    float *fslot;      // [NC][fmax][12]
    float *sd;         // [amax][4]
    SlabRec *rec;      // [amax]
    double *chiq;      // [fmax][4]
    int *ftl;          // [fmax] force slot -> active index
    unsigned *ymask;   // [NC][W]
    unsigned *fbits;   // [W] force atoms among the active ones
    unsigned *zlo;     // [W] atoms whose support in the cube lies in z <= NC/2 - 1/2 (lower half)
    unsigned *zhi;     // [W] atoms whose support in the cube lies in z >= NC/2 - 1/2 (upper half)
    float4 *zero;      // [NZ/2] zero z-table (partner of an unpaired atom)
    int *scan;         // [40]
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <int NC>
__host__ __device__ inline size_t slab_layout(unsigned char *base, int amax, int fmax, SlabSmem *s)
{
    const int W = (amax + 31) / 32;
    constexpr int NZ = Geo<NC>::NZ;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align16(off + bytes);
        return base ? base + o : nullptr;
    };
    const size_t nc3 = (size_t)NC * NC * NC;
    unsigned char *p;
    p = take(sizeof(float) * nc3);                      if (s) s->va = (float *)p;
    p = take(sizeof(float) * nc3);                      if (s) s->vb = (float *)p;
    p = take(sizeof(float2) * (size_t)amax * NC);       if (s) s->tx = (float2 *)p;
    p = take(sizeof(float2) * (size_t)amax * NC);       if (s) s->ty = (float2 *)p;
    p = take(sizeof(float2) * (size_t)amax * NZ);       if (s) s->tz = (float4 *)p;
    p = take(sizeof(float2) * (size_t)fmax * NC);       if (s) s->fx = (float2 *)p;
    p = take(sizeof(float2) * (size_t)fmax * NC);       if (s) s->fy = (float2 *)p;
    p = take(sizeof(float2) * (size_t)fmax * NZ);       if (s) s->fz = (float4 *)p;
    p = take(sizeof(float) * (size_t)NC * amax * 4);    if (s) s->slot = (float *)p;
    p = take(sizeof(float) * (size_t)NC * fmax * 12);   if (s) s->fslot = (float *)p;
    p = take(sizeof(float) * (size_t)amax * 4);         if (s) s->sd = (float *)p;
    p = take(sizeof(SlabRec) * (size_t)amax);           if (s) s->rec = (SlabRec *)p;
    p = take(sizeof(double) * (size_t)fmax * 4);        if (s) s->chiq = (double *)p;
    p = take(sizeof(int) * (size_t)fmax);               if (s) s->ftl = (int *)p;
    p = take(sizeof(unsigned) * (size_t)NC * W);        if (s) s->ymask = (unsigned *)p;
    p = take(sizeof(unsigned) * (size_t)W);             if (s) s->fbits = (unsigned *)p;
    p = take(sizeof(unsigned) * (size_t)W);             if (s) s->zlo = (unsigned *)p;
    p = take(sizeof(unsigned) * (size_t)W);             if (s) s->zhi = (unsigned *)p;
    p = take(sizeof(float4) * (size_t)(NZ / 2));        if (s) s->zero = (float4 *)p;
    p = take(sizeof(int) * 40);                         if (s) s->scan = (int *)p;
    return off;
}

// Per-column counts of active atoms (support meets the cube) and force atoms (support holds x_q).
__global__ void k_slab_counts(const RecursionArgs<float> args, int *counts)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < args.N_d;
         q += (long long)gridDim.x * blockDim.x) {
        const int qa[3] = {(int)(q % args.n[0]), (int)((q / args.n[0]) % args.n[1]),
                           (int)(q / ((long long)args.n[0] * args.n[1]))};
        int nact = 0, nfrc = 0;
        for (int J = 0; J < args.natom; J++) {
            bool on = true, frc = true;
            for (int ax = 0; ax < 3 && on; ax++) {
                const int st = args.sup_start[J * 3 + ax], len = args.sup_len[J * 3 + ax];
                short lo, hi;
                on = window_range(st, len, args.n[ax], args.nc[ax], smod(qa[ax] - args.m[ax], args.n[ax]), lo, hi);
                frc = frc && (len >= args.n[ax] || smod(qa[ax] - st, args.n[ax]) < len);
            }
            nact += on;
            nfrc += on && frc;
        }
        atomicMax(counts, nact);
        atomicMax(counts + 1, nfrc);
    }
}

// Projector contractions of two atoms per pass over z in [C0, C1) (C0 even; the tables are zero
// outside each atom's support, so a range that covers the support gives the full sums).
template <int NC, int C0, int C1>
__device__ __forceinline__ void dots_pairs(unsigned msk, int wd, const SlabSmem &S, const float (&vz)[NC], int b,
                                           int a, bool live, int lane, int amax)
{
    constexpr int NZ = Geo<NC>::NZ;
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
        // per atom: g_x G -> s, hp_x G -> p_x, g_x H -> p_z (y factor g), g_x G -> p_y (y factor hp)
        const float v8[8] = {x0.x * G0, x0.y * G0, x0.x * H0, x0.x * G0, x1.x * G1, x1.y * G1, x1.x * H1, x1.x * G1};
        const float red = reduce8(v8, lane);
        const int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if ((lane & 3) == 0 && (idx < 4 || two)) {
            const int t = idx < 4 ? t0 : t1;
            const int comp = idx & 3;
            const float2 yv = S.ty[t * NC + b];
            S.slot[((size_t)b * amax + t) * 4 + (comp == 2 ? 3 : comp == 3 ? 2 : comp)] = (comp == 3 ? yv.y : yv.x) * red;
        }
    }
}

// KB update of two atoms per pass over z in [C0, C1): w += kappa_l chi (chi^T v) from the dots.
template <int NC, int C0, int C1>
__device__ __forceinline__ void update_pairs(unsigned msk, int wd, const SlabSmem &S, float (&w)[NC], int b, int a,
                                             bool live, float kap0, float kap1)
{
    constexpr int NZ = Geo<NC>::NZ;
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
            const float2 yv = S.ty[t * NC + b];
            const float2 xv = live ? S.tx[t * NC + a] : make_float2(0.f, 0.f);
            // kappa_l chi (chi^T v) over s, p_x, p_y, p_z with the y factor folded in
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

// Per-thread geometry of the slab mapping.
template <int NC, int P>
struct SlabThread {
    int lane, b, a;        // lane, y-slab, x position
    bool live;             // x position inside the cube
    bool centre_xy;        // (a, b) is the column's own (x, y)
    unsigned yvalid;       // bit 2j-2: row b+j exists, bit 2j-1: row b-j exists
    __device__ SlabThread()
    {
        lane = threadIdx.x & 31;
        b = threadIdx.x >> 5;
        a = lane - kOff;
        live = a >= 0 && a < NC;
        centre_xy = live && a == (NC - 1) / 2 && b == (NC - 1) / 2;
        yvalid = 0u;
#pragma unroll
        for (int j = 1; j <= P; j++) {
            if (b + j < NC) yvalid |= 1u << (2 * j - 2);
            if (b - j >= 0) yvalid |= 1u << (2 * j - 1);
        }
    }
};

// Per-column set-up: the ordered list of atoms whose projector support meets the cube, their window
// tables, the force atoms (projectors nonzero at x_q, when args.want_force), and the slab coverage and
// z-half masks.  Returns the number of active atoms with *nfrc_out the force atoms, or -1 (after
// setting *err) when a capacity is exceeded; every thread of the CTA returns the same value.
template <int NC>
__device__ int slab_setup(const RecursionArgs<float> &args, const SlabSmem &S, long long q, int amax, int fmax,
                          int *err, int qa[3], int *nfrc_out)
{
    constexpr int NZ = Geo<NC>::NZ, NTH = NC * 32;
    constexpr int kHalf = Geo<NC>::HALF;
    const int W = (amax + 31) / 32;
    const int natom = args.natom;
    qa[0] = (int)(q % args.n[0]);
    qa[1] = (int)((q / args.n[0]) % args.n[1]);
    qa[2] = (int)(q / ((long long)args.n[0] * args.n[1]));
    int wstart[3];
#pragma unroll
    for (int ax = 0; ax < 3; ax++) wstart[ax] = smod(qa[ax] - args.m[ax], args.n[ax]);
    // ---- active atoms (ordered) ----
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
    if (nact > amax) {   // cannot happen with the pre-pass capacity; report and skip the column
        if (threadIdx.x == 0) atomicExch(err, 1);
        return -1;
    }
    __syncthreads();
    // ---- window tables ----
    for (int it = threadIdx.x; it < nact * NC; it += NTH) {
        const int o = it % NC, t = it / NC;
        const float *base = args.fac + (size_t)S.rec[t].J * args.fac_stride;
        const float *f0 = base + args.fac_off[0] + wstart[0] + o;
        const float *f1 = base + args.fac_off[1] + wstart[1] + o;
        S.tx[it] = make_float2(f0[0], f0[2 * args.n[0]]);
        S.ty[it] = make_float2(f1[0], f1[2 * args.n[1]]);
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
    // ---- force atoms: projectors nonzero at x_q ----
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
            if (threadIdx.x == 0) atomicExch(err, 2);
            return -1;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < nfrc * NC; it += NTH) {
            const int o = it % NC, fi = it / NC;
            const float *base = args.fac + (size_t)S.rec[S.ftl[fi]].J * args.fac_stride;
            const float *f0 = base + args.fac_off[0] + wstart[0] + o;
            const float *f1 = base + args.fac_off[1] + wstart[1] + o;
            S.fx[it] = make_float2(f0[4 * args.n[0]], f0[6 * args.n[0]]);
            S.fy[it] = make_float2(f1[4 * args.n[1]], f1[6 * args.n[1]]);
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
    // ---- slab coverage masks ----
    for (int it = threadIdx.x; it < NC * W; it += NTH) {
        const int wd = it % W, bb = it / W;
        unsigned msk = 0u;
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
    *nfrc_out = nfrc;
    return nact;
}

// Contraction phase of step k for the vector held in vz: projector dots chi^T v (when need_dots) and,
// with args.want_force, the force moments A_k of the force atoms, through the per-slab slots and
// their fixed-order sums into S.sd / A.  Holds the phase's first barrier, not the one after the sums.
template <int NC, int P>
__device__ __forceinline__ void slab_contract(const RecursionArgs<float> &args, const SlabSmem &S,
                                              const SlabThread<NC, P> &th, const float (&vz)[NC], int k,
                                              bool need_dots, int nact, int nfrc, int amax, int fmax)
{
    constexpr int NZ = Geo<NC>::NZ, NTH = NC * 32;
    constexpr int kHalf = Geo<NC>::HALF;
    const int W = (amax + 31) / 32;
    const int b = th.b, a = th.a, lane = th.lane;
    const bool live = th.live;
    if (need_dots || args.want_force) {
        for (int wd = 0; wd < W; wd++) {
            const unsigned all = S.ymask[b * W + wd];
            const unsigned fb = S.fbits[wd];
            // atoms without force moments, two per pass, grouped by the half of the z range their
            // support covers
            if (need_dots) {
                const unsigned nf = all & ~fb, zl = S.zlo[wd], zh = S.zhi[wd];
                dots_pairs<NC, 0, kHalf + 1>(nf & zl, wd, S, vz, b, a, live, lane, amax);
                dots_pairs<NC, kHalf, NC>(nf & zh, wd, S, vz, b, a, live, lane, amax);
                dots_pairs<NC, 0, NC>(nf & ~(zl | zh), wd, S, vz, b, a, live, lane, amax);
            }
            // atoms with force moments: projector and derivative contractions
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
                const float G = Ga + Gb, H = Ha + Hb, Gd = Gda + Gdb, Hd = Hda + Hdb;
                const float2 xv = live ? S.tx[t * NC + a] : make_float2(0.f, 0.f);
                const float2 yv = S.ty[t * NC + b];
                float *sl = S.slot + ((size_t)b * amax + t) * 4;
                const float2 xd = live ? S.fx[fidx * NC + a] : make_float2(0.f, 0.f);
                const float2 yd = S.fy[fidx * NC + b];
                const float v8[8] = {xv.x * G, xv.y * G, xv.x * H, xd.x * G, xv.x * Gd, xd.y * G, xv.y * Gd, xd.x * H};
                const float red = reduce8(v8, lane);
                const float v9 = wsum(xv.x * Hd);
                const int idx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                float *fs = S.fslot + ((size_t)b * fmax + fidx) * 12;
                if ((lane & 3) == 0) {
                    switch (idx) {
                    case 0: sl[0] = yv.x * red; sl[2] = yv.y * red;      // gx G: s, p_y
                            fs[1] = yd.x * red; fs[7] = yd.y * red; break; //  s d/dy, py d/dy
                    case 1: sl[1] = yv.x * red; fs[4] = yd.x * red; break; // hx G: p_x; px d/dy
                    case 2: sl[3] = yv.x * red; fs[10] = yd.x * red; break; // gx H: p_z; pz d/dy
                    case 3: fs[0] = yv.x * red; fs[6] = yv.y * red; break;  // g'x G: s, py d/dx
                    case 4: fs[2] = yv.x * red; fs[8] = yv.y * red; break;  // gx Gd: s, py d/dz
                    case 5: fs[3] = yv.x * red; break;                      // h'x G: px d/dx
                    case 6: fs[5] = yv.x * red; break;                      // hx Gd: px d/dz
                    default: fs[9] = yv.x * red; break;                     // g'x H: pz d/dx
                    }
                }
                if (lane == 0) fs[11] = yv.x * v9;                          // gx Hd: pz d/dz
            }
        }
    }
    __syncthreads();
    // fixed-order sum of the slab slots: dots of v_k, and force moments A_k
    if (need_dots) {
        for (int it = threadIdx.x; it < nact * 4; it += NTH) {
            const int t = it >> 2, comp = it & 3;
            float s = 0.f;
            for (int bb = 0; bb < NC; bb++)
                if ((S.ymask[bb * W + (t >> 5)] >> (t & 31)) & 1u) s += S.slot[((size_t)bb * amax + t) * 4 + comp];
            S.sd[it] = s;
        }
    }
    if (args.want_force) {
        const int nproj = args.nproj, natom = args.natom;
        const int nf = nproj > 1 ? 12 : 3;
        for (int it = threadIdx.x; it < nfrc * nf; it += NTH) {
            const int fi = it / nf, i = it % nf;
            const int t = S.ftl[fi];
            double s = 0.0;
            for (int bb = 0; bb < NC; bb++)
                if ((S.ymask[bb * W + (t >> 5)] >> (t & 31)) & 1u) s += (double)S.fslot[((size_t)bb * fmax + fi) * 12 + i];
            const int lm = i / 3, d = i % 3;
            atomicAdd(args.A + ((((size_t)k * natom + S.rec[t].J) * nproj + lm) * 3 + d),
                      S.chiq[4 * fi + lm] * args.Nnorm * s);
        }
    }
}

// Apply phase: w = ca Hhat v - cb v_prev for the vector v held in vz (registers) and vcur (shared
// copy), with v_prev in vprev, which receives the result (w keeps it too).  The local part comes
// first (v's registers die there), then the KB term from the dots in S.sd.  With INJ the thread that
// owns x_q adds `inj` to the result there (the source term of the reverse recursion).
template <int NC, int P, bool INJ>
__device__ __forceinline__ void slab_apply(const RecursionArgs<float> &args, const SlabSmem &S,
                                           const SlabThread<NC, P> &th, const float (&vz)[NC], float (&w)[NC],
                                           const float *vcur, float *vprev, const float *drow, size_t plane_p,
                                           float ca, float cb, float inj, int amax)
{
    constexpr int kHalf = Geo<NC>::HALF;
    const int W = (amax + 31) / 32;
    const int b = th.b, a = th.a, lane = th.lane;
    const bool live = th.live;
    const float kap0 = args.kappa[0], kap1 = args.kappa[1];
    // ---- local part: stencil + diagonal of Hhat v into w ----
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
        for (int j = 1; j <= P; j++) {
            const float xp = __shfl_sync(0xffffffffu, x, min(lane + j, 31));
            const float xm = __shfl_sync(0xffffffffu, x, lane - j);
            t += args.w[0][j - 1] * (xp + xm);
        }
        if (live) {
            const float *row = vcur + (size_t)(c * NC + b) * NC + a;
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
    // ---- KB term of Hhat v, from the dots ----
    for (int wd = 0; wd < W; wd++) {
        const unsigned all = S.ymask[b * W + wd], zl = S.zlo[wd], zh = S.zhi[wd];
        update_pairs<NC, 0, kHalf + 1>(all & zl, wd, S, w, b, a, live, kap0, kap1);
        update_pairs<NC, kHalf, NC>(all & zh, wd, S, w, b, a, live, kap0, kap1);
        update_pairs<NC, 0, NC>(all & ~(zl | zh), wd, S, w, b, a, live, kap0, kap1);
    }
    // ---- w = ca Hhat v - cb v_prev ----
#pragma unroll
    for (int c = 0; c < NC; c++) {
        if (live) {
            float *pv = vprev + (size_t)(c * NC + b) * NC + a;
            float nv = ca * w[c] - cb * (*pv);
            if (INJ && c == (NC - 1) / 2 && th.centre_xy) nv += inj;
            *pv = nv;
            w[c] = nv;
        } else {
            w[c] = 0.f;
        }
    }
}

template <int NC, int P>
__global__ void __launch_bounds__(NC * 32, 1) slab_kernel(const RecursionArgs<float> args, int amax, int fmax,
                                                          int *err)
{
    constexpr int NZ = Geo<NC>::NZ, NTH = NC * 32;
    static_assert(kOff >= P && kOff + NC <= 31, "lane layout: zero lanes below x = 0 and at lane 31");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SlabSmem S;
    slab_layout<NC>(smem_raw, amax, fmax, &S);
    const SlabThread<NC, P> th;
    const int m = (NC - 1) / 2;
    const long long N_d = args.N_d;
    const size_t plane_p = (size_t)args.pn[0] * args.pn[1];

    for (int i = threadIdx.x; i < NZ / 2; i += NTH) S.zero[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    for (long long q = args.q0 + blockIdx.x; q < args.q1; q += gridDim.x) {
        int qa[3], nfrc = 0;
        const int nact = slab_setup<NC>(args, S, q, amax, fmax, err, qa, &nfrc);
        if (nact < 0) continue;
        // ---- v_0 = e_q, v_{-1} = 0 ----
        float vz[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) {
            vz[c] = (th.centre_xy && c == m) ? 1.0f : 0.0f;
            if (th.live) {
                S.va[(c * NC + th.b) * NC + th.a] = vz[c];
                S.vb[(c * NC + th.b) * NC + th.a] = 0.0f;
            }
        }
        if (threadIdx.x == 0) args.mu[q] = 1.0f;
        __syncthreads();
        float *vcur = S.va, *vprev = S.vb;
        const float *drow = args.dpad + (size_t)qa[2] * plane_p + (size_t)(qa[1] + th.b) * args.pn[0] + qa[0] +
                            (th.live ? th.a : 0);

        for (int k = 0; k <= args.K; k++) {
            slab_contract<NC, P>(args, S, th, vz, k, k < args.K, nact, nfrc, amax, fmax);
            if (k == args.K) break;
            __syncthreads();
            float w[NC];
            slab_apply<NC, P, false>(args, S, th, vz, w, vcur, vprev, drow, plane_p, k == 0 ? 1.f : 2.f,
                                     k == 0 ? 0.f : 1.f, 0.f, amax);
            if (th.centre_xy) args.mu[(size_t)(k + 1) * N_d + q] = w[m];
            // no barrier here: the next reads of the buffer just written, and the next writes of the
            // buffer just read, sit behind the two barriers of the next step's contraction phase
            float *sw = vprev;
            vprev = vcur;
            vcur = sw;
#pragma unroll
            for (int c = 0; c < NC; c++) vz[c] = w[c];
        }
        __syncthreads();
    }
}

// Per-thread pencils of one cube vector in global scratch: element (c, warp, lane) at
// (c NC + warp) 32 + lane, so a warp's 32 lanes touch 128 consecutive bytes per z index.
template <int NC>
__device__ __forceinline__ void pencil_store(float *dst, const float (&v)[NC])
{
#pragma unroll
    for (int c = 0; c < NC; c++) dst[(size_t)c * NC * 32 + threadIdx.x] = v[c];
}

template <int NC>
__device__ __forceinline__ void pencil_load(const float *src, float (&v)[NC])
{
#pragma unroll
    for (int c = 0; c < NC; c++) v[c] = src[(size_t)c * NC * 32 + threadIdx.x];
}

// Shared-memory copy of a pencil (live lanes only) in the cube layout the stencil reads.
template <int NC, int P>
__device__ __forceinline__ void pencil_to_smem(float *dst, const float (&v)[NC], const SlabThread<NC, P> &th)
{
    if (th.live) {
#pragma unroll
        for (int c = 0; c < NC; c++) dst[(c * NC + th.b) * NC + th.a] = v[c];
    }
}

template <int NC, int P>
__device__ __forceinline__ void pencil_from_smem(const float *src, float (&v)[NC], const SlabThread<NC, P> &th)
{
#pragma unroll
    for (int c = 0; c < NC; c++) v[c] = th.live ? src[(c * NC + th.b) * NC + th.a] : 0.f;
}

// Reverse-mode pass (vector-Jacobian product of rho and U wrt V_eff) with the slab mapping; the
// same checkpoint scheme as the generic adjoint kernel.  Per column:
//   forward  v_0 = e_q ... v_K, storing (v_j, v_{j+1}) at j = 0, kc, 2kc, ...;
//   reverse  a_{K+1} = 0, a_K = mubar_K e_q, a_k = 2 Hhat a_{k+1} - a_{k+2} + mubar_k e_q, with
//            Dbar += w_k a_{k+1} .* v_k (w_0 = 1, else 2) for k = K-1 .. 0, the forward vectors of
//            each kc-segment recomputed from its checkpoint pair;
//   scatter  Vbar(x) += Dbar(x) / tau (FP64 atomics).
// Per-CTA scratch (floats, vectors of NC*NC*32): [2 nsegs] checkpoints, [kc + 1] segment vectors,
// saved a_{k+1} and a_{k+2}, and Dbar.
template <int NC, int P>
__global__ void __launch_bounds__(NC * 32, 1) slab_adjoint_kernel(const RecursionArgs<float> args, int amax,
                                                                  int *err, long long scratch_stride)
{
    constexpr int NZ = Geo<NC>::NZ, NTH = NC * 32;
    constexpr size_t VEC = (size_t)NC * NC * 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SlabSmem S;
    slab_layout<NC>(smem_raw, amax, 1, &S);
    const SlabThread<NC, P> th;
    const int m = (NC - 1) / 2;
    const int K = args.K, kc = args.adj_kc;
    const int nsegs = (K + kc - 1) / kc;
    const long long N_d = args.N_d;
    const size_t plane_p = (size_t)args.pn[0] * args.pn[1];
    float *ck = args.scratch + (size_t)blockIdx.x * scratch_stride;   // [2 nsegs]
    float *seg = ck + 2 * (size_t)nsegs * VEC;                        // [kc + 1]
    float *Xs = seg + (size_t)(kc + 1) * VEC;                         // saved a_{k+1}
    float *Zs = Xs + VEC;                                             // saved a_{k+2}
    float *Db = Zs + VEC;                                             // diagonal cotangent

    for (int i = threadIdx.x; i < NZ / 2; i += NTH) S.zero[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    for (long long q = args.q0 + blockIdx.x; q < args.q1; q += gridDim.x) {
        int qa[3], nfrc = 0;
        const int nact = slab_setup<NC>(args, S, q, amax, 1, err, qa, &nfrc);
        if (nact < 0) continue;
        const double rb = args.adj_rho_bar[q];
        const float *drow = args.dpad + (size_t)qa[2] * plane_p + (size_t)(qa[1] + th.b) * args.pn[0] + qa[0] +
                            (th.live ? th.a : 0);
        float vz[NC], w[NC];
        float *vcur = S.va, *vprev = S.vb;
        // ---- forward pass with checkpoints ----
#pragma unroll
        for (int c = 0; c < NC; c++) {
            vz[c] = (th.centre_xy && c == m) ? 1.0f : 0.0f;
            w[c] = 0.f;
        }
        pencil_to_smem(vcur, vz, th);
        pencil_to_smem(vprev, w, th);
        __syncthreads();
        for (int k = 0; k < K; k++) {
            if (k % kc == 0) pencil_store(ck + (size_t)(2 * (k / kc)) * VEC, vz);
            slab_contract<NC, P>(args, S, th, vz, k, true, nact, 0, amax, 1);
            __syncthreads();
            slab_apply<NC, P, false>(args, S, th, vz, w, vcur, vprev, drow, plane_p, k == 0 ? 1.f : 2.f,
                                     k == 0 ? 0.f : 1.f, 0.f, amax);
            float *sw = vprev;
            vprev = vcur;
            vcur = sw;
#pragma unroll
            for (int c = 0; c < NC; c++) vz[c] = w[c];
            if (k % kc == 0) pencil_store(ck + (size_t)(2 * (k / kc) + 1) * VEC, vz);
        }
        // ---- reverse pass: a_K = mubar_K e_q (registers + shared copy), a_{K+1} = 0, Dbar = 0 ----
#pragma unroll
        for (int c = 0; c < NC; c++) {
            vz[c] = (th.centre_xy && c == m) ? (float)(args.adj_alpha[K] * rb + args.adj_beta[K]) : 0.f;
            w[c] = 0.f;
        }
        pencil_store(Db, w);
        __syncthreads();   // every warp is past its last shared-memory access of the forward pass
        pencil_to_smem(vcur, vz, th);
        pencil_to_smem(vprev, w, th);
        for (int s = nsegs - 1; s >= 0; s--) {
            const int j = s * kc;
            const int jend = min(j + kc - 1, K - 1);
            if (jend > j + 1) {
                // save a_{k+1} (registers) and a_{k+2} (shared), then recompute v_{j+2} .. v_jend
                pencil_store(Xs, vz);
                __syncthreads();
                pencil_from_smem(vprev, w, th);
                pencil_store(Zs, w);
                pencil_load(ck + (size_t)(2 * s) * VEC, w);             // v_j
                pencil_load(ck + (size_t)(2 * s + 1) * VEC, vz);        // v_{j+1}
                __syncthreads();
                pencil_to_smem(vprev, w, th);
                pencil_to_smem(vcur, vz, th);
                __syncthreads();
                for (int i = 1; j + i < jend; i++) {
                    slab_contract<NC, P>(args, S, th, vz, 0, true, nact, 0, amax, 1);
                    __syncthreads();
                    slab_apply<NC, P, false>(args, S, th, vz, w, vcur, vprev, drow, plane_p, 2.f, 1.f, 0.f, amax);
                    float *sw = vprev;
                    vprev = vcur;
                    vcur = sw;
#pragma unroll
                    for (int c = 0; c < NC; c++) vz[c] = w[c];
                    pencil_store(seg + (size_t)(i + 1) * VEC, vz);      // v_{j+i+1}
                }
                // restore a_{k+1}, a_{k+2}
                __syncthreads();
                pencil_load(Xs, vz);
                pencil_load(Zs, w);
                pencil_to_smem(vcur, vz, th);
                pencil_to_smem(vprev, w, th);
            }
            __syncthreads();
            for (int k = jend; k >= j; k--) {
                // Dbar += w_k a_{k+1} .* v_k
                const float *vk = k == j ? ck + (size_t)(2 * s) * VEC
                                         : (k == j + 1 ? ck + (size_t)(2 * s + 1) * VEC : seg + (size_t)(k - j) * VEC);
                const float wk = k >= 1 ? 2.f : 1.f;
#pragma unroll
                for (int c = 0; c < NC; c++) {
                    const size_t o = (size_t)c * NC * 32 + threadIdx.x;
                    Db[o] += wk * vz[c] * vk[o];
                }
                if (k >= 1) {
                    slab_contract<NC, P>(args, S, th, vz, 0, true, nact, 0, amax, 1);
                    __syncthreads();
                    slab_apply<NC, P, true>(args, S, th, vz, w, vcur, vprev, drow, plane_p, 2.f, 1.f,
                                            (float)(args.adj_alpha[k] * rb + args.adj_beta[k]), amax);
                    float *sw = vprev;
                    vprev = vcur;
                    vcur = sw;
#pragma unroll
                    for (int c = 0; c < NC; c++) vz[c] = w[c];
                }
            }
        }
        // ---- scatter Dbar / tau onto the grid ----
        if (th.live) {
            const int g0 = smod(qa[0] - args.m[0] + th.a, args.n[0]);
            const int g1 = smod(qa[1] - args.m[1] + th.b, args.n[1]);
#pragma unroll
            for (int c = 0; c < NC; c++) {
                const double v = (double)Db[(size_t)c * NC * 32 + threadIdx.x] * args.adj_inv_tau;
                const int g2 = smod(qa[2] - args.m[2] + c, args.n[2]);
                if (v != 0.0) atomicAdd(args.adj_vbar + (g0 + (long long)args.n[0] * (g1 + (long long)args.n[1] * g2)), v);
            }
        }
        __syncthreads();
    }
}

template <int NC, int P>
cudaError_t launch_nc(const RecursionArgs<float> &args, int amax, int fmax, int grid, size_t smem, int *err,
                      cudaStream_t stream)
{
    auto kern = slab_kernel<NC, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, Geo<NC>::NW * 32, smem, stream>>>(args, amax, fmax, err);
    return cudaGetLastError();
}

template <int NC, int P>
cudaError_t launch_adjoint_nc(const RecursionArgs<float> &args, int amax, int grid, size_t smem, int *err,
                              long long scratch_stride, cudaStream_t stream)
{
    auto kern = slab_adjoint_kernel<NC, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, Geo<NC>::NW * 32, smem, stream>>>(args, amax, err, scratch_stride);
    return cudaGetLastError();
}

}  // namespace

bool slab_supported(const int nc[3], int fd_half)
{
    return nc[0] == nc[1] && nc[1] == nc[2] && (nc[0] == 21 || nc[0] == 25) && fd_half == 6;
}

size_t slab_smem_bytes(int nc, int amax, int fmax)
{
    switch (nc) {
    case 21: return slab_layout<21>(nullptr, amax, fmax, nullptr);
    case 25: return slab_layout<25>(nullptr, amax, fmax, nullptr);
    default: return ~size_t(0);
    }
}

cudaError_t slab_counts(const RecursionArgs<float> &args, int *d_counts, int num_sms, cudaStream_t stream)
{
    k_slab_counts<<<num_sms * 4, 128, 0, stream>>>(args, d_counts);
    return cudaGetLastError();
}

cudaError_t launch_slab(const RecursionArgs<float> &args, int amax, int fmax, int grid, size_t smem, int *err,
                        cudaStream_t stream)
{
    switch (args.nc[0]) {
    case 21: return launch_nc<21, 6>(args, amax, fmax, grid, smem, err, stream);
    case 25: return launch_nc<25, 6>(args, amax, fmax, grid, smem, err, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_slab_adjoint(const RecursionArgs<float> &args, int amax, int grid, size_t smem, int *err,
                                long long scratch_stride, cudaStream_t stream)
{
    switch (args.nc[0]) {
    case 21: return launch_adjoint_nc<21, 6>(args, amax, grid, smem, err, scratch_stride, stream);
    case 25: return launch_adjoint_nc<25, 6>(args, amax, grid, smem, err, scratch_stride, stream);
    default: return cudaErrorInvalidValue;
    }
}

long long slab_vector_floats(int nc) { return (long long)nc * nc * 32; }

}  // namespace sq
