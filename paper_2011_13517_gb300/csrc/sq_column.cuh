// The per-column machinery of the generic recursion kernels (internal to libsq): column set-up, the
// projector-contraction and operator-application phases, and the loops that run them for the
// Chebyshev recursion (Eq. Chebyshev), the reverse-mode pass and the Lanczos iteration (Eq. Lanczos).
// Included by the translation units that instantiate those kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sq_internal.h"

namespace sq {
namespace {

constexpr int kSeg = 8;   // x-segment length of phase 2

struct AtomRec {
    int J;          // atom index
    int fidx;       // index into the force table, or -1
    short lo[3];    // bounding local range [lo, hi] of the support inside the cube, per axis
    short hi[3];
    int base[3];    // fac offset of factor 0 of this atom's window start, per axis
};

__device__ __forceinline__ int pmod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide ordered compaction of a flag: returns this thread's output slot (or -1) and the
// total count through *total.  `scan` holds >= 33 ints of shared memory.
__device__ int block_compact(bool flag, int *scan, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    unsigned bal = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) scan[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < nwarp; w++) {
            int c = scan[w];
            scan[w] = acc;
            acc += c;
        }
        scan[32] = acc;
    }
    __syncthreads();
    int slot = flag ? scan[warp] + __popc(bal & ((1u << lane) - 1u)) : -1;
    *total = scan[32];
    __syncthreads();
    return slot;
}


// Reverse-mode derivative of the moments of one column with respect to the diagonal of Hhat_q
// (i.e. V_eff / tau on the cube), for the cotangent mubar_k = alpha_k rhobar_q + beta_k:
//   a_K = mubar_K e_q,  a_k = 2 Hhat a_{k+1} - a_{k+2} + mubar_k e_q   (reverse Clenshaw),
//   Dbar = sum_{k>=1} 2 a_{k+1} (.) v_k + a_1 (.) v_0,   Vbar(x) += Dbar(x) / tau.
// The forward vectors are kept as checkpoint pairs (v_j, v_{j+1}) every kc steps and recomputed
// segment by segment during the backward sweep.  vA/vB hold v_0 = e_q and v_{-1} = 0 on entry;
// work points to the CTA's remaining scratch: [2 nseg + kc + 1 + 3] vectors.
template <typename T, typename Dots, typename Update>
__device__ __forceinline__ void adjoint_column(const RecursionArgs<T> &args, long long q, int centre, Dots &dots,
                                               Update &update, T *vA, T *vB, T *work)
{
    const int nc3 = args.nc3, K = args.K, kc = args.adj_kc;
    const int nsegs = (K + kc - 1) / kc;
    T *ck = work;                                   // [2 nsegs][nc3]
    T *seg = ck + (size_t)2 * nsegs * nc3;          // [kc + 1][nc3]
    T *X = seg + (size_t)(kc + 1) * nc3;            // a_{k+1}
    T *Z = X + nc3;                                 // a_{k+2}
    T *Db = Z + nc3;                                // diagonal cotangent
    const double rb = args.adj_rho_bar[q];
    auto mubar = [&](int k) { return (T)(args.adj_alpha[k] * rb + args.adj_beta[k]); };
    auto copy = [&](const T *src, T *dst) {
        for (int i = threadIdx.x; i < nc3; i += blockDim.x) dst[i] = src[i];
    };
    // forward pass, storing (v_j, v_{j+1}) at j = 0, kc, 2kc, ...
    T *vc = vA, *vp = vB;
    for (int k = 0; k < K; k++) {
        if (k % kc == 0) copy(vc, ck + (size_t)(2 * (k / kc)) * nc3);
        dots(vc, k, true);
        __syncthreads();
        update(vc, vp, vp, k == 0 ? T(1) : T(2), k == 0 ? T(0) : T(1));
        __syncthreads();
        T *sw = vp;
        vp = vc;
        vc = sw;
        if (k % kc == 0) copy(vc, ck + (size_t)(2 * (k / kc) + 1) * nc3);
    }
    // seeds: a_{K+1} = 0, a_K = mubar_K e_q
    for (int i = threadIdx.x; i < nc3; i += blockDim.x) {
        X[i] = (i == centre) ? mubar(K) : T(0);
        Z[i] = T(0);
        Db[i] = T(0);
    }
    __syncthreads();
    for (int s = nsegs - 1; s >= 0; s--) {
        const int j = s * kc;
        const int jend = min(j + kc - 1, K - 1);
        copy(ck + (size_t)(2 * s) * nc3, seg);
        if (jend > j) copy(ck + (size_t)(2 * s + 1) * nc3, seg + nc3);
        __syncthreads();
        for (int i = 1; j + i < jend; i++) {       // seg[i+1] = v_{j+i+1}
            dots(seg + (size_t)i * nc3, 0, true);
            __syncthreads();
            update(seg + (size_t)i * nc3, seg + (size_t)(i - 1) * nc3, seg + (size_t)(i + 1) * nc3, T(2), T(1));
            __syncthreads();
        }
        for (int k = jend; k >= j; k--) {
            const T wk = k >= 1 ? T(2) : T(1);
            const T *vk = seg + (size_t)(k - j) * nc3;
            for (int i = threadIdx.x; i < nc3; i += blockDim.x) Db[i] += wk * X[i] * vk[i];
            if (k >= 1) {
                dots(X, 0, true);
                __syncthreads();
                update(X, Z, Z, T(2), T(1));
                __syncthreads();
                if (threadIdx.x == 0) Z[centre] += mubar(k);
                __syncthreads();
                T *sw = X;
                X = Z;
                Z = sw;
            }
            __syncthreads();
        }
    }
    // scatter Dbar / tau onto the global grid
    const int q1 = (int)(q % args.n[0]);
    const int q2 = (int)((q / args.n[0]) % args.n[1]);
    const int q3 = (int)(q / ((long long)args.n[0] * args.n[1]));
    for (int i = threadIdx.x; i < nc3; i += blockDim.x) {
        const int a = i % args.nc[0], b = (i / args.nc[0]) % args.nc[1], c = i / (args.nc[0] * args.nc[1]);
        const int g0 = pmod(q1 - args.m[0] + a, args.n[0]);
        const int g1 = pmod(q2 - args.m[1] + b, args.n[1]);
        const int g2 = pmod(q3 - args.m[2] + c, args.n[2]);
        const double v = (double)Db[i] * args.adj_inv_tau;
        if (v != 0.0) atomicAdd(args.adj_vbar + (g0 + (long long)args.n[0] * (g1 + (long long)args.n[1] * g2)), v);
    }
    __syncthreads();
}

// Sums of two doubles per thread over the CTA, the same values in every thread (fixed order: warp
// shuffles, then the warps' partials in index order).  `red` holds 32 double2 of shared memory.
__device__ __forceinline__ double2 block_sum2(double2 v, double2 *red)
{
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        t.x += red[w].x;
        t.y += red[w].y;
    }
    __syncthreads();
    return t;
}

// Columns q_begin, q_begin + q_step, ... < q_end of one cell (or, with args.cols, the listed columns
// at those list positions), processed by the calling CTA.  smem_raw is the CTA's dynamic shared
// memory; scratch its two cube vectors when !VSMEM.
template <typename T, int P, int BLOCK, bool VSMEM, bool ADJ = false, bool LANCZOS = false>
__device__ __forceinline__ void column_range(const RecursionArgs<T> &args, long long q_begin, long long q_end,
                                             long long q_step, unsigned char *smem_raw, T *scratch)
{
    const int natom = args.natom;
    const int ncx = args.nc[0], ncy = args.nc[1], ncz = args.nc[2];
    const int nc3 = args.nc3;
    const int nsx = (ncx + kSeg - 1) / kSeg;
    const int maskw = (natom + 31) / 32;     // mask words per row/plane/segment
    // shared memory carve-up (sizes mirrored by recursion_smem_bytes)
    AtomRec *act = reinterpret_cast<AtomRec *>(smem_raw);
    T *sdot = reinterpret_cast<T *>(act + natom);                       // [natom][4]
    double *chiq = reinterpret_cast<double *>(sdot + 4 * natom + 1);   // [natom][4]
    chiq = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(chiq) + 15) & ~uintptr_t(15));
    int *scan = reinterpret_cast<int *>(chiq + 4 * natom);             // [40]
    // bit t of ymask[b] / zmask[c] / xmask[segment] is set when active atom t's support box covers
    // y-row b / z-plane c / part of x-segment
    unsigned *ymask = reinterpret_cast<unsigned *>(scan + 40);
    unsigned *zmask = ymask + ncy * maskw;
    unsigned *xmask = zmask + ncz * maskw;
    T *vec = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(xmask + nsx * maskw) + 15) & ~uintptr_t(15));

    T *va, *vb;
    if constexpr (VSMEM) {
        va = vec;
        vb = vec + nc3;
    } else {
        va = scratch;
        vb = va + nc3;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int nproj = args.nproj;
    const int centre = args.m[0] + ncx * (args.m[1] + ncy * args.m[2]);
    const long long N_d = args.N_d;
    const int nseg = nsx * ncy * ncz;
    const size_t plane_p = (size_t)args.pn[0] * args.pn[1];

    for (long long qi = q_begin; qi < q_end; qi += q_step) {
        const long long q = args.cols ? args.cols[qi] : qi;
        const int q1 = (int)(q % args.n[0]);
        const int q2 = (int)((q / args.n[0]) % args.n[1]);
        const int q3 = (int)(q / ((long long)args.n[0] * args.n[1]));
        const int qa[3] = {q1, q2, q3};
        int wstart[3];
#pragma unroll
        for (int a = 0; a < 3; a++) wstart[a] = pmod(qa[a] - args.m[a], args.n[a]);

        // ---- column set-up: atoms whose projector support meets the cube (ordered) ----------
        int nact = 0;
        for (int base = 0; base < natom; base += BLOCK) {
            const int J = base + threadIdx.x;
            bool on = J < natom;
            short lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
            if (on) {
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const int na = args.n[a], nca = args.nc[a];
                    const int st = args.sup_start[J * 3 + a], len = args.sup_len[J * 3 + a];
                    if (len >= na) {
                        lo[a] = 0;
                        hi[a] = (short)(nca - 1);
                        continue;
                    }
                    const bool first_in = pmod(wstart[a] - st, na) < len;     // cube start inside support
                    const int d = pmod(st - wstart[a], na);                   // support start offset
                    const bool starts_in = d < nca;
                    if (!first_in && !starts_in) {
                        on = false;
                        break;
                    }
                    const bool last_in = pmod(wstart[a] + nca - 1 - st, na) < len;
                    lo[a] = (short)(first_in ? 0 : d);
                    if (last_in || (first_in && starts_in && d > 0)) {
                        hi[a] = (short)(nca - 1);
                    } else {
                        hi[a] = (short)pmod(st + len - 1 - wstart[a], na);
                    }
                }
            }
            int total;
            const int slot = block_compact(on, scan, &total);
            if (slot >= 0) {
                AtomRec r;
                r.J = J;
                r.fidx = -1;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    r.lo[a] = lo[a];
                    r.hi[a] = hi[a];
                    r.base[a] = J * args.fac_stride + args.fac_off[a] + wstart[a];
                }
                act[nact + slot] = r;
            }
            nact += total;
        }
        __syncthreads();
        // coverage masks of the active atoms
        {
            const int wcol = (nact + 31) / 32;
            const int nitems = (ncy + ncz + nsx) * maskw;
            for (int it = threadIdx.x; it < nitems; it += BLOCK) {
                const int w = it % maskw;
                const int idx = it / maskw;
                unsigned m = 0u;
                if (w < wcol) {
                    const int tend = min(nact, 32 * w + 32);
                    for (int t = 32 * w; t < tend; t++) {
                        const AtomRec &r = act[t];
                        bool cov;
                        if (idx < ncy) cov = idx >= r.lo[1] && idx <= r.hi[1];
                        else if (idx < ncy + ncz) cov = (idx - ncy) >= r.lo[2] && (idx - ncy) <= r.hi[2];
                        else {
                            const int a0 = (idx - ncy - ncz) * kSeg;
                            cov = r.lo[0] <= a0 + kSeg - 1 && r.hi[0] >= a0;
                        }
                        if (cov) m |= 1u << (t - 32 * w);
                    }
                }
                ymask[it] = m;   // ymask, zmask and xmask are contiguous
            }
        }
        // force atoms: projectors nonzero at x_q; chi_Jlm(x_q) in FP64
        if (args.want_force) {
            for (int t = threadIdx.x; t < nact; t += BLOCK) {
                AtomRec &r = act[t];
                const double *f = args.fac64 + (size_t)r.J * args.fac64_stride;
                const double gx = f[args.fac64_off[0] + 0 * args.n[0] + q1];
                const double gy = f[args.fac64_off[1] + 0 * args.n[1] + q2];
                const double gz = f[args.fac64_off[2] + 0 * args.n[2] + q3];
                if (gx != 0.0 && gy != 0.0 && gz != 0.0) {
                    r.fidx = t;
                    const double hx = f[args.fac64_off[0] + 1 * args.n[0] + q1];
                    const double hy = f[args.fac64_off[1] + 1 * args.n[1] + q2];
                    const double hz = f[args.fac64_off[2] + 1 * args.n[2] + q3];
                    chiq[4 * t + 0] = args.Nnorm * gx * gy * gz;
                    chiq[4 * t + 1] = args.Nnorm * hx * gy * gz;
                    chiq[4 * t + 2] = args.Nnorm * gx * hy * gz;
                    chiq[4 * t + 3] = args.Nnorm * gx * gy * hz;
                }
            }
        }
        // v_0 = e_q, v_{-1} = 0
        for (int i = threadIdx.x; i < nc3; i += BLOCK) {
            va[i] = (i == centre) ? T(1) : T(0);
            vb[i] = T(0);
        }
        if (!LANCZOS && threadIdx.x == 0) args.mu[q] = T(1);   // the Lanczos mode writes only args.ab
        __syncthreads();

        T *vcur = va, *vprev = vb;
        const size_t dbase = (size_t)q3 * plane_p + (size_t)q2 * args.pn[0] + q1;
        const int two_nx = 2 * args.n[0], two_ny = 2 * args.n[1], two_nz = 2 * args.n[2];

        const bool wforce = ADJ ? false : (bool)args.want_force;
        // phase 1: projector contractions chi^T X (and, at step k, force moments of X)
        auto dots = [&](const T *X, int k, bool need_dots) {
            if (need_dots || wforce) {
                for (int t = warp; t < nact; t += nwarp) {
                    const AtomRec r = act[t];
                    const bool frc = wforce && r.fidx >= 0;
                    if (!need_dots && !frc) continue;
                    const T *fx = args.fac + r.base[0];
                    const T *fy = args.fac + r.base[1];
                    const T *fz = args.fac + r.base[2];
                    const int nry = r.hi[1] - r.lo[1] + 1;
                    const int nrows = nry * (r.hi[2] - r.lo[2] + 1);
                    T s0 = 0, spx = 0, spy = 0, spz = 0;
                    T f[12];
#pragma unroll
                    for (int i = 0; i < 12; i++) f[i] = 0;
                    for (int row = lane; row < nrows; row += 32) {
                        const int b = r.lo[1] + row % nry;
                        const int c = r.lo[2] + row / nry;
                        const T *vr = X + (c * ncy + b) * ncx;
                        T Gs = 0, Hs = 0, Gd = 0, Hd = 0;
                        for (int a = r.lo[0]; a <= r.hi[0]; a++) {
                            const T val = vr[a];
                            Gs += fx[a] * val;
                            if (nproj > 1) Hs += fx[two_nx + a] * val;
                            if (frc) {
                                Gd += fx[2 * two_nx + a] * val;
                                if (nproj > 1) Hd += fx[3 * two_nx + a] * val;
                            }
                        }
                        const T gy = fy[b], gz = fz[c];
                        const T gyz = gy * gz;
                        s0 += Gs * gyz;
                        T hy = 0, hz = 0;
                        if (nproj > 1) {
                            hy = fy[two_ny + b];
                            hz = fz[two_nz + c];
                            spx += Hs * gyz;
                            spy += Gs * hy * gz;
                            spz += Gs * gy * hz;
                        }
                        if (frc) {
                            const T gdy = fy[2 * two_ny + b], gdz = fz[2 * two_nz + c];
                            f[0] += Gd * gyz;          // s, d/dx
                            f[1] += Gs * gdy * gz;     // s, d/dy
                            f[2] += Gs * gy * gdz;     // s, d/dz
                            if (nproj > 1) {
                                const T hdy = fy[3 * two_ny + b], hdz = fz[3 * two_nz + c];
                                f[3] += Hd * gyz;          // p_x
                                f[4] += Hs * gdy * gz;
                                f[5] += Hs * gy * gdz;
                                f[6] += Gd * hy * gz;      // p_y
                                f[7] += Gs * hdy * gz;
                                f[8] += Gs * hy * gdz;
                                f[9] += Gd * gy * hz;      // p_z
                                f[10] += Gs * gdy * hz;
                                f[11] += Gs * gy * hdz;
                            }
                        }
                    }
                    if (need_dots) {
                        s0 = warp_sum(s0);
                        if (nproj > 1) {
                            spx = warp_sum(spx);
                            spy = warp_sum(spy);
                            spz = warp_sum(spz);
                        }
                        if (lane == 0) {
                            sdot[4 * t + 0] = s0;
                            sdot[4 * t + 1] = spx;
                            sdot[4 * t + 2] = spy;
                            sdot[4 * t + 3] = spz;
                        }
                    }
                    if (frc) {
                        const int nf = nproj > 1 ? 12 : 3;
#pragma unroll
                        for (int i = 0; i < 12; i++)
                            if (i < nf) f[i] = warp_sum(f[i]);
                        if (lane < nf) {
                            T mine = f[0];
#pragma unroll
                            for (int i = 1; i < 12; i++)
                                if (lane == i) mine = f[i];
                            const int lm = lane / 3, d = lane % 3;
                            const double val = chiq[4 * r.fidx + lm] * args.Nnorm * (double)mine;
                            atomicAdd(args.A + ((((size_t)k * natom + r.J) * nproj + lm) * 3 + d), val);
                        }
                    }
                }
            }
        };
        // phase 2: O = ca Hhat X - cb Z (O may alias Z), KB term from the dots of X
        auto update = [&](const T *X, const T *Z, T *O, T ca, T cb) {
            for (int sg = threadIdx.x; sg < nseg; sg += BLOCK) {
                const int sx = sg % nsx;
                const int rest = sg / nsx;
                const int b = rest % ncy;
                const int c = rest / ncy;
                const int a0 = sx * kSeg;
                const int rowbase = (c * ncy + b) * ncx;
                T cen[kSeg + 2 * P];
#pragma unroll
                for (int i = 0; i < kSeg + 2 * P; i++) {
                    const int a = a0 - P + i;
                    cen[i] = (a >= 0 && a < ncx) ? X[rowbase + a] : T(0);
                }
                T acc[kSeg];
                const T *drow = args.dpad + dbase + (size_t)c * plane_p + (size_t)b * args.pn[0];
#pragma unroll
                for (int s = 0; s < kSeg; s++) {
                    const int a = a0 + s;
                    T sum = 0;
                    if (a < ncx) {
                        sum = drow[a] * cen[P + s];
#pragma unroll
                        for (int j = 1; j <= P; j++) sum += args.w[0][j - 1] * (cen[P + s + j] + cen[P + s - j]);
#pragma unroll
                        for (int j = 1; j <= P; j++) {
                            const T yp = (b + j < ncy) ? X[rowbase + a + j * ncx] : T(0);
                            const T ym = (b - j >= 0) ? X[rowbase + a - j * ncx] : T(0);
                            sum += args.w[1][j - 1] * (yp + ym);
                        }
#pragma unroll
                        for (int j = 1; j <= P; j++) {
                            const T zp = (c + j < ncz) ? X[rowbase + a + j * ncx * ncy] : T(0);
                            const T zm = (c - j >= 0) ? X[rowbase + a - j * ncx * ncy] : T(0);
                            sum += args.w[2][j - 1] * (zp + zm);
                        }
                    }
                    acc[s] = sum;
                }
                // Kleinman-Bylander term, gathered from the atoms whose support box covers this
                // segment (intersection of the row, plane and segment coverage masks)
                for (int w = 0; w < maskw; w++) {
                    unsigned msk = ymask[b * maskw + w] & zmask[c * maskw + w] & xmask[sx * maskw + w];
                    while (msk) {
                        const int t = 32 * w + __ffs(msk) - 1;
                        msk &= msk - 1u;
                        const int bx = act[t].base[0], by = act[t].base[1], bz = act[t].base[2];
                        const T *fx = args.fac + bx;
                        const T gy = args.fac[by + b], gz = args.fac[bz + c];
                        const T s0 = sdot[4 * t];
                        T alpha = args.kappa[0] * s0 * gy * gz;
                        T beta = 0;
                        if (nproj > 1) {
                            const T hy = args.fac[by + two_ny + b];
                            const T hz = args.fac[bz + two_nz + c];
                            alpha += args.kappa[1] * (sdot[4 * t + 2] * hy * gz + sdot[4 * t + 3] * gy * hz);
                            beta = args.kappa[1] * sdot[4 * t + 1] * gy * gz;
                        }
#pragma unroll
                        for (int s = 0; s < kSeg; s++) {
                            const int a = a0 + s;
                            if (a < ncx) {
                                T add = fx[a] * alpha;
                                if (nproj > 1) add += fx[two_nx + a] * beta;
                                acc[s] += add;
                            }
                        }
                    }
                }
#pragma unroll
                for (int s = 0; s < kSeg; s++) {
                    const int a = a0 + s;
                    if (a < ncx) {
                        const int idx = rowbase + a;
                        O[idx] = ca * acc[s] - cb * Z[idx];
                    }
                }
            }
        };
        if constexpr (LANCZOS) {
            // Lanczos iteration (Eq. Lanczos) from v_0 = e_q, v_{-1} = 0:
            //   a_{k+1} = (Hhat v_k, v_k),  r = Hhat v_k - a_{k+1} v_k - b_k v_{k-1},  b_{k+1} = ||r||,
            //   v_{k+1} = r / b_{k+1}.
            // The operator phase writes Hhat v_k - b_k v_{k-1} over v_{k-1}, so a_{k+1} is formed as
            // (that, v_k) + b_k (v_{k-1}, v_k), the second dot carried over from the previous step's
            // normalisation; sums in FP64, two CTA reductions per step.
            __shared__ double2 lred[32];
            const int K = args.K;
            double bprev = 0.0, cross = 0.0;   // cross: this thread's part of (v_{k-1}, v_k)
            bool done = false;
            for (int k = 0; k < K; k++) {
                if (done) {
                    if (threadIdx.x == 0) {
                        args.ab[(size_t)k * N_d + q] = 0.0;
                        args.ab[(size_t)(K + k) * N_d + q] = 0.0;
                    }
                    continue;
                }
                dots(vcur, 0, true);
                __syncthreads();
                update(vcur, vprev, vprev, T(1), (T)bprev);
                __syncthreads();
                double s = 0.0;
                for (int i = threadIdx.x; i < nc3; i += BLOCK) s += (double)vprev[i] * (double)vcur[i];
                const double2 t = block_sum2(make_double2(s, cross), lred);
                const double alpha = t.x + bprev * t.y;
                s = 0.0;
                for (int i = threadIdx.x; i < nc3; i += BLOCK) {
                    const T r = vprev[i] - (T)alpha * vcur[i];
                    vprev[i] = r;
                    s += (double)r * (double)r;
                }
                const double beta = sqrt(block_sum2(make_double2(s, 0.0), lred).x);
                if (threadIdx.x == 0) {
                    args.ab[(size_t)k * N_d + q] = alpha;
                    args.ab[(size_t)(K + k) * N_d + q] = beta;
                }
                if (beta == 0.0) {   // exhausted Krylov space (the same value in every thread)
                    done = true;
                    continue;
                }
                cross = 0.0;
                for (int i = threadIdx.x; i < nc3; i += BLOCK) {
                    const T nv = (T)((double)vprev[i] / beta);
                    vprev[i] = nv;
                    cross += (double)vcur[i] * (double)nv;
                }
                __syncthreads();
                T *sw = vprev;
                vprev = vcur;
                vcur = sw;
                bprev = beta;
            }
        } else if constexpr (!ADJ) {
            for (int k = 0; k <= args.K; k++) {
                dots(vcur, k, k < args.K);
                if (k == args.K) break;
                __syncthreads();
                update(vcur, vprev, vprev, k == 0 ? T(1) : T(2), k == 0 ? T(0) : T(1));
                __syncthreads();
                T *sw = vprev;
                vprev = vcur;
                vcur = sw;
                if (threadIdx.x == 0) args.mu[(size_t)(k + 1) * N_d + q] = vcur[centre];
            }
        } else {
            adjoint_column<T>(args, q, centre, dots, update, va, vb, scratch + 2 * (size_t)nc3);
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace sq
