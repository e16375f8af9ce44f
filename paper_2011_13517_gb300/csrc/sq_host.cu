// libsq: C ABI entry points, set-up kernels (projector tables, bounds), moment sums, the Fermi-level
// bisection and the observables.  The per-column recursion lives in sq_recursion.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include "sq_gauss_rule.h"
#include "sq_internal.h"

using namespace sq;

// ------------------------------------------------------------------------------------------------
// error reporting

static thread_local char g_last_error[512] = "";

static sq_status fail(sq_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

#define SQ_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? SQ_ERR_OOM : SQ_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                    \
    } while (0)

extern "C" const char *sq_last_error(void) { return g_last_error; }

// number of kernels launched by this library (host-side count of launch sites executed)
static long long g_launches = 0;
#define SQ_COUNT(n) (g_launches += (n))

extern "C" long long sq_kernel_launches(void) { return g_launches; }

void sq::count_launches(long long n) { g_launches += n; }

extern "C" const char *sq_status_string(sq_status s)
{
    switch (s) {
    case SQ_OK: return "ok";
    case SQ_ERR_ARG: return "invalid argument";
    case SQ_ERR_CUBE_EXCEEDS_BOX: return "truncation cube plus stencil reach exceeds the periodic box";
    case SQ_ERR_NO_BRACKET: return "electron count not bracketed by the spectral bounds";
    case SQ_ERR_NOT_FINITE: return "non-finite input or result";
    case SQ_ERR_CUDA: return "CUDA runtime error";
    case SQ_ERR_TIMEOUT: return "bounded device wait timed out";
    case SQ_ERR_OOM: return "device allocation failed";
    case SQ_ERR_STATE: return "call made in the wrong state";
    case SQ_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

// ------------------------------------------------------------------------------------------------
// handle

struct sq_handle_s {
    int dev = 0;
    int num_sms = 0;
    int n[3] = {0, 0, 0};
    double L[3] = {0, 0, 0}, h[3] = {0, 0, 0}, dV = 0;
    int fd_order = 0, p = 0;
    double fd[kMaxHalfWidth + 1] = {0};
    int m[3] = {0, 0, 0}, nc[3] = {0, 0, 0};
    long long N_d = 0;
    int nc3 = 0;
    int natom = 0, lmax = 0, nproj = 1;
    double sigma = 0, rc = 0, cl[2] = {0, 0}, Nnorm = 0;
    double lmin = 0, lmax_ = 0, omega = 0, tau = 0, kdiag = 0;
    // device set-up data
    double *d_veff = nullptr;       // [N_d]
    double *d_fac64 = nullptr;      // [natom][3][4][n_a]
    double *d_fac2_64 = nullptr;    // doubled FP64 tables
    float *d_fac2_32 = nullptr;     // doubled FP32 tables
    int *d_sup = nullptr;           // [natom][3] start, then [natom][3] len
    int fac64_off[3] = {0, 0, 0}, fac64_stride = 0;
    int fac2_off[3] = {0, 0, 0}, fac2_stride = 0;
    double *d_dpad64 = nullptr;
    float *d_dpad32 = nullptr;
    int pn[3] = {0, 0, 0};
    double *d_small = nullptr;      // small scratch: reductions, bisection state
    // density state
    int have_density = 0, K = 0, precision = 0, have_force = 0;
    int have_moments = 0;           // moments of columns [q0, q1) are in d_mu, their sums in d_msum
    int gauss = 0;                  // the last sq_density used Gauss (Lanczos) quadrature
    double gU = 0, gS = 0;          // Gauss path: U and S at the last Fermi level
    double *d_ab = nullptr;         // Gauss path: Lanczos coefficients [2K][N_d]
    size_t ab_cap = 0;
    double *d_gnode = nullptr;      // Gauss path: nodes [K][N_d] then weights [K][N_d]
    size_t gnode_cap = 0;
    long long q0 = 0, q1 = 0;
    double kT = 0, N_e = 0, lam_f = 0;
    int M = 0;
    void *d_mu = nullptr;
    size_t mu_bytes = 0;
    double *d_msum = nullptr, *d_msum_part = nullptr;
    size_t msum_cap = 0, part_cap = 0;
    double *d_A = nullptr;
    size_t A_cap = 0;
    double *d_coef = nullptr;       // [3][K+1]: c, d, e
    size_t coef_cap = 0;
    double *d_nodes = nullptr;      // [3][M]: lambda_j, D_j, scratch f_j
    size_t nodes_cap = 0;
    void *d_scratch = nullptr;      // per-CTA vectors when not in shared memory
    size_t scratch_cap = 0;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int kernel_used = 0;            // 0: generic recursion kernel, 1: FP32 slab kernel, 2: FP32 cluster kernel
                                    // (tensor-core projector term), 3: Lanczos kernel, 4: FP32 cluster kernel
                                    // (CUDA-core projector term)
    int kb_fma = 0;                 // SQ_KB_FMA of the last sq_density / sq_moments_range call
    float t_rec = 0, t_msum = 0, t_fermi = 0;
};

template <typename P>
static sq_status ensure(P **ptr, size_t *cap, size_t bytes)
{
    if (*cap >= bytes && *ptr) return SQ_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc((void **)ptr, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) return fail(SQ_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    *cap = bytes;
    return SQ_OK;
}

// ------------------------------------------------------------------------------------------------
// set-up kernels

// Periodised 1D projector factors g, hp, g', hp' of atom J on axis a at grid index i (FP64).
__global__ void k_factors(int natom, const double *R, double L0, double L1, double L2, int n0, int n1, int n2,
                          double sigma, double rc, double *fac64, int stride, int off0, int off1, int off2)
{
    const int n[3] = {n0, n1, n2};
    const double Lx[3] = {L0, L1, L2};
    const int off[3] = {off0, off1, off2};
    const int total = n0 + n1 + n2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)natom * total;
         t += (long long)gridDim.x * blockDim.x) {
        const int J = (int)(t / total);
        int r = (int)(t % total);
        int a = 0;
        while (r >= n[a]) {
            r -= n[a];
            a++;
        }
        const int i = r;
        const double La = Lx[a];
        const double h = La / n[a];
        const double x = i * h;
        const double Ra = R[3 * J + a];
        const double pf = sqrt(2.0) / sigma;
        double sg = 0, sh = 0, sgd = 0, shd = 0;
        const int lo = (int)floor((x - Ra - rc) / La) - 1;
        const int hi = (int)ceil((x - Ra + rc) / La) + 1;
        for (int im = lo; im <= hi; im++) {
            const double tt = x - Ra - im * La;
            if (fabs(tt) >= rc) continue;
            const double u = 1.0 - tt * tt / (rc * rc);
            const double e = exp(-tt * tt / (2.0 * sigma * sigma));
            const double w = e * u * u * u;
            const double wd = e * (-tt / (sigma * sigma) * u * u * u - 6.0 * tt / (rc * rc) * u * u);
            sg += w;
            sgd += wd;
            sh += pf * tt * w;
            shd += pf * (w + tt * wd);
        }
        double *base = fac64 + (size_t)J * stride + off[a];
        base[0 * n[a] + i] = sg;
        base[1 * n[a] + i] = sh;
        base[2 * n[a] + i] = sgd;
        base[3 * n[a] + i] = shd;
    }
}

// Support (periodic interval where g != 0) of atom J on axis a: start and length.
// Central first-derivative weights a_1..a_p of order 2p (host side, closed form).
struct Fd1Weights {
    double a[kMaxHalfWidth + 1];
    int p;
};

// SQ_GRAD_FD: the derivative factors g', hp' of every atom and axis replaced by the periodic central
// first difference of g, hp (order 2p, the order of the Laplacian), so the force moments contract
// D_h chi instead of the analytic gradient (Sec. 3 "Atomic forces", discrete nonlocal force).
__global__ void k_fd_gradient(int natom, double *fac64, int stride, int off0, int off1, int off2, int n0, int n1,
                              int n2, double h0, double h1, double h2, Fd1Weights wt)
{
    const long long per_atom = (long long)n0 + n1 + n2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < natom * per_atom;
         t += (long long)gridDim.x * blockDim.x) {
        const int J = (int)(t / per_atom);
        int r = (int)(t % per_atom);
        int ax = 0;
        if (r >= n0) { r -= n0; ax = 1; }
        if (ax == 1 && r >= n1) { r -= n1; ax = 2; }
        const int n = ax == 0 ? n0 : (ax == 1 ? n1 : n2);
        const double h = ax == 0 ? h0 : (ax == 1 ? h1 : h2);
        double *base = fac64 + (size_t)J * stride + (ax == 0 ? off0 : (ax == 1 ? off1 : off2));
        double sg = 0.0, sh = 0.0;
        for (int j = 1; j <= wt.p; j++) {
            const int ip = (r + j) % n, im = ((r - j) % n + n) % n;
            sg += wt.a[j] * (base[ip] - base[im]);
            sh += wt.a[j] * (base[n + ip] - base[n + im]);
        }
        base[2 * n + r] = sg / h;
        base[3 * n + r] = sh / h;
    }
}

// Support interval of every atom's factor g along each axis (start, length); with widen > 0 the
// interval is extended by widen points on both sides (the reach of the FD gradient of SQ_GRAD_FD,
// whose derivative tables are nonzero up to p points outside the support of g).
__global__ void k_support(int natom, const double *fac64, int stride, int off0, int off1, int off2, int n0,
                          int n1, int n2, int *sup, int *bad, int widen)
{
    const int n[3] = {n0, n1, n2};
    const int off[3] = {off0, off1, off2};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < natom * 3; t += gridDim.x * blockDim.x) {
        const int J = t / 3, a = t % 3;
        const double *g = fac64 + (size_t)J * stride + off[a];
        int cnt = 0, starts = 0, st = 0;
        for (int i = 0; i < n[a]; i++) {
            const bool on = g[i] != 0.0;
            const bool prev = g[(i + n[a] - 1) % n[a]] != 0.0;
            cnt += on;
            if (on && !prev) {
                starts++;
                st = i;
            }
        }
        if (cnt == n[a]) st = 0;
        else if (starts != 1) atomicExch(bad, 1);
        if (widen > 0 && cnt < n[a]) {
            st = ((st - widen) % n[a] + n[a]) % n[a];
            cnt = cnt + 2 * widen < n[a] ? cnt + 2 * widen : n[a];
            if (cnt == n[a]) st = 0;
        }
        sup[J * 3 + a] = st;
        sup[natom * 3 + J * 3 + a] = cnt;
    }
}

// Doubled tables in precision T: element (J, a, f, i), i < 2 n_a, = fac64(J, a, f, i mod n_a).
template <typename T>
__global__ void k_double_tables(int natom, const double *fac64, int s64, int o0, int o1, int o2, int n0, int n1,
                                int n2, T *fac2, int s2, int p0, int p1, int p2)
{
    const int n[3] = {n0, n1, n2};
    const int o64[3] = {o0, o1, o2};
    const int o2x[3] = {p0, p1, p2};
    const int per = 2 * kNumFactors * (n0 + n1 + n2);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)natom * per;
         t += (long long)gridDim.x * blockDim.x) {
        const int J = (int)(t / per);
        int r = (int)(t % per);
        int a = 0;
        while (r >= 2 * kNumFactors * n[a]) {
            r -= 2 * kNumFactors * n[a];
            a++;
        }
        const int f = r / (2 * n[a]);
        const int i = r % (2 * n[a]);
        fac2[(size_t)J * s2 + o2x[a] + f * 2 * n[a] + i] =
            (T)fac64[(size_t)J * s64 + o64[a] + f * n[a] + (i % n[a])];
    }
}

// min and max of V_eff, and a non-finite flag; out[0] = min, out[1] = max (as ordered bit patterns)
__global__ void k_vrange(const double *v, long long n, unsigned long long *mn, unsigned long long *mx, int *bad)
{
    double lo = INFINITY, hi = -INFINITY;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = v[i];
        if (!isfinite(x)) atomicExch(bad, 1);
        lo = fmin(lo, x);
        hi = fmax(hi, x);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        // order-preserving map of doubles onto unsigned integers
        auto key = [](double d) {
            unsigned long long b = (unsigned long long)__double_as_longlong(d);
            return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
        };
        atomicMin(mn, key(lo));
        atomicMax(mx, key(hi));
    }
}

// Gershgorin bound of the weighted projector Gram matrix: max_P sum_P' sqrt|c_P c_P'| dV |<chi_P, chi_P'>|
__global__ void k_gram_bound(int natom, int nproj, const double *fac64, int stride, int o0, int o1, int o2,
                             int n0, int n1, int n2, double c0, double c1, double scale, unsigned long long *out)
{
    const int n[3] = {n0, n1, n2};
    const int off[3] = {o0, o1, o2};
    const int P = blockIdx.x;
    if (P >= natom * nproj) return;
    const int J = P / nproj, lm = P % nproj;
    const double cP = fabs(lm == 0 ? c0 : c1);
    double row = 0.0;
    for (int Q = threadIdx.x; Q < natom * nproj; Q += blockDim.x) {
        const int J2 = Q / nproj, lm2 = Q % nproj;
        const double cQ = fabs(lm2 == 0 ? c0 : c1);
        double prod = 1.0;
        for (int a = 0; a < 3; a++) {
            const double *f1 = fac64 + (size_t)J * stride + off[a] + (lm == 1 + a ? 1 : 0) * n[a];
            const double *f2 = fac64 + (size_t)J2 * stride + off[a] + (lm2 == 1 + a ? 1 : 0) * n[a];
            double s = 0.0;
            for (int i = 0; i < n[a]; i++) s += f1[i] * f2[i];
            prod *= s;
        }
        row += sqrt(cP * cQ) * fabs(prod);
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) row += __shfl_xor_sync(0xffffffffu, row, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = row;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        atomicMax(out, (unsigned long long)__double_as_longlong(s * scale));  // s >= 0
    }
}

// Hhat diagonal on the padded grid: (kdiag + V(g) - omega)/tau, g = padded index - m (periodic)
template <typename T>
__global__ void k_dpad(const double *veff, int n0, int n1, int n2, int m0, int m1, int m2, double kdiag,
                       double omega, double tau, T *dpad)
{
    const int p0 = n0 + 2 * m0, p1 = n1 + 2 * m1, p2 = n2 + 2 * m2;
    const long long tot = (long long)p0 * p1 * p2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % p0);
        const int j = (int)((t / p0) % p1);
        const int k = (int)(t / ((long long)p0 * p1));
        const int g0 = ((i - m0) % n0 + n0) % n0;
        const int g1 = ((j - m1) % n1 + n1) % n1;
        const int g2 = ((k - m2) % n2 + n2) % n2;
        const double v = veff[g0 + (long long)n0 * (g1 + (long long)n1 * g2)];
        dpad[t] = (T)((kdiag + v - omega) / tau);
    }
}

// ------------------------------------------------------------------------------------------------
// moment sums M_k = sum_q mu_k^q (FP64, deterministic two-stage reduction)

constexpr int kSumBlocks = 64;

template <typename T>
__global__ void k_msum_partial(const T *mu, long long N_d, int K, double *part, long long q0, long long q1)
{
    const int k = blockIdx.y;
    double s = 0.0;
    for (long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; q < q1; q += (long long)gridDim.x * blockDim.x)
        s += (double)mu[(size_t)k * N_d + q];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        part[(size_t)k * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void k_msum_final(const double *part, int nblk, int K, double *msum, int *bad)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++) s += part[(size_t)k * nblk + b];
        if (!isfinite(s)) atomicExch(bad, 1);
        msum[k] = s;
    }
}

// ------------------------------------------------------------------------------------------------
// Fermi level.  Nodes x_j = cos(theta_j), theta_j = pi (j + 1/2)/M;
// D_j = sum_k (2 - delta_k0)/M M_k cos(k theta_j), so that N(lambda_f) = 2 sum_k c_k M_k
// = 2 sum_j g(tau x_j + omega; lambda_f) D_j.

__device__ __forceinline__ double cos_k_theta(int k, int j, int M)
{
    // cos(k pi (2j+1)/(2M)) with exact argument reduction modulo 2 pi
    const long long r = ((long long)k * (2LL * j + 1)) % (4LL * M);
    return cospi((double)r / (2.0 * M));
}

__device__ __forceinline__ double fermi_fn(double lam, double lam_f, double kT)
{
    return 0.5 * (1.0 - tanh((lam - lam_f) / (2.0 * kT)));
}

__global__ void k_nodes(const double *msum, int K, int M, double omega, double tau, double *lam, double *D)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        lam[j] = tau * cospi((j + 0.5) / M) + omega;
        double s = msum[0];
        for (int k = 1; k <= K; k++) s += 2.0 * msum[k] * cos_k_theta(k, j, M);
        D[j] = s / M;
    }
}

struct FermiState {
    double lo, hi;        // bracket
    double x;             // current evaluation point
    double N_lo, N_hi;    // values at the bracket ends (diagnostics)
    int phase;            // 0: evaluate at lo, 1: at hi, 2: bisecting, 3: done, 4: no bracket
    int iter;
    unsigned int arrived; // last-block counter
    int pad;
};

constexpr int kFermiBlocks = 96;

// One bisection step: all blocks sum 2 g(lam_j) D_j at the state's point; the last block to finish
// reduces the per-block partials in fixed order and advances the state.  Sequence:
// phase 0 evaluates N(lo), phase 1 N(hi) (bracket check), phase 2 bisects
// (mid = lo + (hi-lo)/2; N(mid) < N_e -> lo = mid else hi = mid) until the midpoint no longer
// separates the bracket.
__global__ void k_fermi_step(const double *lam, const double *D, int M, double kT, double N_e, FermiState *st,
                             double *part)
{
    __shared__ double red[32];
    __shared__ bool last;
    const int phase = st->phase;
    if (phase >= 3) return;
    double x;
    if (phase == 0) x = st->lo;
    else if (phase == 1) x = st->hi;
    else x = st->lo + 0.5 * (st->hi - st->lo);
    double s = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
        s += fermi_fn(lam[j], x, kT) * D[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        part[blockIdx.x] = t;
        __threadfence();
        const unsigned int prev = atomicAdd(&st->arrived, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double N = 0.0;
    for (int b = 0; b < (int)gridDim.x; b++) N += ((volatile double *)part)[b];
    N *= 2.0;
    st->arrived = 0;
    if (phase == 0) {
        st->N_lo = N;
        st->phase = (N > N_e) ? 4 : 1;
    } else if (phase == 1) {
        st->N_hi = N;
        st->phase = (N < N_e) ? 4 : 2;
    } else {
        if (N < N_e) st->lo = x;
        else st->hi = x;
        st->iter++;
        const double nm = st->lo + 0.5 * (st->hi - st->lo);
        if (nm <= st->lo || nm >= st->hi || st->iter >= 200) {
            st->x = nm;
            st->phase = 3;
        }
    }
}

// f_j for the three expansions: g, lam g, s(g) at the Fermi level
__global__ void k_node_functions(const double *lam, int M, double lam_f, double kT, double *fg, double *flg,
                                 double *fs)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const double l = lam[j];
        const double g = fermi_fn(l, lam_f, kT);
        const double y = fabs((l - lam_f) / kT);
        fg[j] = g;
        flg[j] = l * g;
        fs[j] = -(log1p(exp(-y)) + y * fermi_fn(y, 0.0, 1.0));
    }
}

// a_k = (2 - delta_k0)/M sum_j f_j cos(k theta_j) for the three functions (block per (k, function))
__global__ void k_coeffs(const double *f0, const double *f1, const double *f2, int M, int K, double *coef)
{
    const int k = blockIdx.x, which = blockIdx.y;
    const double *f = which == 0 ? f0 : (which == 1 ? f1 : f2);
    double s = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) s += f[j] * cos_k_theta(k, j, M);
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        coef[which * (K + 1) + k] = t * (k == 0 ? 1.0 : 2.0) / M;
    }
}

// rho(x_q) = 2 sum_k c_k mu_k^q / dV for q in [q0, q1), written to rho[q - q0]
template <typename T>
__global__ void k_density(const T *mu, long long N_d, int K, const double *c, double inv_dV, double *rho,
                          long long q0, long long q1)
{
    __shared__ double cs[512];
    for (int k = threadIdx.x; k <= K && k < 512; k += blockDim.x) cs[k] = c[k];
    __syncthreads();
    for (long long q = q0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; q < q1; q += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k <= K; k++) s += (k < 512 ? cs[k] : c[k]) * (double)mu[(size_t)k * N_d + q];
        rho[q - q0] = 2.0 * s * inv_dV;
    }
}

// U = 2 sum d_k M_k, S = -2 sum e_k M_k
__global__ void k_energy(const double *msum, const double *coef, int K, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double U = 0.0, S = 0.0;
    for (int k = 0; k <= K; k++) {
        U += coef[(K + 1) + k] * msum[k];
        S += coef[2 * (K + 1) + k] * msum[k];
    }
    out[0] = 2.0 * U;
    out[1] = -2.0 * S;
}

// f_J,d = 4 dV sum_lm c_l sum_k c_k A_k^{J,lm,d}
__global__ void k_force(const double *A, const double *c, int K, int natom, int nproj, double c0, double c1,
                        double dV, double *force)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < natom * 3; t += gridDim.x * blockDim.x) {
        const int J = t / 3, d = t % 3;
        double f = 0.0;
        for (int lm = 0; lm < nproj; lm++) {
            double s = 0.0;
            for (int k = 0; k <= K; k++) s += c[k] * A[(((size_t)k * natom + J) * nproj + lm) * 3 + d];
            f += (lm == 0 ? c0 : c1) * s;
        }
        force[t] = 4.0 * dV * f;
    }
}

// Gauss path (Sec. 2.2, Eqs. rhoq, uq, sq): rho(x_q) = 2 sum_k w_k g(lambda_k) / dV over the column's
// nodes; U = 2 sum_q sum_k w lambda g and S = -2 sum_q sum_k w s(lambda) over all nodes (FP64,
// deterministic two-stage sums).
__global__ void k_gauss_density(const double *nodes, const double *weights, long long N_d, int K, double lam_f,
                                double kT, double inv_dV, double *rho)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N_d; q += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < K; k++) s += weights[(size_t)k * N_d + q] * fermi_fn(nodes[(size_t)k * N_d + q], lam_f, kT);
        rho[q] = 2.0 * s * inv_dV;
    }
}

__device__ __forceinline__ double entropy_fn(double lam, double lam_f, double kT)
{
    // s(g) = g ln g + (1-g) ln(1-g) in the overflow-free form -(log1p(e^-|y|) + |y| g(|y|)), y = (lam - lam_f)/kT
    const double y = fabs((lam - lam_f) / kT);
    return -(log1p(exp(-y)) + y * fermi_fn(y, 0.0, 1.0));
}

__global__ void k_gauss_energy_partial(const double *nodes, const double *weights, long long n, double lam_f, double kT,
                                       double *part)
{
    double u = 0.0, sv = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double l = nodes[i], w = weights[i];
        u += w * l * fermi_fn(l, lam_f, kT);
        sv += w * entropy_fn(l, lam_f, kT);
    }
    __shared__ double r0[32], r1[32];
    for (int o = 16; o > 0; o >>= 1) {
        u += __shfl_xor_sync(0xffffffffu, u, o);
        sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r0[threadIdx.x >> 5] = u;
        r1[threadIdx.x >> 5] = sv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a += r0[w];
            b += r1[w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_gauss_energy_final(const double *part, int nblk, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nblk; i++) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    out[0] = 2.0 * a;
    out[1] = -2.0 * b;
}

__global__ void k_check_cols(const long long *cols, long long n, long long N_d, int *bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (cols[i] < 0 || cols[i] >= N_d) atomicExch(bad, 1);
}

// ------------------------------------------------------------------------------------------------
// host helpers

static void fd_coefficients(int order, double *c)
{
    // central second-derivative weights: c_j = 2 (-1)^(j+1) (p!)^2 / (j^2 (p-j)! (p+j)!)
    const int p = order / 2;
    double sum = 0.0;
    for (int j = 1; j <= p; j++) {
        double r = 1.0;
        for (int i = 1; i <= j; i++) r *= (double)(p - j + i) / (double)(p + i);
        c[j] = 2.0 * ((j % 2) ? 1.0 : -1.0) * r / ((double)j * j);
        sum += c[j];
    }
    c[0] = -2.0 * sum;
}

static Fd1Weights fd1_coefficients(int order)
{
    // central first-derivative weights: a_j = (-1)^(j+1) (p!)^2 / (j (p-j)! (p+j)!)
    Fd1Weights w;
    memset(&w, 0, sizeof(w));
    w.p = order / 2;
    for (int j = 1; j <= w.p; j++) {
        double r = 1.0;
        for (int i = 1; i <= j; i++) r *= (double)(w.p - j + i) / (double)(w.p + i);
        w.a[j] = ((j % 2) ? 1.0 : -1.0) * r / (double)j;
    }
    return w;
}

static double kinetic_max(const sq_handle_s *h)
{
    // eigenvalues of -1/2 Lap_h on the periodic grid: sum_i -(c_0 + 2 sum_j c_j cos(j theta)) / (2 h_i^2)
    double tot = 0.0;
    for (int a = 0; a < 3; a++) {
        double best = -INFINITY;
        for (int k = 0; k < h->n[a]; k++) {
            const double th = 2.0 * M_PI * k / h->n[a];
            double s = h->fd[0];
            for (int j = 1; j <= h->p; j++) s += 2.0 * h->fd[j] * cos(j * th);
            best = fmax(best, -s / (2.0 * h->h[a] * h->h[a]));
        }
        tot += best;
    }
    return tot;
}

static double key_to_double(unsigned long long k)
{
    unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

static int grid_for(long long work, int block, int num_sms)
{
    long long g = (work + block - 1) / block;
    long long cap = (long long)num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// ------------------------------------------------------------------------------------------------
// ABI

extern "C" sq_status sq_build_hamiltonian(const sq_grid *grid, const double *d_veff, const sq_atoms *atoms,
                                          double R_cut, int flags, double lambda_min, double lambda_max,
                                          void *stream_, sq_handle *out)
{
    g_last_error[0] = 0;
    if (!grid || !d_veff || !atoms || !out) return fail(SQ_ERR_ARG, "null argument");
    if (flags & ~SQ_GRAD_FD) return fail(SQ_ERR_ARG, "flags %d", flags);
    cudaStream_t stream = (cudaStream_t)stream_;
    for (int a = 0; a < 3; a++)
        if (grid->n[a] < 1 || !(grid->L[a] > 0) || !std::isfinite(grid->L[a]))
            return fail(SQ_ERR_ARG, "grid axis %d: n=%d L=%g", a, grid->n[a], grid->L[a]);
    if (grid->fd_order < 2 || grid->fd_order % 2 || grid->fd_order / 2 > kMaxHalfWidth)
        return fail(grid->fd_order > 2 * kMaxHalfWidth ? SQ_ERR_UNSUPPORTED : SQ_ERR_ARG, "fd_order %d", grid->fd_order);
    if (atoms->natom < 0 || (atoms->natom > 0 && !atoms->R) || (atoms->lmax != 0 && atoms->lmax != 1) ||
        !(atoms->sigma > 0) || !(atoms->rc > 0) || !atoms->energy)
        return fail(SQ_ERR_ARG, "atoms: natom=%d lmax=%d sigma=%g rc=%g", atoms->natom, atoms->lmax, atoms->sigma,
                    atoms->rc);
    if (!(R_cut >= 0) || !std::isfinite(R_cut)) return fail(SQ_ERR_ARG, "R_cut %g", R_cut);
    for (int i = 0; i < 3 * atoms->natom; i++)
        if (!std::isfinite(atoms->R[i])) return fail(SQ_ERR_NOT_FINITE, "atom position %d", i);
    const bool want_bounds = std::isnan(lambda_min) || std::isnan(lambda_max);
    if (!want_bounds && !(lambda_max > lambda_min)) return fail(SQ_ERR_ARG, "lambda_max <= lambda_min");

    sq_handle_s *h = new sq_handle_s();
    auto cleanup = [&](sq_status s) {
        sq_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->dev) != cudaSuccess) return cleanup(fail(SQ_ERR_CUDA, "no CUDA device"));
    for (int i = 0; i < 5; i++) SQ_CUDA(cudaEventCreate(&h->ev[i]));
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev);
    h->fd_order = grid->fd_order;
    h->p = grid->fd_order / 2;
    fd_coefficients(h->fd_order, h->fd);
    h->N_d = 1;
    h->dV = 1.0;
    h->kdiag = 0.0;
    for (int a = 0; a < 3; a++) {
        h->n[a] = grid->n[a];
        h->L[a] = grid->L[a];
        h->h[a] = grid->L[a] / grid->n[a];
        h->dV *= h->h[a];
        h->N_d *= grid->n[a];
        h->m[a] = (int)std::nearbyint(R_cut / h->h[a]);
        h->nc[a] = 2 * h->m[a] + 1;
        h->kdiag += -h->fd[0] / (2.0 * h->h[a] * h->h[a]);
        if (h->nc[a] + h->p > h->n[a])
            return cleanup(fail(SQ_ERR_CUBE_EXCEEDS_BOX, "axis %d: 2m+1+p = %d > n = %d", a, h->nc[a] + h->p, h->n[a]));
        h->pn[a] = h->n[a] + 2 * h->m[a];
    }
    h->nc3 = h->nc[0] * h->nc[1] * h->nc[2];
    h->natom = atoms->natom;
    h->lmax = atoms->lmax;
    h->nproj = atoms->lmax == 0 ? 1 : 4;
    h->sigma = atoms->sigma;
    h->rc = atoms->rc;
    h->cl[0] = atoms->energy[0];
    h->cl[1] = atoms->lmax ? atoms->energy[1] : 0.0;
    if (!std::isfinite(h->cl[0]) || !std::isfinite(h->cl[1])) return cleanup(fail(SQ_ERR_NOT_FINITE, "KB energy"));
    h->Nnorm = pow(M_PI * h->sigma * h->sigma, -0.75);

    size_t cap = 0;
    sq_status s;
    if ((s = ensure(&h->d_veff, &cap, sizeof(double) * h->N_d))) return cleanup(s);
    SQ_CUDA(cudaMemcpyAsync(h->d_veff, d_veff, sizeof(double) * h->N_d, cudaMemcpyDeviceToDevice, stream));

    // projector tables
    h->fac64_off[0] = 0;
    h->fac64_off[1] = kNumFactors * h->n[0];
    h->fac64_off[2] = kNumFactors * (h->n[0] + h->n[1]);
    h->fac64_stride = kNumFactors * (h->n[0] + h->n[1] + h->n[2]);
    h->fac2_off[0] = 0;
    h->fac2_off[1] = 2 * kNumFactors * h->n[0];
    h->fac2_off[2] = 2 * kNumFactors * (h->n[0] + h->n[1]);
    h->fac2_stride = 2 * kNumFactors * (h->n[0] + h->n[1] + h->n[2]);
    const int na = h->natom > 0 ? h->natom : 1;
    double *d_R = nullptr;
    cap = 0;
    if ((s = ensure(&h->d_fac64, &cap, sizeof(double) * (size_t)na * h->fac64_stride))) return cleanup(s);
    cap = 0;
    if ((s = ensure(&h->d_fac2_64, &cap, sizeof(double) * (size_t)na * h->fac2_stride))) return cleanup(s);
    cap = 0;
    if ((s = ensure(&h->d_fac2_32, &cap, sizeof(float) * (size_t)na * h->fac2_stride))) return cleanup(s);
    cap = 0;
    if ((s = ensure(&h->d_sup, &cap, sizeof(int) * 6 * (size_t)na))) return cleanup(s);
    cap = 0;
    if ((s = ensure(&h->d_small, &cap, 4096))) return cleanup(s);
    SQ_CUDA(cudaMemsetAsync(h->d_small, 0, 4096, stream));
    int *d_bad = reinterpret_cast<int *>(h->d_small);
    unsigned long long *d_keys = reinterpret_cast<unsigned long long *>(h->d_small) + 8;
    if (h->natom > 0) {
        SQ_CUDA(cudaMalloc(&d_R, sizeof(double) * 3 * h->natom));
        SQ_CUDA(cudaMemcpyAsync(d_R, atoms->R, sizeof(double) * 3 * h->natom, cudaMemcpyHostToDevice, stream));
        const long long work = (long long)h->natom * (h->n[0] + h->n[1] + h->n[2]);
        SQ_COUNT(1);
        k_factors<<<grid_for(work, 256, h->num_sms), 256, 0, stream>>>(
            h->natom, d_R, h->L[0], h->L[1], h->L[2], h->n[0], h->n[1], h->n[2], h->sigma, h->rc, h->d_fac64,
            h->fac64_stride, h->fac64_off[0], h->fac64_off[1], h->fac64_off[2]);
        SQ_CUDA(cudaGetLastError());
        if (flags & SQ_GRAD_FD) {
            SQ_COUNT(1);
            k_fd_gradient<<<grid_for(work, 256, h->num_sms), 256, 0, stream>>>(
                h->natom, h->d_fac64, h->fac64_stride, h->fac64_off[0], h->fac64_off[1], h->fac64_off[2], h->n[0],
                h->n[1], h->n[2], h->h[0], h->h[1], h->h[2], fd1_coefficients(h->fd_order));
            SQ_CUDA(cudaGetLastError());
        }
        SQ_COUNT(1);
        k_support<<<grid_for(3LL * h->natom, 128, h->num_sms), 128, 0, stream>>>(
            h->natom, h->d_fac64, h->fac64_stride, h->fac64_off[0], h->fac64_off[1], h->fac64_off[2], h->n[0],
            h->n[1], h->n[2], h->d_sup, d_bad + 1, (flags & SQ_GRAD_FD) ? h->p : 0);
        SQ_CUDA(cudaGetLastError());
        const long long work2 = (long long)h->natom * h->fac2_stride;
        SQ_COUNT(2);
        k_double_tables<double><<<grid_for(work2, 256, h->num_sms), 256, 0, stream>>>(
            h->natom, h->d_fac64, h->fac64_stride, h->fac64_off[0], h->fac64_off[1], h->fac64_off[2], h->n[0],
            h->n[1], h->n[2], h->d_fac2_64, h->fac2_stride, h->fac2_off[0], h->fac2_off[1], h->fac2_off[2]);
        SQ_CUDA(cudaGetLastError());
        k_double_tables<float><<<grid_for(work2, 256, h->num_sms), 256, 0, stream>>>(
            h->natom, h->d_fac64, h->fac64_stride, h->fac64_off[0], h->fac64_off[1], h->fac64_off[2], h->n[0],
            h->n[1], h->n[2], h->d_fac2_32, h->fac2_stride, h->fac2_off[0], h->fac2_off[1], h->fac2_off[2]);
        SQ_CUDA(cudaGetLastError());
    }
    // V_eff range and finiteness
    {
        unsigned long long init[2] = {~0ull, 0ull};
        SQ_CUDA(cudaMemcpyAsync(d_keys, init, sizeof(init), cudaMemcpyHostToDevice, stream));
        SQ_COUNT(1);
        k_vrange<<<grid_for(h->N_d, 256, h->num_sms), 256, 0, stream>>>(h->d_veff, h->N_d, d_keys, d_keys + 1, d_bad);
        SQ_CUDA(cudaGetLastError());
    }
    if (want_bounds && h->natom > 0) {
        const double scale = h->dV * h->Nnorm * h->Nnorm;
        SQ_COUNT(1);
        k_gram_bound<<<h->natom * h->nproj, 256, 0, stream>>>(
            h->natom, h->nproj, h->d_fac64, h->fac64_stride, h->fac64_off[0], h->fac64_off[1], h->fac64_off[2],
            h->n[0], h->n[1], h->n[2], h->cl[0], h->cl[1], scale, d_keys + 2);
        SQ_CUDA(cudaGetLastError());
    }
    int bad[2];
    unsigned long long keys[3];
    SQ_CUDA(cudaMemcpyAsync(bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaMemcpyAsync(keys, d_keys, sizeof(keys), cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    if (d_R) cudaFree(d_R);
    if (bad[0]) return cleanup(fail(SQ_ERR_NOT_FINITE, "V_eff has non-finite values"));
    if (bad[1]) return cleanup(fail(SQ_ERR_ARG, "projector support is not a periodic interval"));
    if (want_bounds) {
        const double vmin = key_to_double(keys[0]), vmax = key_to_double(keys[1]);
        double nl = 0.0;
        if (h->natom > 0) memcpy(&nl, &keys[2], sizeof(nl));
        const bool cpos = h->cl[0] >= 0 && (h->nproj == 1 || h->cl[1] >= 0);
        const bool cneg = h->cl[0] <= 0 && (h->nproj == 1 || h->cl[1] <= 0);
        const double nlo = cpos ? 0.0 : -nl, nhi = cneg ? 0.0 : nl;
        h->lmin = vmin + nlo;
        h->lmax_ = kinetic_max(h) + vmax + nhi;
    } else {
        h->lmin = lambda_min;
        h->lmax_ = lambda_max;
    }
    h->omega = 0.5 * (h->lmax_ + h->lmin);
    h->tau = 0.5 * (h->lmax_ - h->lmin);
    *out = h;
    return SQ_OK;
}

extern "C" void sq_destroy(sq_handle h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->d_veff);
    cudaFree(h->d_fac64);
    cudaFree(h->d_fac2_64);
    cudaFree(h->d_fac2_32);
    cudaFree(h->d_sup);
    cudaFree(h->d_dpad64);
    cudaFree(h->d_dpad32);
    cudaFree(h->d_small);
    cudaFree(h->d_mu);
    cudaFree(h->d_msum);
    cudaFree(h->d_msum_part);
    cudaFree(h->d_A);
    cudaFree(h->d_coef);
    cudaFree(h->d_nodes);
    cudaFree(h->d_scratch);
    cudaFree(h->d_ab);
    cudaFree(h->d_gnode);
    for (int i = 0; i < 5; i++)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    delete h;
}

template <typename T>
static void fill_args(sq_handle h, int K, int want_force, RecursionArgs<T> &a)
{
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < 3; i++) {
        a.n[i] = h->n[i];
        a.m[i] = h->m[i];
        a.nc[i] = h->nc[i];
        a.pn[i] = h->pn[i];
        a.fac_off[i] = h->fac2_off[i];
        a.fac64_off[i] = h->fac64_off[i];
        for (int j = 1; j <= h->p; j++) a.w[i][j - 1] = (T)(-h->fd[j] / (2.0 * h->h[i] * h->h[i] * h->tau));
    }
    a.nc3 = h->nc3;
    a.N_d = h->N_d;
    a.q0 = 0;
    a.q1 = h->N_d;
    a.K = K;
    a.natom = h->natom;
    a.nproj = h->nproj;
    a.want_force = want_force;
    a.kb_fma = h->kb_fma;
    if constexpr (sizeof(T) == 8) {
        a.dpad = reinterpret_cast<const T *>(h->d_dpad64);
        a.fac = reinterpret_cast<const T *>(h->d_fac2_64);
    } else {
        a.dpad = reinterpret_cast<const T *>(h->d_dpad32);
        a.fac = reinterpret_cast<const T *>(h->d_fac2_32);
    }
    a.kappa[0] = (T)(h->cl[0] * h->dV * h->Nnorm * h->Nnorm / h->tau);
    a.kappa[1] = (T)(h->cl[1] * h->dV * h->Nnorm * h->Nnorm / h->tau);
    a.fac_stride = h->fac2_stride;
    a.fac64 = h->d_fac64;
    a.fac64_stride = h->fac64_stride;
    a.sup_start = h->d_sup;
    a.sup_len = h->d_sup + 3 * (h->natom > 0 ? h->natom : 1);
    a.Nnorm = h->Nnorm;
    a.mu = reinterpret_cast<T *>(h->d_mu);
    a.A = want_force ? h->d_A : nullptr;
}

template <typename T>
static sq_status run_recursion(sq_handle h, int K, int want_force, long long q0, long long q1, cudaStream_t stream,
                               const long long *cols = nullptr)
{
    sq_status s;
    const size_t pad = (size_t)h->pn[0] * h->pn[1] * h->pn[2];
    T **dpad = nullptr;
    if constexpr (sizeof(T) == 8) dpad = reinterpret_cast<T **>(&h->d_dpad64);
    else dpad = reinterpret_cast<T **>(&h->d_dpad32);
    if (!*dpad) {
        size_t cap = 0;
        if ((s = ensure(dpad, &cap, sizeof(T) * pad))) return s;
    }
    SQ_COUNT(1);
    k_dpad<T><<<grid_for((long long)pad, 256, h->num_sms), 256, 0, stream>>>(
        h->d_veff, h->n[0], h->n[1], h->n[2], h->m[0], h->m[1], h->m[2], h->kdiag, h->omega, h->tau, *dpad);
    SQ_CUDA(cudaGetLastError());

    RecursionArgs<T> a;
    fill_args<T>(h, K, want_force, a);
    a.dpad = *dpad;
    a.q0 = q0;
    a.q1 = q1;
    a.cols = cols;

    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    if constexpr (sizeof(T) == 4) if (!cols) {
        // FP32 on a cubic 29^3 cube with the 12th-order stencil: the two-CTA cluster kernel, sized by
        // the largest number of atoms touching one cube
        if (h->natom > 0 && cluster_supported(h->nc, h->p)) {
            int *d_cnt = reinterpret_cast<int *>(h->d_small) + 40;   // bytes 160..171 of the small scratch
            SQ_CUDA(cudaMemsetAsync(d_cnt, 0, 3 * sizeof(int), stream));
            SQ_COUNT(1);
            SQ_CUDA(slab_counts(a, d_cnt, h->num_sms, stream));
            int cnt[2];
            SQ_CUDA(cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, stream));
            SQ_CUDA(cudaStreamSynchronize(stream));
            const int amax = cnt[0] > 0 ? cnt[0] : 1, fmax = cnt[1] > 0 ? cnt[1] : 1;
            size_t sm = 0;
            int maxc = 0;
            if (cluster_prepare(h->nc[0], amax, fmax, a.kb_fma, &sm, &maxc) == cudaSuccess && sm <= (size_t)dev_smem &&
                maxc > 0) {
                long long ncl = maxc;
                if (ncl > q1 - q0) ncl = q1 - q0;
                if ((s = ensure(&h->d_scratch, &h->scratch_cap,
                                sizeof(float) * (size_t)cluster_scratch_floats(h->nc[0]) * 2 * ncl)))
                    return s;
                a.scratch = reinterpret_cast<T *>(h->d_scratch);
                h->kernel_used = a.kb_fma ? 4 : 2;
                SQ_CUDA(cudaEventRecord(h->ev[0], stream));
                SQ_COUNT(1);
                SQ_CUDA(launch_cluster(a, amax, fmax, (int)ncl, sm, d_cnt + 2, stream));
                SQ_CUDA(cudaEventRecord(h->ev[1], stream));
                dim3 g2(kSumBlocks, K + 1);
                SQ_COUNT(1);
                k_msum_partial<T><<<g2, 256, 0, stream>>>(reinterpret_cast<const T *>(h->d_mu), h->N_d, K,
                                                          h->d_msum_part, q0, q1);
                SQ_CUDA(cudaGetLastError());
                return SQ_OK;
            }
            cudaGetLastError();   // a configuration the cluster kernel cannot take falls through
        }
        // FP32 on a cubic 21^3 / 25^3 cube with the 12th-order stencil: the slab kernel, sized by the
        // largest number of atoms touching one cube
        if (h->natom > 0 && slab_supported(h->nc, h->p)) {
            int *d_cnt = reinterpret_cast<int *>(h->d_small) + 40;   // bytes 160..171 of the small scratch
            SQ_CUDA(cudaMemsetAsync(d_cnt, 0, 3 * sizeof(int), stream));
            SQ_COUNT(1);
            SQ_CUDA(slab_counts(a, d_cnt, h->num_sms, stream));
            int cnt[2];
            SQ_CUDA(cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, stream));
            SQ_CUDA(cudaStreamSynchronize(stream));
            const int amax = cnt[0] > 0 ? cnt[0] : 1, fmax = cnt[1] > 0 ? cnt[1] : 1;
            const size_t sm = slab_smem_bytes(h->nc[0], amax, fmax);
            if (sm <= (size_t)dev_smem) {
                long long grid = h->num_sms;
                if (grid > q1 - q0) grid = q1 - q0;
                h->kernel_used = 1;
                SQ_CUDA(cudaEventRecord(h->ev[0], stream));
                SQ_COUNT(1);
                SQ_CUDA(launch_slab(a, amax, fmax, (int)grid, sm, d_cnt + 2, stream));
                SQ_CUDA(cudaEventRecord(h->ev[1], stream));
                dim3 g2(kSumBlocks, K + 1);
                SQ_COUNT(1);
                k_msum_partial<T><<<g2, 256, 0, stream>>>(reinterpret_cast<const T *>(h->d_mu), h->N_d, K,
                                                          h->d_msum_part, q0, q1);
                SQ_CUDA(cudaGetLastError());
                return SQ_OK;
            }
        }
    }
    h->kernel_used = 0;
    const size_t smem_vec = recursion_smem_bytes<T>(h->natom, h->nc, 1);
    const size_t smem_glob = recursion_smem_bytes<T>(h->natom, h->nc, 0);
    // Vector placement: FP32 keeps both cube vectors in shared memory whenever they fit (512-thread
    // CTAs for large cubes); FP64 only when two CTAs still fit per SM, else per-CTA global scratch.
    const int nseg = ((h->nc[0] + 7) / 8) * h->nc[1] * h->nc[2];
    int block = 256;
    if (sizeof(T) == 4 && smem_vec <= (size_t)dev_smem) {
        a.vec_in_smem = 1;
        block = nseg >= 1024 ? 512 : 256;
    } else {
        a.vec_in_smem = (smem_vec * 2 + 2048 <= (size_t)dev_smem) ? 1 : 0;
    }
    const size_t smem = a.vec_in_smem ? smem_vec : smem_glob;
    if (smem > (size_t)dev_smem) return fail(SQ_ERR_UNSUPPORTED, "too many atoms for shared memory (%zu B)", smem);
    int per_sm = recursion_blocks_per_sm<T>(h->p, block, smem, a.vec_in_smem);
    if (per_sm < 1) return fail(SQ_ERR_UNSUPPORTED, "recursion kernel does not fit on an SM");
    long long grid = (long long)per_sm * h->num_sms;
    if (grid > q1 - q0) grid = q1 - q0;
    if (!a.vec_in_smem) {
        if ((s = ensure(&h->d_scratch, &h->scratch_cap, sizeof(T) * 2 * (size_t)h->nc3 * grid))) return s;
        a.scratch = reinterpret_cast<T *>(h->d_scratch);
    }
    SQ_CUDA(cudaEventRecord(h->ev[0], stream));
    SQ_COUNT(1);
    SQ_CUDA(launch_recursion<T>(a, h->p, (int)grid, block, smem, stream));
    SQ_CUDA(cudaEventRecord(h->ev[1], stream));
    if (cols) return SQ_OK;   // a column list: no range sums
    // moment sums
    dim3 g2(kSumBlocks, K + 1);
    SQ_COUNT(1);
    k_msum_partial<T><<<g2, 256, 0, stream>>>(reinterpret_cast<const T *>(h->d_mu), h->N_d, K, h->d_msum_part,
                                              q0, q1);
    SQ_CUDA(cudaGetLastError());
    return SQ_OK;
}

// Number of Chebyshev-Gauss nodes of the weight quadrature: M = 2^ceil(log2 max(4(K+1), 16 tau/kT)),
// or 0 when that exceeds 2^26.
static int fermi_nodes(int K, double tau, double kT)
{
    const double need = fmax(4.0 * (K + 1), 16.0 * tau / kT);
    int M = 1;
    while (M < need && M <= (1 << 26)) M <<= 1;
    return M > (1 << 26) ? 0 : M;
}

// Node arrays (lambda_j, D_j) from the stored moment sums, sized for (K, kT).
static sq_status nodes_at(sq_handle h, double kT, int *M_out, cudaStream_t stream)
{
    const int K = h->K;
    const int M = fermi_nodes(K, h->tau, kT);
    if (!M) return fail(SQ_ERR_UNSUPPORTED, "kT/tau too small for the weight quadrature");
    sq_status s;
    if ((s = ensure(&h->d_nodes, &h->nodes_cap, sizeof(double) * 5 * (size_t)M))) return s;
    if ((s = ensure(&h->d_coef, &h->coef_cap, sizeof(double) * 3 * (size_t)(K + 1)))) return s;
    SQ_COUNT(1);
    k_nodes<<<grid_for(M, 256, h->num_sms), 256, 0, stream>>>(h->d_msum, K, M, h->omega, h->tau, h->d_nodes,
                                                               h->d_nodes + M);
    SQ_CUDA(cudaGetLastError());
    *M_out = M;
    return SQ_OK;
}

// Chebyshev weights c_k, d_k, e_k of g, lam g and s(g) at the Fermi level lf (nodes already set).
static sq_status coeffs_at(sq_handle h, int M, double lf, double kT, cudaStream_t stream)
{
    const int K = h->K;
    double *lam = h->d_nodes, *f0 = h->d_nodes + 2 * M, *f1 = h->d_nodes + 3 * M, *f2 = h->d_nodes + 4 * M;
    SQ_COUNT(2);
    k_node_functions<<<grid_for(M, 256, h->num_sms), 256, 0, stream>>>(lam, M, lf, kT, f0, f1, f2);
    SQ_CUDA(cudaGetLastError());
    k_coeffs<<<dim3(K + 1, 3), 256, 0, stream>>>(f0, f1, f2, M, K, h->d_coef);
    SQ_CUDA(cudaGetLastError());
    h->M = M;
    return SQ_OK;
}

// Weights at a given Fermi level (the level itself solved elsewhere).
static sq_status weights_at(sq_handle h, double lf, double kT, cudaStream_t stream)
{
    int M = 0;
    sq_status s;
    if ((s = nodes_at(h, kT, &M, stream))) return s;
    return coeffs_at(h, M, lf, kT, stream);
}

// Fermi level, weights and (optionally) the density from the stored moment sums.
static sq_status fermi_and_density(sq_handle h, double kT, double N_e, double *d_rho, double *lambda_f,
                                   cudaStream_t stream)
{
    const int K = h->K;
    SQ_CUDA(cudaEventRecord(h->ev[3], stream));
    int M = 0;
    sq_status s;
    if ((s = nodes_at(h, kT, &M, stream))) return s;
    double *lam = h->d_nodes, *D = h->d_nodes + M;
    // bisection state lives in the small scratch (after the first 256 bytes)
    FermiState *st = reinterpret_cast<FermiState *>(reinterpret_cast<char *>(h->d_small) + 256);
    double *part = reinterpret_cast<double *>(reinterpret_cast<char *>(h->d_small) + 512);
    FermiState init;
    memset(&init, 0, sizeof(init));
    init.lo = h->lmin;
    init.hi = h->lmax_;
    SQ_CUDA(cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, stream));
    FermiState fin;
    for (int round = 0; round < 16; round++) {
        SQ_COUNT(16);
        for (int i = 0; i < 16; i++) k_fermi_step<<<kFermiBlocks, 256, 0, stream>>>(lam, D, M, kT, N_e, st, part);
        SQ_CUDA(cudaGetLastError());
        SQ_CUDA(cudaMemcpyAsync(&fin, st, sizeof(fin), cudaMemcpyDeviceToHost, stream));
        SQ_CUDA(cudaStreamSynchronize(stream));
        if (fin.phase >= 3) break;
    }
    if (fin.phase == 4)
        return fail(SQ_ERR_NO_BRACKET, "N(lambda_min) = %.6g, N(lambda_max) = %.6g, N_e = %.6g", fin.N_lo, fin.N_hi, N_e);
    if (fin.phase != 3) return fail(SQ_ERR_TIMEOUT, "bisection did not finish");
    const double lf = fin.x;
    if (!std::isfinite(lf)) return fail(SQ_ERR_NOT_FINITE, "Fermi level is not finite");
    if ((s = coeffs_at(h, M, lf, kT, stream))) return s;
    if (d_rho) {
        SQ_COUNT(1);
        if (h->precision == SQ_FP64)
            k_density<double><<<grid_for(h->N_d, 256, h->num_sms), 256, 0, stream>>>(
                reinterpret_cast<const double *>(h->d_mu), h->N_d, K, h->d_coef, 1.0 / h->dV, d_rho, 0LL, h->N_d);
        else
            k_density<float><<<grid_for(h->N_d, 256, h->num_sms), 256, 0, stream>>>(
                reinterpret_cast<const float *>(h->d_mu), h->N_d, K, h->d_coef, 1.0 / h->dV, d_rho, 0LL, h->N_d);
        SQ_CUDA(cudaGetLastError());
    }
    SQ_CUDA(cudaEventRecord(h->ev[4], stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    h->kT = kT;
    h->N_e = N_e;
    h->lam_f = lf;
    if (lambda_f) *lambda_f = lf;
    return SQ_OK;
}

// ------------------------------------------------------------------------------------------------
// Gauss (Lanczos) quadrature path: Lanczos coefficients of every column, the Gauss rule of each
// column's Jacobi matrix, the Fermi level over all nodes (Eq. Ne), rho, U and S.

template <typename T>
static sq_status run_lanczos(sq_handle h, int K, cudaStream_t stream)
{
    sq_status s;
    const size_t pad = (size_t)h->pn[0] * h->pn[1] * h->pn[2];
    T **dpad = nullptr;
    if constexpr (sizeof(T) == 8) dpad = reinterpret_cast<T **>(&h->d_dpad64);
    else dpad = reinterpret_cast<T **>(&h->d_dpad32);
    if (!*dpad) {
        size_t cap = 0;
        if ((s = ensure(dpad, &cap, sizeof(T) * pad))) return s;
    }
    SQ_COUNT(1);
    k_dpad<T><<<grid_for((long long)pad, 256, h->num_sms), 256, 0, stream>>>(
        h->d_veff, h->n[0], h->n[1], h->n[2], h->m[0], h->m[1], h->m[2], h->kdiag, h->omega, h->tau, *dpad);
    SQ_CUDA(cudaGetLastError());
    RecursionArgs<T> a;
    fill_args<T>(h, K, 0, a);
    a.dpad = *dpad;
    a.ab = h->d_ab;
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    const size_t smem_vec = recursion_smem_bytes<T>(h->natom, h->nc, 1);
    const size_t smem_glob = recursion_smem_bytes<T>(h->natom, h->nc, 0);
    const int nseg = ((h->nc[0] + 7) / 8) * h->nc[1] * h->nc[2];
    int block = 256;
    if (sizeof(T) == 4 && smem_vec <= (size_t)dev_smem) {
        a.vec_in_smem = 1;
        block = nseg >= 1024 ? 512 : 256;
    } else {
        a.vec_in_smem = (smem_vec * 2 + 2048 <= (size_t)dev_smem) ? 1 : 0;
    }
    const size_t smem = a.vec_in_smem ? smem_vec : smem_glob;
    if (smem > (size_t)dev_smem) return fail(SQ_ERR_UNSUPPORTED, "too many atoms for shared memory (%zu B)", smem);
    const int per_sm = lanczos_blocks_per_sm<T>(h->p, block, smem, a.vec_in_smem);
    if (per_sm < 1) return fail(SQ_ERR_UNSUPPORTED, "Lanczos kernel does not fit on an SM");
    long long grid = (long long)per_sm * h->num_sms;
    if (grid > h->N_d) grid = h->N_d;
    if (!a.vec_in_smem) {
        if ((s = ensure(&h->d_scratch, &h->scratch_cap, sizeof(T) * 2 * (size_t)h->nc3 * grid))) return s;
        a.scratch = reinterpret_cast<T *>(h->d_scratch);
    }
    h->kernel_used = 3;
    SQ_CUDA(cudaEventRecord(h->ev[0], stream));
    SQ_COUNT(1);
    SQ_CUDA(launch_lanczos<T>(a, h->p, (int)grid, block, smem, stream));
    SQ_CUDA(cudaEventRecord(h->ev[1], stream));
    return SQ_OK;
}

// Fermi level over the Gauss nodes (same bisection state machine as the Chebyshev path, with the
// node energies and weights of all columns in place of the Chebyshev-Gauss nodes), then rho, U, S.
static sq_status gauss_fermi_and_observables(sq_handle h, double kT, double N_e, double *d_rho, double *lambda_f,
                                             cudaStream_t stream)
{
    const int K = h->K;
    const long long nK = (long long)K * h->N_d;
    const double *nodes = h->d_gnode, *weights = h->d_gnode + nK;
    SQ_CUDA(cudaEventRecord(h->ev[3], stream));
    FermiState *st = reinterpret_cast<FermiState *>(reinterpret_cast<char *>(h->d_small) + 256);
    double *part = reinterpret_cast<double *>(reinterpret_cast<char *>(h->d_small) + 512);
    FermiState init;
    memset(&init, 0, sizeof(init));
    init.lo = h->lmin;
    init.hi = h->lmax_;
    SQ_CUDA(cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, stream));
    FermiState fin;
    for (int round = 0; round < 16; round++) {
        SQ_COUNT(16);
        for (int i = 0; i < 16; i++)
            k_fermi_step<<<kFermiBlocks, 256, 0, stream>>>(nodes, weights, (int)nK, kT, N_e, st, part);
        SQ_CUDA(cudaGetLastError());
        SQ_CUDA(cudaMemcpyAsync(&fin, st, sizeof(fin), cudaMemcpyDeviceToHost, stream));
        SQ_CUDA(cudaStreamSynchronize(stream));
        if (fin.phase >= 3) break;
    }
    if (fin.phase == 4)
        return fail(SQ_ERR_NO_BRACKET, "N(lambda_min) = %.6g, N(lambda_max) = %.6g, N_e = %.6g", fin.N_lo, fin.N_hi, N_e);
    if (fin.phase != 3) return fail(SQ_ERR_TIMEOUT, "bisection did not finish");
    const double lf = fin.x;
    if (!std::isfinite(lf)) return fail(SQ_ERR_NOT_FINITE, "Fermi level is not finite");
    if (d_rho) {
        SQ_COUNT(1);
        k_gauss_density<<<grid_for(h->N_d, 256, h->num_sms), 256, 0, stream>>>(nodes, weights, h->N_d, K, lf, kT,
                                                                             1.0 / h->dV, d_rho);
        SQ_CUDA(cudaGetLastError());
    }
    double *epart = h->d_msum_part;   // 2 x kEnergyBlocks doubles (sized by sq_density)
    double *eout = reinterpret_cast<double *>(h->d_small) + 4;
    SQ_COUNT(2);
    k_gauss_energy_partial<<<kSumBlocks, 256, 0, stream>>>(nodes, weights, nK, lf, kT, epart);
    k_gauss_energy_final<<<1, 32, 0, stream>>>(epart, kSumBlocks, eout);
    SQ_CUDA(cudaGetLastError());
    double us[2];
    SQ_CUDA(cudaMemcpyAsync(us, eout, sizeof(us), cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaEventRecord(h->ev[4], stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    h->gU = us[0];
    h->gS = us[1];
    h->kT = kT;
    h->N_e = N_e;
    h->lam_f = lf;
    if (lambda_f) *lambda_f = lf;
    return SQ_OK;
}

static sq_status gauss_density(sq_handle h, int K, double kT, double N_e, int precision, double *d_rho,
                               double *lambda_f, cudaStream_t stream)
{
    h->have_density = 0;
    h->have_moments = 0;
    sq_status s;
    const size_t nK = (size_t)K * h->N_d;
    if ((s = ensure(&h->d_ab, &h->ab_cap, sizeof(double) * 2 * nK))) return s;
    if ((s = ensure(&h->d_gnode, &h->gnode_cap, sizeof(double) * 2 * nK))) return s;
    if ((s = ensure(&h->d_msum_part, &h->part_cap, sizeof(double) * (size_t)(K + 1) * kSumBlocks))) return s;
    h->precision = precision;
    h->K = K;
    s = precision == SQ_FP64 ? run_lanczos<double>(h, K, stream) : run_lanczos<float>(h, K, stream);
    if (s) return s;
    int *d_bad = reinterpret_cast<int *>(h->d_small);
    SQ_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), stream));
    SQ_COUNT(1);
    SQ_CUDA(launch_gauss_rule(h->d_ab, h->N_d, 0, h->N_d, K, h->omega, h->tau, h->d_gnode, h->d_gnode + nK, d_bad,
                              h->num_sms, stream));
    SQ_CUDA(cudaEventRecord(h->ev[2], stream));
    int bad = 0;
    SQ_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    if (bad) return fail(SQ_ERR_NOT_FINITE, "a Jacobi eigensolve did not converge");
    SQ_CUDA(cudaEventElapsedTime(&h->t_rec, h->ev[0], h->ev[1]));
    SQ_CUDA(cudaEventElapsedTime(&h->t_msum, h->ev[1], h->ev[2]));
    h->gauss = 1;
    h->have_force = 0;
    h->q0 = 0;
    h->q1 = h->N_d;
    if ((s = gauss_fermi_and_observables(h, kT, N_e, d_rho, lambda_f, stream))) return s;
    SQ_CUDA(cudaEventElapsedTime(&h->t_fermi, h->ev[3], h->ev[4]));
    h->have_density = 1;
    return SQ_OK;
}

// Recursion over columns [q0, q1), moments into the handle's [K+1][N_d] buffer, and the moment sums of
// those columns into h->d_msum (FP64).  Leaves the handle without a density (have_density = 0).
static sq_status moments_stage(sq_handle h, int K, int precision, int want_force, long long q0, long long q1,
                               cudaStream_t stream)
{
    h->have_density = 0;
    h->have_moments = 0;
    sq_status s;
    const size_t esz = precision == SQ_FP64 ? 8 : 4;
    if ((s = ensure(&h->d_mu, &h->mu_bytes, esz * (size_t)(K + 1) * h->N_d))) return s;
    if ((s = ensure(&h->d_msum, &h->msum_cap, sizeof(double) * (size_t)(K + 1)))) return s;
    if ((s = ensure(&h->d_msum_part, &h->part_cap, sizeof(double) * (size_t)(K + 1) * kSumBlocks))) return s;
    const size_t abytes = sizeof(double) * (size_t)(K + 1) * h->natom * h->nproj * 3;
    if (want_force && (s = ensure(&h->d_A, &h->A_cap, abytes))) return s;
    h->precision = precision;
    h->K = K;
    int bad = 0, slab_err = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        if (want_force) SQ_CUDA(cudaMemsetAsync(h->d_A, 0, abytes, stream));
        s = precision == SQ_FP64 ? run_recursion<double>(h, K, want_force, q0, q1, stream)
                                 : run_recursion<float>(h, K, want_force, q0, q1, stream);
        if (s) return s;
        int *d_bad = reinterpret_cast<int *>(h->d_small);
        SQ_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), stream));
        SQ_COUNT(1);
        k_msum_final<<<1, 256, 0, stream>>>(h->d_msum_part, kSumBlocks, K, h->d_msum, d_bad);
        SQ_CUDA(cudaGetLastError());
        SQ_CUDA(cudaEventRecord(h->ev[2], stream));
        bad = 0;
        slab_err = 0;
        SQ_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, stream));
        if (h->kernel_used != 0)
            SQ_CUDA(cudaMemcpyAsync(&slab_err, reinterpret_cast<int *>(h->d_small) + 42, sizeof(int),
                                    cudaMemcpyDeviceToHost, stream));
        SQ_CUDA(cudaStreamSynchronize(stream));
        // a warp's atom list longer than the tensor-core projector path takes: redo the launch with the
        // CUDA-core form of the projector term
        if (slab_err == 3 && h->kernel_used == 2 && attempt == 0) {
            h->kb_fma = 1;
            continue;
        }
        break;
    }
    if (slab_err) return fail(SQ_ERR_UNSUPPORTED, "a column exceeded the FP32 kernel's atom capacity (%d)", slab_err);
    if (bad) return fail(SQ_ERR_NOT_FINITE, "moment sums are not finite");
    SQ_CUDA(cudaEventElapsedTime(&h->t_rec, h->ev[0], h->ev[1]));
    SQ_CUDA(cudaEventElapsedTime(&h->t_msum, h->ev[1], h->ev[2]));
    h->have_force = want_force;
    h->q0 = q0;
    h->q1 = q1;
    h->have_moments = 1;
    return SQ_OK;
}

static sq_status check_density_args(sq_handle h, int K, double kT, double N_e, int precision, int flags)
{
    if (K < 1 || K > 4096) return fail(SQ_ERR_ARG, "K = %d", K);
    if (!(kT > 0) || !std::isfinite(kT)) return fail(SQ_ERR_ARG, "kT = %g", kT);
    if (!(N_e > 0) || !(N_e < 2.0 * h->N_d)) return fail(SQ_ERR_ARG, "N_e = %g", N_e);
    if (precision != SQ_FP64 && precision != SQ_FP32) return fail(SQ_ERR_ARG, "precision %d", precision);
    if (flags & ~(SQ_WANT_FORCE | SQ_GAUSS | SQ_KB_FMA)) return fail(SQ_ERR_ARG, "flags %d", flags);
    if ((flags & SQ_GAUSS) && (flags & SQ_WANT_FORCE))
        return fail(SQ_ERR_ARG, "SQ_GAUSS gives rho, U and S; the force moments need the Chebyshev path");
    if ((flags & SQ_GAUSS) && K > kGaussMaxK) return fail(SQ_ERR_ARG, "K = %d above the Gauss path's %d", K, kGaussMaxK);
    return SQ_OK;
}

extern "C" sq_status sq_density(sq_handle h, int K, double kT, double N_e, int precision, int flags, double *d_rho,
                                double *lambda_f, void *stream_)
{
    g_last_error[0] = 0;
    if (!h || !d_rho || !lambda_f) return fail(SQ_ERR_ARG, "null argument");
    sq_status s;
    if ((s = check_density_args(h, K, kT, N_e, precision, flags))) return s;
    cudaStream_t stream = (cudaStream_t)stream_;
    if (flags & SQ_GAUSS) return gauss_density(h, K, kT, N_e, precision, d_rho, lambda_f, stream);
    h->gauss = 0;
    h->kb_fma = (flags & SQ_KB_FMA) ? 1 : 0;
    const int want_force = (flags & SQ_WANT_FORCE) && h->natom > 0;
    if ((s = moments_stage(h, K, precision, want_force, 0, h->N_d, stream))) return s;
    if ((s = fermi_and_density(h, kT, N_e, d_rho, lambda_f, stream))) return s;
    SQ_CUDA(cudaEventElapsedTime(&h->t_fermi, h->ev[3], h->ev[4]));
    h->have_density = 1;
    return SQ_OK;
}

extern "C" sq_status sq_fermi_resolve(sq_handle h, double kT, double N_e, double *d_rho, double *lambda_f,
                                      void *stream_)
{
    g_last_error[0] = 0;
    if (!h || !lambda_f) return fail(SQ_ERR_ARG, "null argument");
    if (!h->have_density || h->q0 != 0 || h->q1 != h->N_d)
        return fail(SQ_ERR_STATE, "sq_fermi_resolve needs a whole-grid sq_density first");
    if (!(kT > 0) || !(N_e > 0) || !(N_e < 2.0 * h->N_d)) return fail(SQ_ERR_ARG, "kT = %g, N_e = %g", kT, N_e);
    if (h->gauss) return gauss_fermi_and_observables(h, kT, N_e, d_rho, lambda_f, (cudaStream_t)stream_);
    return fermi_and_density(h, kT, N_e, d_rho, lambda_f, (cudaStream_t)stream_);
}

// ------------------------------------------------------------------------------------------------
// Column-range form of the path (one shard of the grid), for callers that split the columns over
// processes or GPUs and sum the moments themselves (Eq. Ne needs one global sum).

extern "C" sq_status sq_moments_range(sq_handle h, int K, int precision, int flags, long long q_begin, long long q_end,
                                      double *msum, double *A, void *stream_)
{
    g_last_error[0] = 0;
    if (!h || !msum) return fail(SQ_ERR_ARG, "null argument");
    if (K < 1 || K > 4096) return fail(SQ_ERR_ARG, "K = %d", K);
    if (precision != SQ_FP64 && precision != SQ_FP32) return fail(SQ_ERR_ARG, "precision %d", precision);
    if (flags & ~(SQ_WANT_FORCE | SQ_KB_FMA)) return fail(SQ_ERR_ARG, "flags %d", flags);
    if (q_begin < 0 || q_end > h->N_d || q_begin >= q_end)
        return fail(SQ_ERR_ARG, "column range [%lld, %lld) of %lld", q_begin, q_end, h->N_d);
    const int want_force = (flags & SQ_WANT_FORCE) && h->natom > 0;
    if (want_force && !A) return fail(SQ_ERR_ARG, "SQ_WANT_FORCE needs the force-moment output A");
    cudaStream_t stream = (cudaStream_t)stream_;
    sq_status s;
    h->gauss = 0;
    h->kb_fma = (flags & SQ_KB_FMA) ? 1 : 0;
    if ((s = moments_stage(h, K, precision, want_force, q_begin, q_end, stream))) return s;
    SQ_CUDA(cudaMemcpyAsync(msum, h->d_msum, sizeof(double) * (K + 1), cudaMemcpyDeviceToHost, stream));
    if (want_force)
        SQ_CUDA(cudaMemcpyAsync(A, h->d_A, sizeof(double) * (size_t)(K + 1) * h->natom * h->nproj * 3,
                                cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    return SQ_OK;
}

template <typename T>
__global__ void k_gather_mu(const T *mu, long long N_d, int K, const long long *cols, long long ncols, T *out)
{
    const long long tot = (long long)(K + 1) * ncols;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const long long k = t / ncols, i = t % ncols;
        out[t] = mu[(size_t)k * N_d + cols[i]];
    }
}

extern "C" sq_status sq_moments_cols(sq_handle h, int K, int precision, const long long *d_cols, long long ncols,
                                     void *d_mu_out, void *stream_)
{
    g_last_error[0] = 0;
    if (!h || !d_cols || !d_mu_out) return fail(SQ_ERR_ARG, "null argument");
    if (K < 1 || K > 4096) return fail(SQ_ERR_ARG, "K = %d", K);
    if (precision != SQ_FP64 && precision != SQ_FP32) return fail(SQ_ERR_ARG, "precision %d", precision);
    if (ncols < 1 || ncols > h->N_d) return fail(SQ_ERR_ARG, "ncols = %lld", ncols);
    cudaStream_t stream = (cudaStream_t)stream_;
    h->have_density = 0;
    h->have_moments = 0;
    h->gauss = 0;
    sq_status s;
    const size_t esz = precision == SQ_FP64 ? 8 : 4;
    if ((s = ensure(&h->d_mu, &h->mu_bytes, esz * (size_t)(K + 1) * h->N_d))) return s;
    h->precision = precision;
    h->K = K;
    // column indices are checked on the device against the grid before any use
    int *d_bad = reinterpret_cast<int *>(h->d_small);
    SQ_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), stream));
    SQ_COUNT(1);
    k_check_cols<<<grid_for(ncols, 256, h->num_sms), 256, 0, stream>>>(d_cols, ncols, h->N_d, d_bad);
    SQ_CUDA(cudaGetLastError());
    int bad = 0;
    SQ_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    if (bad) return fail(SQ_ERR_ARG, "a column index is outside [0, N_d)");
    s = precision == SQ_FP64 ? run_recursion<double>(h, K, 0, 0, ncols, stream, d_cols)
                             : run_recursion<float>(h, K, 0, 0, ncols, stream, d_cols);
    if (s) return s;
    SQ_COUNT(1);
    if (precision == SQ_FP64)
        k_gather_mu<double><<<grid_for((K + 1) * ncols, 256, h->num_sms), 256, 0, stream>>>(
            reinterpret_cast<const double *>(h->d_mu), h->N_d, K, d_cols, ncols, reinterpret_cast<double *>(d_mu_out));
    else
        k_gather_mu<float><<<grid_for((K + 1) * ncols, 256, h->num_sms), 256, 0, stream>>>(
            reinterpret_cast<const float *>(h->d_mu), h->N_d, K, d_cols, ncols, reinterpret_cast<float *>(d_mu_out));
    SQ_CUDA(cudaGetLastError());
    SQ_CUDA(cudaStreamSynchronize(stream));
    return SQ_OK;
}

extern "C" sq_status sq_observables(sq_handle h, double lambda_f, double kT, double N_e, const double *msum,
                                    const double *A, double *d_rho, void *stream_)
{
    g_last_error[0] = 0;
    if (!h || !msum) return fail(SQ_ERR_ARG, "null argument");
    if (!h->have_moments) return fail(SQ_ERR_STATE, "sq_observables before sq_moments_range");
    if (!(kT > 0) || !std::isfinite(kT) || !std::isfinite(lambda_f) || !(N_e > 0))
        return fail(SQ_ERR_ARG, "lambda_f = %g, kT = %g, N_e = %g", lambda_f, kT, N_e);
    for (int k = 0; k <= h->K; k++)
        if (!std::isfinite(msum[k])) return fail(SQ_ERR_NOT_FINITE, "moment sum %d", k);
    cudaStream_t stream = (cudaStream_t)stream_;
    const int K = h->K;
    h->have_density = 0;
    SQ_CUDA(cudaMemcpyAsync(h->d_msum, msum, sizeof(double) * (K + 1), cudaMemcpyHostToDevice, stream));
    const int force = h->have_force && A;
    if (force)
        SQ_CUDA(cudaMemcpyAsync(h->d_A, A, sizeof(double) * (size_t)(K + 1) * h->natom * h->nproj * 3,
                                cudaMemcpyHostToDevice, stream));
    sq_status s;
    if ((s = weights_at(h, lambda_f, kT, stream))) return s;
    if (d_rho) {
        const long long n = h->q1 - h->q0;
        SQ_COUNT(1);
        if (h->precision == SQ_FP64)
            k_density<double><<<grid_for(n, 256, h->num_sms), 256, 0, stream>>>(
                reinterpret_cast<const double *>(h->d_mu), h->N_d, K, h->d_coef, 1.0 / h->dV, d_rho, h->q0, h->q1);
        else
            k_density<float><<<grid_for(n, 256, h->num_sms), 256, 0, stream>>>(
                reinterpret_cast<const float *>(h->d_mu), h->N_d, K, h->d_coef, 1.0 / h->dV, d_rho, h->q0, h->q1);
        SQ_CUDA(cudaGetLastError());
    }
    SQ_CUDA(cudaStreamSynchronize(stream));
    h->kT = kT;
    h->N_e = N_e;
    h->lam_f = lambda_f;
    h->have_force = force;
    h->have_density = 1;
    return SQ_OK;
}

// ------------------------------------------------------------------------------------------------
// Pure host form of the Fermi-level solve (Eq. Ne) and of the Chebyshev weights (Eq.
// ChebyshevWeights), in FP64, for moment sums that were reduced outside the library.  Same node rule,
// node functions and bisection rule as the device path.

static double host_cos_k_theta(int k, int j, int M)
{
    // cos(k pi (2j+1)/(2M)) with exact argument reduction modulo 2 pi
    const long long r = ((long long)k * (2LL * j + 1)) % (4LL * M);
    return cos(M_PI * (double)r / (2.0 * M));
}

static double host_fermi_fn(double lam, double lam_f, double kT) { return 0.5 * (1.0 - tanh((lam - lam_f) / (2.0 * kT))); }

static void host_node_lambdas(int M, double omega, double tau, std::vector<double> &lam)
{
    lam.resize(M);
    for (int j = 0; j < M; j++) lam[j] = tau * cos(M_PI * (j + 0.5) / M) + omega;
}

static bool host_scalar_ok(double x) { return std::isfinite(x); }

extern "C" sq_status sq_fermi_level(const double *msum, int K, double omega, double tau, double lambda_min,
                                    double lambda_max, double kT, double N_e, double *lambda_f)
{
    g_last_error[0] = 0;
    if (!msum || !lambda_f) return fail(SQ_ERR_ARG, "null argument");
    if (K < 1 || K > 4096) return fail(SQ_ERR_ARG, "K = %d", K);
    if (!(tau > 0) || !host_scalar_ok(omega) || !host_scalar_ok(tau)) return fail(SQ_ERR_ARG, "omega = %g, tau = %g", omega, tau);
    if (!(lambda_max > lambda_min) || !host_scalar_ok(lambda_min) || !host_scalar_ok(lambda_max))
        return fail(SQ_ERR_ARG, "bracket [%g, %g]", lambda_min, lambda_max);
    if (!(kT > 0) || !host_scalar_ok(kT) || !(N_e > 0) || !host_scalar_ok(N_e))
        return fail(SQ_ERR_ARG, "kT = %g, N_e = %g", kT, N_e);
    for (int k = 0; k <= K; k++)
        if (!host_scalar_ok(msum[k])) return fail(SQ_ERR_NOT_FINITE, "moment sum %d", k);
    const int M = fermi_nodes(K, tau, kT);
    if (!M) return fail(SQ_ERR_UNSUPPORTED, "kT/tau too small for the weight quadrature");
    std::vector<double> lam, D(M);
    host_node_lambdas(M, omega, tau, lam);
    for (int j = 0; j < M; j++) {
        double s = msum[0];
        for (int k = 1; k <= K; k++) s += 2.0 * msum[k] * host_cos_k_theta(k, j, M);
        D[j] = s / M;
    }
    auto count = [&](double x) {
        double N = 0.0;
        for (int j = 0; j < M; j++) N += host_fermi_fn(lam[j], x, kT) * D[j];
        return 2.0 * N;
    };
    double lo = lambda_min, hi = lambda_max;
    const double N_lo = count(lo), N_hi = count(hi);
    if (N_lo > N_e || N_hi < N_e)
        return fail(SQ_ERR_NO_BRACKET, "N(lambda_min) = %.6g, N(lambda_max) = %.6g, N_e = %.6g", N_lo, N_hi, N_e);
    double x = lo + 0.5 * (hi - lo);
    for (int iter = 1; iter <= 200; iter++) {
        if (count(x) < N_e) lo = x;
        else hi = x;
        x = lo + 0.5 * (hi - lo);
        if (x <= lo || x >= hi) break;
    }
    if (!host_scalar_ok(x)) return fail(SQ_ERR_NOT_FINITE, "Fermi level is not finite");
    *lambda_f = x;
    return SQ_OK;
}

extern "C" sq_status sq_fermi_weights(double lambda_f, int K, double omega, double tau, double kT, double *c,
                                      double *d, double *e)
{
    g_last_error[0] = 0;
    if (K < 1 || K > 4096) return fail(SQ_ERR_ARG, "K = %d", K);
    if (!(tau > 0) || !host_scalar_ok(omega) || !host_scalar_ok(tau) || !(kT > 0) || !host_scalar_ok(kT) ||
        !host_scalar_ok(lambda_f))
        return fail(SQ_ERR_ARG, "lambda_f = %g, omega = %g, tau = %g, kT = %g", lambda_f, omega, tau, kT);
    const int M = fermi_nodes(K, tau, kT);
    if (!M) return fail(SQ_ERR_UNSUPPORTED, "kT/tau too small for the weight quadrature");
    std::vector<double> lam, f0(M), f1(M), f2(M);
    host_node_lambdas(M, omega, tau, lam);
    for (int j = 0; j < M; j++) {
        const double l = lam[j];
        const double g = host_fermi_fn(l, lambda_f, kT);
        const double y = fabs((l - lambda_f) / kT);
        f0[j] = g;
        f1[j] = l * g;
        f2[j] = -(log1p(exp(-y)) + y * host_fermi_fn(y, 0.0, 1.0));
    }
    for (int k = 0; k <= K; k++) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int j = 0; j < M; j++) {
            const double ck = host_cos_k_theta(k, j, M);
            s0 += f0[j] * ck;
            s1 += f1[j] * ck;
            s2 += f2[j] * ck;
        }
        const double w = (k == 0 ? 1.0 : 2.0) / M;
        if (c) c[k] = w * s0;
        if (d) d[k] = w * s1;
        if (e) e[k] = w * s2;
    }
    return SQ_OK;
}

extern "C" sq_status sq_gauss_rule(const double *a, const double *b, int K, double omega, double tau, double *nodes,
                                   double *weights)
{
    g_last_error[0] = 0;
    if (!a || !b || !nodes || !weights) return fail(SQ_ERR_ARG, "null argument");
    if (K < 1 || K > kGaussMaxK) return fail(SQ_ERR_ARG, "K = %d", K);
    if (!(tau > 0) || !std::isfinite(omega) || !std::isfinite(tau)) return fail(SQ_ERR_ARG, "omega = %g, tau = %g", omega, tau);
    double d[kGaussMaxK], e[kGaussMaxK], z[kGaussMaxK];
    for (int k = 0; k < K; k++) {
        if (!std::isfinite(a[k]) || !std::isfinite(b[k])) return fail(SQ_ERR_NOT_FINITE, "coefficient %d", k);
        d[k] = a[k];
        e[k] = b[k];
    }
    const int n = gauss_rule_inplace(d, e, z, K);
    if (n < 0) return fail(SQ_ERR_NOT_FINITE, "the Jacobi eigensolve did not converge");
    for (int k = 0; k < K; k++) {
        nodes[k] = k < n ? tau * d[k] + omega : omega;
        weights[k] = k < n ? z[k] * z[k] : 0.0;
    }
    return SQ_OK;
}

extern "C" sq_status sq_energy(sq_handle h, double *U, double *S, double *F, void *stream_)
{
    g_last_error[0] = 0;
    if (!h) return fail(SQ_ERR_ARG, "null handle");
    if (!h->have_density) return fail(SQ_ERR_STATE, "sq_energy before sq_density");
    if (h->gauss) {
        if (U) *U = h->gU;
        if (S) *S = h->gS;
        if (F) *F = h->gU - h->kT * h->gS;
        return SQ_OK;
    }
    cudaStream_t stream = (cudaStream_t)stream_;
    double *d_out = reinterpret_cast<double *>(h->d_small) + 4;
    SQ_COUNT(1);
    k_energy<<<1, 32, 0, stream>>>(h->d_msum, h->d_coef, h->K, d_out);
    SQ_CUDA(cudaGetLastError());
    double out[2];
    SQ_CUDA(cudaMemcpyAsync(out, d_out, sizeof(out), cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    if (U) *U = out[0];
    if (S) *S = out[1];
    if (F) *F = out[0] - h->kT * out[1];
    return SQ_OK;
}

extern "C" sq_status sq_nonlocal_force(sq_handle h, double *d_force, void *stream_)
{
    g_last_error[0] = 0;
    if (!h || (!d_force && h->natom > 0)) return fail(SQ_ERR_ARG, "null argument");
    if (!h->have_density) return fail(SQ_ERR_STATE, "sq_nonlocal_force before sq_density");
    if (h->natom == 0) return SQ_OK;
    if (!h->have_force) return fail(SQ_ERR_STATE, "sq_density was called without SQ_WANT_FORCE");
    cudaStream_t stream = (cudaStream_t)stream_;
    SQ_COUNT(1);
    k_force<<<grid_for(3LL * h->natom, 128, h->num_sms), 128, 0, stream>>>(
        h->d_A, h->d_coef, h->K, h->natom, h->nproj, h->cl[0], h->cl[1], h->dV, d_force);
    SQ_CUDA(cudaGetLastError());
    return SQ_OK;
}

extern "C" sq_status sq_get_spectral_bounds(sq_handle h, double *lambda_min, double *lambda_max)
{
    if (!h) return fail(SQ_ERR_ARG, "null handle");
    if (lambda_min) *lambda_min = h->lmin;
    if (lambda_max) *lambda_max = h->lmax_;
    return SQ_OK;
}

extern "C" sq_status sq_get_moments(sq_handle h, int *K, int *precision, const void **d_mu, const double **d_msum)
{
    if (!h) return fail(SQ_ERR_ARG, "null handle");
    if (!h->have_density || h->gauss) return fail(SQ_ERR_STATE, "no Chebyshev moments yet");
    if (K) *K = h->K;
    if (precision) *precision = h->precision;
    if (d_mu) *d_mu = h->d_mu;
    if (d_msum) *d_msum = h->d_msum;
    return SQ_OK;
}

extern "C" sq_status sq_copy_moments(sq_handle h, void *d_mu, double *d_msum, void *stream_)
{
    if (!h) return fail(SQ_ERR_ARG, "null handle");
    if (!h->have_density || h->gauss) return fail(SQ_ERR_STATE, "no Chebyshev moments yet");
    cudaStream_t stream = (cudaStream_t)stream_;
    const size_t esz = h->precision == SQ_FP64 ? 8 : 4;
    if (d_mu) SQ_CUDA(cudaMemcpyAsync(d_mu, h->d_mu, esz * (size_t)(h->K + 1) * h->N_d, cudaMemcpyDeviceToDevice, stream));
    if (d_msum) SQ_CUDA(cudaMemcpyAsync(d_msum, h->d_msum, sizeof(double) * (h->K + 1), cudaMemcpyDeviceToDevice, stream));
    return SQ_OK;
}

extern "C" sq_status sq_get_timing(sq_handle h, double *recursion_ms, double *msum_ms, double *fermi_ms)
{
    if (!h) return fail(SQ_ERR_ARG, "null handle");
    if (!h->have_density) return fail(SQ_ERR_STATE, "no sq_density yet");
    if (recursion_ms) *recursion_ms = h->t_rec;
    if (msum_ms) *msum_ms = h->t_msum;
    if (fermi_ms) *fermi_ms = h->t_fermi;
    return SQ_OK;
}

extern "C" const char *sq_kernel_name(sq_handle h)
{
    if (!h || !h->have_density) return "";
    if (h->kernel_used == 1) return h->nc[0] == 21 ? "slab_kernel<21,6>" : "slab_kernel<25,6>";
    if (h->kernel_used == 2) return h->nc[0] == 25 ? "cluster_kernel<25,6,mma>" : "cluster_kernel<29,6,mma>";
    if (h->kernel_used == 4) return h->nc[0] == 25 ? "cluster_kernel<25,6,fma>" : "cluster_kernel<29,6,fma>";
    if (h->kernel_used == 3) return h->precision == SQ_FP64 ? "lanczos_kernel<double>" : "lanczos_kernel<float>";
    return h->precision == SQ_FP64 ? "recursion_kernel<double>" : "recursion_kernel<float>";
}

extern "C" sq_status sq_get_cube(sq_handle h, int m[3])
{
    if (!h || !m) return fail(SQ_ERR_ARG, "null argument");
    for (int a = 0; a < 3; a++) m[a] = h->m[a];
    return SQ_OK;
}

// ------------------------------------------------------------------------------------------------
// Allocation-free moments.
//
// Some callers cannot let the library allocate device memory once their steady state has begun:
// applications that give the library a fixed device-memory budget up front, latency-critical loops
// where cudaMalloc/cudaFree would synchronise the device, or code that must not grow the memory
// footprint of a GPU it shares.  sq_moments_noalloc serves them: it runs the same per-column
// recursion kernel as sq_density, but keeps that kernel's working vectors (and the padded Hhat
// diagonal) in the fixed-size device array below instead of handle-owned allocations.
//
// The array is a file-scope __device__ object, so every GPU that loads this library holds it until
// the process exits.  Host code cannot use the symbol itself as a device address; the address is
// looked up with cudaGetSymbolAddress once per device (with that device current) and cached.

static constexpr size_t kStaticScratchBytes = 32u << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static constexpr int kMaxDevices = 64;
static void *g_static_scratch_ptr[kMaxDevices] = {nullptr};

static sq_status static_scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(SQ_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    if (!g_static_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(SQ_ERR_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        g_static_scratch_ptr[dev] = p;
    }
    *out = g_static_scratch_ptr[dev];
    return SQ_OK;
}

template <typename T>
static sq_status moments_noalloc(sq_handle h, int K, void *d_mu, cudaStream_t stream)
{
    void *base = nullptr;
    sq_status s = static_scratch_address(h->dev, &base);
    if (s) return s;
    const size_t pad = (size_t)h->pn[0] * h->pn[1] * h->pn[2];
    const size_t dpad_bytes = (sizeof(T) * pad + 255) & ~size_t(255);
    const size_t per_cta = sizeof(T) * 2 * (size_t)h->nc3;
    if (dpad_bytes + per_cta > kStaticScratchBytes)
        return fail(SQ_ERR_UNSUPPORTED,
                    "static scratch of %zu bytes cannot hold the padded diagonal (%zu B) and one cube's two "
                    "vectors (%zu B)", kStaticScratchBytes, dpad_bytes, per_cta);
    T *dpad = reinterpret_cast<T *>(base);
    T *vecs = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(base) + dpad_bytes);
    // every byte the kernels read is written first in this call: the diagonal here, and each
    // column's vectors at the start of that column inside the recursion kernel
    SQ_COUNT(1);
    k_dpad<T><<<grid_for((long long)pad, 256, h->num_sms), 256, 0, stream>>>(
        h->d_veff, h->n[0], h->n[1], h->n[2], h->m[0], h->m[1], h->m[2], h->kdiag, h->omega, h->tau, dpad);
    SQ_CUDA(cudaGetLastError());

    RecursionArgs<T> a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < 3; i++) {
        a.n[i] = h->n[i];
        a.m[i] = h->m[i];
        a.nc[i] = h->nc[i];
        a.pn[i] = h->pn[i];
        a.fac_off[i] = h->fac2_off[i];
        a.fac64_off[i] = h->fac64_off[i];
        for (int j = 1; j <= h->p; j++) a.w[i][j - 1] = (T)(-h->fd[j] / (2.0 * h->h[i] * h->h[i] * h->tau));
    }
    a.nc3 = h->nc3;
    a.N_d = h->N_d;
    a.q0 = 0;
    a.q1 = h->N_d;
    a.K = K;
    a.natom = h->natom;
    a.nproj = h->nproj;
    a.want_force = 0;
    a.dpad = dpad;
    a.kappa[0] = (T)(h->cl[0] * h->dV * h->Nnorm * h->Nnorm / h->tau);
    a.kappa[1] = (T)(h->cl[1] * h->dV * h->Nnorm * h->Nnorm / h->tau);
    if constexpr (sizeof(T) == 8) a.fac = reinterpret_cast<const T *>(h->d_fac2_64);
    else a.fac = reinterpret_cast<const T *>(h->d_fac2_32);
    a.fac_stride = h->fac2_stride;
    a.fac64 = h->d_fac64;
    a.fac64_stride = h->fac64_stride;
    a.sup_start = h->d_sup;
    a.sup_len = h->d_sup + 3 * (h->natom > 0 ? h->natom : 1);
    a.Nnorm = h->Nnorm;
    a.mu = reinterpret_cast<T *>(d_mu);
    a.A = nullptr;
    a.vec_in_smem = 0;
    a.scratch = vecs;

    const int block = 256;
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    const size_t smem = recursion_smem_bytes<T>(h->natom, h->nc, 0);
    if (smem > (size_t)dev_smem) return fail(SQ_ERR_UNSUPPORTED, "too many atoms for shared memory (%zu B)", smem);
    const int per_sm = recursion_blocks_per_sm<T>(h->p, block, smem, 0);
    if (per_sm < 1) return fail(SQ_ERR_UNSUPPORTED, "recursion kernel does not fit on an SM");
    long long grid = (long long)per_sm * h->num_sms;
    const long long fit = (long long)((kStaticScratchBytes - dpad_bytes) / per_cta);
    if (grid > fit) grid = fit;
    if (grid > h->N_d) grid = h->N_d;
    SQ_COUNT(1);
    SQ_CUDA(launch_recursion<T>(a, h->p, (int)grid, block, smem, stream));
    return SQ_OK;
}

extern "C" sq_status sq_moments_noalloc(sq_handle h, int K, int precision, void *d_mu, void *stream_)
{
    g_last_error[0] = 0;
    if (!h || !d_mu) return fail(SQ_ERR_ARG, "null argument");
    if (K < 1 || K > 4096) return fail(SQ_ERR_ARG, "K = %d", K);
    if (precision != SQ_FP64 && precision != SQ_FP32) return fail(SQ_ERR_ARG, "precision %d", precision);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != h->dev)
        return fail(SQ_ERR_ARG, "the handle's device (%d) is not the current device (%d)", h->dev, cur);
    cudaStream_t stream = (cudaStream_t)stream_;
    return precision == SQ_FP64 ? moments_noalloc<double>(h, K, d_mu, stream)
                                : moments_noalloc<float>(h, K, d_mu, stream);
}

// ------------------------------------------------------------------------------------------------
// Batched evaluation: many cells, one persistent recursion launch, a CUDA graph.  In FP32, cells whose
// cubes the slab kernel covers (cubic 21^3 / 25^3, 12th-order stencil) run as one slab launch each,
// captured in the same graph after the persistent launch over the other cells.

// Fermi state initialised on the device (capturable: no host memory behind the copy)
__global__ void k_fermi_init(FermiState *st, double lo, double hi)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        FermiState s;
        memset(&s, 0, sizeof(s));
        s.lo = lo;
        s.hi = hi;
        *st = s;
    }
}

// node functions at the Fermi level held in the device state (valid once phase == 3)
__global__ void k_node_functions_state(const double *lam, int M, const FermiState *st, double kT, double *fg,
                                       double *flg, double *fs)
{
    if (st->phase != 3) return;
    const double lam_f = st->x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const double l = lam[j];
        const double g = fermi_fn(l, lam_f, kT);
        const double y = fabs((l - lam_f) / kT);
        fg[j] = g;
        flg[j] = l * g;
        fs[j] = -(log1p(exp(-y)) + y * fermi_fn(y, 0.0, 1.0));
    }
}

constexpr int kBatchBisectSteps = 96;   // bisection launches captured in the graph (2 bracket + 94)

struct sq_batch_s {
    std::vector<sq_handle> cells;
    std::vector<int> K, M;
    std::vector<double> kT, N_e;
    int precision = 0, want_force = 0, fd_half = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<double *> graph_rho;          // d_rho pointers the graph was captured with
    void *d_cells = nullptr;                  // RecursionArgs<T> [ncells]
    BatchItem *d_items = nullptr;
    unsigned *d_counter = nullptr;
    void *d_scratch = nullptr;
    size_t scratch_cap = 0;
    int nitems = 0, chunk = 0, config = -1, grid = 0, block = 0, vec_in_smem = 0;
    size_t smem = 0;
    long long scratch_stride = 0;
    double tuned_ms = 0;
    size_t graph_nodes = 0;
    long long kernels_per_replay = 0;
    // FP32 slab cells: atom capacities and shared memory per cell (0: the cell is in the work queue)
    int slab_ready = 0, ngeneric = 0;
    std::vector<int> slab_amax, slab_fmax;
    std::vector<size_t> slab_smem;
    std::vector<int> slab_kind;               // 1: slab kernel (21^3, 25^3), 2: cluster kernel (29^3)
    std::vector<int> slab_ncl;                // clusters of a cluster launch
    void *d_cscratch = nullptr;               // v_{k-1} scratch of the cluster launches
    size_t cscratch_cap = 0;
};

extern "C" void sq_batch_destroy(sq_batch b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_cells);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    cudaFree(b->d_scratch);
    cudaFree(b->d_cscratch);
    delete b;
}

extern "C" sq_status sq_batch_create(const sq_handle *cells, int ncells, const int *K, const double *kT,
                                     const double *N_e, int precision, int flags, sq_batch *out)
{
    g_last_error[0] = 0;
    if (!cells || !K || !kT || !N_e || !out || ncells < 1) return fail(SQ_ERR_ARG, "null argument or ncells < 1");
    if (precision != SQ_FP64 && precision != SQ_FP32) return fail(SQ_ERR_ARG, "precision %d", precision);
    if (flags & ~(SQ_WANT_FORCE | SQ_KB_FMA)) return fail(SQ_ERR_ARG, "flags %d", flags);
    sq_batch_s *b = new sq_batch_s();
    auto cleanup = [&](sq_status s) {
        sq_batch_destroy(b);
        return s;
    };
    b->precision = precision;
    b->want_force = (flags & SQ_WANT_FORCE) ? 1 : 0;
    for (int i = 0; i < ncells; i++) {
        sq_handle h = cells[i];
        if (!h) return cleanup(fail(SQ_ERR_ARG, "cell %d: null handle", i));
        if (i > 0 && (h->p != cells[0]->p || h->dev != cells[0]->dev))
            return cleanup(fail(SQ_ERR_UNSUPPORTED, "cell %d: all cells must share the FD order and device", i));
        if (K[i] < 1 || K[i] > 4096 || !(kT[i] > 0) || !(N_e[i] > 0) || !(N_e[i] < 2.0 * h->N_d))
            return cleanup(fail(SQ_ERR_ARG, "cell %d: K=%d kT=%g N_e=%g", i, K[i], kT[i], N_e[i]));
        const double need = fmax(4.0 * (K[i] + 1), 16.0 * h->tau / kT[i]);
        int M = 1;
        while (M < need) M <<= 1;
        if (M > (1 << 26)) return cleanup(fail(SQ_ERR_UNSUPPORTED, "cell %d: kT/tau too small", i));
        h->kb_fma = (flags & SQ_KB_FMA) ? 1 : 0;
        b->cells.push_back(h);
        b->K.push_back(K[i]);
        b->kT.push_back(kT[i]);
        b->N_e.push_back(N_e[i]);
        b->M.push_back(M);
    }
    b->fd_half = cells[0]->p;
    // every buffer the graph touches is allocated now, never during capture
    const size_t esz = precision == SQ_FP64 ? 8 : 4;
    size_t max_nc3 = 0;
    int max_natom = 0;
    int max_nc[3] = {0, 0, 0};
    for (int i = 0; i < ncells; i++) {
        sq_handle h = b->cells[i];
        sq_status s;
        const int Ki = b->K[i];
        if ((s = ensure(&h->d_mu, &h->mu_bytes, esz * (size_t)(Ki + 1) * h->N_d))) return cleanup(s);
        if ((s = ensure(&h->d_msum, &h->msum_cap, sizeof(double) * (size_t)(Ki + 1)))) return cleanup(s);
        if ((s = ensure(&h->d_msum_part, &h->part_cap, sizeof(double) * (size_t)(Ki + 1) * kSumBlocks))) return cleanup(s);
        if (b->want_force && h->natom > 0)
            if ((s = ensure(&h->d_A, &h->A_cap, sizeof(double) * (size_t)(Ki + 1) * h->natom * h->nproj * 3))) return cleanup(s);
        if ((s = ensure(&h->d_coef, &h->coef_cap, sizeof(double) * 3 * (size_t)(Ki + 1)))) return cleanup(s);
        if ((s = ensure(&h->d_nodes, &h->nodes_cap, sizeof(double) * 5 * (size_t)b->M[i]))) return cleanup(s);
        const size_t pad = (size_t)h->pn[0] * h->pn[1] * h->pn[2];
        size_t cap = 0;
        if (precision == SQ_FP64 && !h->d_dpad64) {
            if ((s = ensure(&h->d_dpad64, &cap, sizeof(double) * pad))) return cleanup(s);
        } else if (precision == SQ_FP32 && !h->d_dpad32) {
            if ((s = ensure(&h->d_dpad32, &cap, sizeof(float) * pad))) return cleanup(s);
        }
        max_nc3 = std::max(max_nc3, (size_t)h->nc3);
        max_natom = std::max(max_natom, h->natom);
        for (int a = 0; a < 3; a++) max_nc[a] = std::max(max_nc[a], h->nc[a]);
    }
    int dev_smem = 0, num_sms = b->cells[0]->num_sms;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->cells[0]->dev);
    SQ_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    SQ_CUDA(cudaMalloc(&b->d_cells, (precision == SQ_FP64 ? sizeof(RecursionArgs<double>) : sizeof(RecursionArgs<float>)) * ncells));
    SQ_CUDA(cudaMalloc(&b->d_counter, 64));
    // candidate configurations: vectors in shared memory (512 or 256 threads) or in global scratch
    b->smem = 0;
    const size_t smem_vec = precision == SQ_FP64 ? recursion_smem_bytes<double>(max_natom, max_nc, 1)
                                                 : recursion_smem_bytes<float>(max_natom, max_nc, 1);
    const size_t smem_glob = precision == SQ_FP64 ? recursion_smem_bytes<double>(max_natom, max_nc, 0)
                                                  : recursion_smem_bytes<float>(max_natom, max_nc, 0);
    if (smem_glob > (size_t)dev_smem) return cleanup(fail(SQ_ERR_UNSUPPORTED, "too many atoms for shared memory"));
    b->scratch_stride = 2 * (long long)max_nc3;
    const long long scratch_bytes = (long long)esz * b->scratch_stride * num_sms * 2;
    SQ_CUDA(cudaMalloc(&b->d_scratch, scratch_bytes));
    b->scratch_cap = scratch_bytes;
    (void)smem_vec;
    *out = b;
    return SQ_OK;
}

template <typename T>
static sq_status batch_enqueue(sq_batch b, const RecursionArgs<T> *host_args, double *const *d_rho,
                               cudaStream_t stream, int config, int chunk, int limit_items, float *ms_out)
{
    const int nc = (int)b->cells.size();
    int dev_smem = 0, num_sms = b->cells[0]->num_sms;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->cells[0]->dev);
    // work items: column chunks of every cell outside the slab path
    std::vector<BatchItem> items;
    int max_natom = 0, max_nc[3] = {0, 0, 0};
    for (int i = 0; i < nc; i++) {
        if (b->slab_amax[i] != 0) continue;
        sq_handle h = b->cells[i];
        max_natom = std::max(max_natom, h->natom);
        for (int a = 0; a < 3; a++) max_nc[a] = std::max(max_nc[a], h->nc[a]);
        for (long long q = 0; q < h->N_d; q += chunk) items.push_back({i, 0, q, q + chunk});
    }
    if (items.empty() && ms_out) return fail(SQ_ERR_UNSUPPORTED, "no cell in the work queue");
    int nitems = (int)items.size();
    if (limit_items > 0 && nitems > limit_items) nitems = limit_items;
    BatchLaunch<T> L;
    memset(&L, 0, sizeof(L));
    if (nitems > 0) {
        L.vec_in_smem = config != 2;
        L.block = config == 0 ? 512 : 256;
        L.smem = recursion_smem_bytes<T>(max_natom, max_nc, L.vec_in_smem);
        if (L.smem > (size_t)dev_smem) return fail(SQ_ERR_UNSUPPORTED, "configuration %d does not fit", config);
        const int per_sm = batch_blocks_per_sm<T>(b->fd_half, L.block, L.smem, L.vec_in_smem);
        if (per_sm < 1) return fail(SQ_ERR_UNSUPPORTED, "configuration %d does not fit on an SM", config);
        L.grid = per_sm * num_sms;
        if (!L.vec_in_smem && (size_t)L.grid * b->scratch_stride * sizeof(T) > b->scratch_cap)
            L.grid = (int)(b->scratch_cap / (b->scratch_stride * sizeof(T)));
        if (!b->d_items || b->nitems < (int)items.size() || b->chunk != chunk) {
            if (b->d_items) cudaFree(b->d_items);
            SQ_CUDA(cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size()));
            SQ_CUDA(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
            b->nitems = (int)items.size();
            b->chunk = chunk;
        }
    }
    L.cells = reinterpret_cast<const RecursionArgs<T> *>(b->d_cells);
    L.items = b->d_items;
    L.nitems = nitems;
    L.counter = b->d_counter;
    L.scratch = reinterpret_cast<T *>(b->d_scratch);
    L.scratch_stride = b->scratch_stride;
    b->grid = L.grid;
    b->block = L.block;
    b->vec_in_smem = L.vec_in_smem;
    b->smem = L.smem;

    // per-cell diagonal and force accumulators
    for (int i = 0; i < nc; i++) {
        sq_handle h = b->cells[i];
        const size_t pad = (size_t)h->pn[0] * h->pn[1] * h->pn[2];
        T *dp = sizeof(T) == 8 ? reinterpret_cast<T *>(h->d_dpad64) : reinterpret_cast<T *>(h->d_dpad32);
        SQ_COUNT(1);
        k_dpad<T><<<grid_for((long long)pad, 256, h->num_sms), 256, 0, stream>>>(
            h->d_veff, h->n[0], h->n[1], h->n[2], h->m[0], h->m[1], h->m[2], h->kdiag, h->omega, h->tau, dp);
        SQ_CUDA(cudaGetLastError());
        if (b->want_force && h->natom > 0)
            SQ_CUDA(cudaMemsetAsync(h->d_A, 0, sizeof(double) * (size_t)(b->K[i] + 1) * h->natom * h->nproj * 3, stream));
    }
    SQ_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        SQ_CUDA(cudaEventCreate(&e0));
        SQ_CUDA(cudaEventCreate(&e1));
        SQ_CUDA(cudaEventRecord(e0, stream));
    }
    if (nitems > 0) {
        SQ_COUNT(1);
        SQ_CUDA(launch_batch<T>(L, b->fd_half, stream));
    }
    if (ms_out) {
        SQ_CUDA(cudaEventRecord(e1, stream));
        SQ_CUDA(cudaEventSynchronize(e1));
        SQ_CUDA(cudaEventElapsedTime(ms_out, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return SQ_OK;   // timing run of the recursion only
    }
    if constexpr (sizeof(T) == 4) {
        for (int i = 0; i < nc; i++) {
            if (b->slab_amax[i] == 0) continue;
            sq_handle h = b->cells[i];
            int *d_err = reinterpret_cast<int *>(h->d_small) + 42;
            SQ_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), stream));
            SQ_COUNT(1);
            if (b->slab_kind[i] == 2)
                SQ_CUDA(launch_cluster(host_args[i], b->slab_amax[i], b->slab_fmax[i],
                                       (int)std::min<long long>(b->slab_ncl[i], h->N_d), b->slab_smem[i], d_err, stream));
            else
                SQ_CUDA(launch_slab(host_args[i], b->slab_amax[i], b->slab_fmax[i],
                                    (int)std::min<long long>(h->num_sms, h->N_d), b->slab_smem[i], d_err, stream));
        }
    }
    // per-cell moment sums, Fermi level (fixed number of bisection launches), weights and density
    for (int i = 0; i < nc; i++) {
        sq_handle h = b->cells[i];
        const int K = b->K[i], M = b->M[i];
        int *d_bad = reinterpret_cast<int *>(h->d_small);
        SQ_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), stream));
        dim3 g2(kSumBlocks, K + 1);
        SQ_COUNT(2);
        k_msum_partial<T><<<g2, 256, 0, stream>>>(reinterpret_cast<const T *>(h->d_mu), h->N_d, K, h->d_msum_part,
                                              0LL, h->N_d);
        k_msum_final<<<1, 256, 0, stream>>>(h->d_msum_part, kSumBlocks, K, h->d_msum, d_bad);
        SQ_CUDA(cudaGetLastError());
        double *lam = h->d_nodes, *D = h->d_nodes + M, *f0 = h->d_nodes + 2 * M, *f1 = h->d_nodes + 3 * M,
               *f2 = h->d_nodes + 4 * M;
        FermiState *st = reinterpret_cast<FermiState *>(reinterpret_cast<char *>(h->d_small) + 256);
        double *part = reinterpret_cast<double *>(reinterpret_cast<char *>(h->d_small) + 512);
        SQ_COUNT(2 + kBatchBisectSteps);
        k_nodes<<<grid_for(M, 256, h->num_sms), 256, 0, stream>>>(h->d_msum, K, M, h->omega, h->tau, lam, D);
        k_fermi_init<<<1, 32, 0, stream>>>(st, h->lmin, h->lmax_);
        for (int it = 0; it < kBatchBisectSteps; it++)
            k_fermi_step<<<kFermiBlocks, 256, 0, stream>>>(lam, D, M, b->kT[i], b->N_e[i], st, part);
        SQ_CUDA(cudaGetLastError());
        SQ_COUNT(3);
        k_node_functions_state<<<grid_for(M, 256, h->num_sms), 256, 0, stream>>>(lam, M, st, b->kT[i], f0, f1, f2);
        k_coeffs<<<dim3(K + 1, 3), 256, 0, stream>>>(f0, f1, f2, M, K, h->d_coef);
        k_density<T><<<grid_for(h->N_d, 256, h->num_sms), 256, 0, stream>>>(reinterpret_cast<const T *>(h->d_mu),
                                                                           h->N_d, K, h->d_coef, 1.0 / h->dV, d_rho[i], 0LL, h->N_d);
        SQ_CUDA(cudaGetLastError());
    }
    return SQ_OK;
}

template <typename T>
static sq_status batch_run(sq_batch b, double *const *d_rho, double *lambda_f, cudaStream_t stream)
{
    const int nc = (int)b->cells.size();
    // device argument blocks of every cell
    std::vector<RecursionArgs<T>> args(nc);
    for (int i = 0; i < nc; i++) fill_args<T>(b->cells[i], b->K[i], b->want_force && b->cells[i]->natom > 0, args[i]);
    SQ_CUDA(cudaMemcpy(b->d_cells, args.data(), sizeof(RecursionArgs<T>) * nc, cudaMemcpyHostToDevice));
    // once: which cells take the FP32 slab kernel, with the atom capacities of their cubes
    if (!b->slab_ready) {
        b->slab_amax.assign(nc, 0);
        b->slab_fmax.assign(nc, 0);
        b->slab_smem.assign(nc, 0);
        b->slab_kind.assign(nc, 0);
        b->slab_ncl.assign(nc, 0);
        if constexpr (sizeof(T) == 4) {
            int dev_smem = 0;
            cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->cells[0]->dev);
            for (int i = 0; i < nc; i++) {
                sq_handle h = b->cells[i];
                const bool cl = cluster_supported(h->nc, h->p);
                if (h->natom == 0 || !(cl || slab_supported(h->nc, h->p))) continue;
                int *d_cnt = reinterpret_cast<int *>(h->d_small) + 40;
                SQ_CUDA(cudaMemsetAsync(d_cnt, 0, 3 * sizeof(int), b->cap_stream));
                SQ_COUNT(1);
                SQ_CUDA(slab_counts(args[i], d_cnt, h->num_sms, b->cap_stream));
                int cnt[2];
                SQ_CUDA(cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, b->cap_stream));
                SQ_CUDA(cudaStreamSynchronize(b->cap_stream));
                const int amax = cnt[0] > 0 ? cnt[0] : 1, fmax = cnt[1] > 0 ? cnt[1] : 1;
                size_t sm = 0;
                int maxc = 0;
                if (cl) {
                    if (cluster_prepare(h->nc[0], amax, fmax, args[i].kb_fma, &sm, &maxc) != cudaSuccess || maxc < 1 ||
                        sm > (size_t)dev_smem) {
                        cudaGetLastError();
                        continue;
                    }
                } else {
                    sm = slab_smem_bytes(h->nc[0], amax, fmax);
                    if (sm > (size_t)dev_smem) continue;
                }
                b->slab_amax[i] = amax;
                b->slab_fmax[i] = fmax;
                b->slab_smem[i] = sm;
                b->slab_kind[i] = cl ? 2 : 1;
                b->slab_ncl[i] = maxc;
            }
        }
        b->ngeneric = 0;
        for (int i = 0; i < nc; i++) b->ngeneric += b->slab_amax[i] == 0;
        b->slab_ready = 1;
        if (b->ngeneric == 0) {   // no work queue: nothing to tune
            b->config = 1;
            b->chunk = 128;
        }
    }
    // cells on the cluster kernel keep v_{k-1} in per-CTA scratch; their launches run one after
    // another on the stream, so they share one buffer owned by the batch
    if (sizeof(T) == 4) {
        size_t need = 0;
        for (int i = 0; i < nc; i++)
            if (b->slab_kind[i] == 2)
                need = std::max(need, sizeof(float) * (size_t)cluster_scratch_floats(b->cells[i]->nc[0]) * 2 *
                                          (size_t)b->slab_ncl[i]);
        if (need > 0) {
            sq_status s = ensure(&b->d_cscratch, &b->cscratch_cap, need);
            if (s) return s;
            for (int i = 0; i < nc; i++)
                if (b->slab_kind[i] == 2) args[i].scratch = reinterpret_cast<T *>(b->d_cscratch);
        }
    }

    // autotune once: kernel configuration x work-item size, timed on a prefix of the work queue
    if (b->config < 0) {
        SQ_CUDA(cudaStreamSynchronize(stream));
        const int cfg_list[3] = {0, 1, 2};
        const int chunks[2] = {32, 128};
        float best = 1e30f;
        int bc = -1, bk = 128;
        for (int ci = 0; ci < 3; ci++)
            for (int ki = 0; ki < 2; ki++) {
                float ms = 0;
                // each probe times the same number of columns, 256 per SM (one 128-column item per CTA at
                // two CTAs per SM), at most a sixth of the work queue
                long long total = 0;
                for (int i = 0; i < nc; i++)
                    if (b->slab_amax[i] == 0) total += b->cells[i]->N_d;
                long long cols = std::min<long long>((long long)b->cells[0]->num_sms * 2 * 128, total / 6);
                const int probe = (int)std::max<long long>(1, cols / chunks[ki]);
                if (batch_enqueue<T>(b, args.data(), d_rho, b->cap_stream, cfg_list[ci], chunks[ki], probe, &ms) != SQ_OK)
                    continue;
                if (ms < best) {
                    best = ms;
                    bc = cfg_list[ci];
                    bk = chunks[ki];
                }
            }
        if (bc < 0) return fail(SQ_ERR_UNSUPPORTED, "no recursion configuration fits this batch");
        b->config = bc;
        b->chunk = -1;   // force the item table for the chosen chunk
        b->tuned_ms = best;
        b->nitems = 0;
        g_last_error[0] = 0;
        sq_status s = batch_enqueue<T>(b, args.data(), d_rho, b->cap_stream, bc, bk, 1, &best);   // item table
        if (s) return s;
        b->chunk = bk;
    }
    bool same = b->exec && (int)b->graph_rho.size() == nc;
    for (int i = 0; same && i < nc; i++) same = b->graph_rho[i] == d_rho[i];
    if (!same) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        SQ_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        const long long before = g_launches;
        sq_status s = batch_enqueue<T>(b, args.data(), d_rho, b->cap_stream, b->config, b->chunk, 0, nullptr);
        b->kernels_per_replay = g_launches - before;
        g_launches = before;
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &g);
        if (s) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        SQ_CUDA(ce);
        b->graph = g;
        SQ_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
        SQ_CUDA(cudaGraphGetNodes(g, nullptr, &b->graph_nodes));
        b->graph_rho.assign(d_rho, d_rho + nc);
    }
    SQ_CUDA(cudaGraphLaunch(b->exec, stream));
    SQ_COUNT(b->kernels_per_replay);
    SQ_CUDA(cudaStreamSynchronize(stream));
    // results and checks; a bisection that needs more than the captured steps continues here with the
    // same rule (rare: the Fermi level within a few ulp of zero)
    for (int i = 0; i < nc; i++) {
        sq_handle h = b->cells[i];
        int bad = 0;
        FermiState fin;
        FermiState *st = reinterpret_cast<FermiState *>(reinterpret_cast<char *>(h->d_small) + 256);
        SQ_CUDA(cudaMemcpy(&bad, h->d_small, sizeof(int), cudaMemcpyDeviceToHost));
        SQ_CUDA(cudaMemcpy(&fin, st, sizeof(fin), cudaMemcpyDeviceToHost));
        if (bad) return fail(SQ_ERR_NOT_FINITE, "cell %d: moment sums are not finite", i);
        h->kernel_used = b->slab_amax[i] > 0 ? b->slab_kind[i] : 0;
        if (h->kernel_used) {
            int slab_err = 0;
            SQ_CUDA(cudaMemcpy(&slab_err, reinterpret_cast<int *>(h->d_small) + 42, sizeof(int), cudaMemcpyDeviceToHost));
            if (slab_err == 3)
                return fail(SQ_ERR_UNSUPPORTED,
                            "cell %d: a warp's atom list exceeds the tensor-core projector path; create the batch "
                            "with SQ_KB_FMA", i);
            if (slab_err) return fail(SQ_ERR_UNSUPPORTED, "cell %d: a column exceeded the slab kernel's atom capacity", i);
        }
        if (fin.phase == 4)
            return fail(SQ_ERR_NO_BRACKET, "cell %d: N(lambda_min) = %.6g, N(lambda_max) = %.6g, N_e = %.6g", i,
                        fin.N_lo, fin.N_hi, b->N_e[i]);
        h->precision = b->precision;
        h->K = b->K[i];
        if (fin.phase != 3) {
            sq_status s = fermi_and_density(h, b->kT[i], b->N_e[i], d_rho[i], &fin.x, stream);
            if (s) return s;
        }
        h->kT = b->kT[i];
        h->N_e = b->N_e[i];
        h->lam_f = fin.x;
        h->M = b->M[i];
        h->have_force = b->want_force && h->natom > 0;
        h->q0 = 0;
        h->q1 = h->N_d;
        h->have_moments = 1;
        h->have_density = 1;
        if (lambda_f) lambda_f[i] = fin.x;
    }
    return SQ_OK;
}

extern "C" sq_status sq_batch_density(sq_batch b, double *const *d_rho, double *lambda_f, void *stream_)
{
    g_last_error[0] = 0;
    if (!b || !d_rho) return fail(SQ_ERR_ARG, "null argument");
    for (size_t i = 0; i < b->cells.size(); i++)
        if (!d_rho[i]) return fail(SQ_ERR_ARG, "cell %zu: null density buffer", i);
    cudaStream_t stream = (cudaStream_t)stream_;
    return b->precision == SQ_FP64 ? batch_run<double>(b, d_rho, lambda_f, stream)
                                   : batch_run<float>(b, d_rho, lambda_f, stream);
}

extern "C" sq_status sq_batch_info(sq_batch b, int *config, int *chunk, int *grid, double *tuned_ms, long long *graph_nodes)
{
    if (!b) return fail(SQ_ERR_ARG, "null batch");
    if (config) *config = b->config;
    if (chunk) *chunk = b->chunk;
    if (grid) *grid = b->grid;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    if (graph_nodes) *graph_nodes = (long long)b->graph_nodes;
    return SQ_OK;
}

// ------------------------------------------------------------------------------------------------
// Vector-Jacobian product of (rho, U) with respect to V_eff (reverse mode through the recursion).

// derivative functions at the Fermi level: dg/dlambda_f = g (1 - g)/kT, and lam * dg/dlambda_f
__global__ void k_node_deriv(const double *lam, int M, double lam_f, double kT, double *f0, double *f1)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const double g = fermi_fn(lam[j], lam_f, kT);
        const double gp = g * (1.0 - g) / kT;
        f0[j] = gp;
        f1[j] = lam[j] * gp;
    }
}

// R_k = sum_q rhobar_q mu_k^q (partial sums per block, then k_msum_final)
template <typename T>
__global__ void k_wsum_partial(const T *mu, const double *w, long long N_d, int K, double *part)
{
    const int k = blockIdx.y;
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N_d; q += (long long)gridDim.x * blockDim.x)
        s += w[q] * (double)mu[(size_t)k * N_d + q];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int wd = 0; wd < (int)(blockDim.x >> 5); wd++) t += red[wd];
        part[(size_t)k * gridDim.x + blockIdx.x] = t;
    }
}

// cotangent of the moments: mubar_k^q = alpha_k rhobar_q + beta_k with
//   alpha_k = 2 c_k / dV,  beta_k = 2 Ubar d_k - 2 c_k lambar / N',
//   N' = 2 sum c'_k M_k,  lambar = (2/dV) sum_k c'_k R_k + 2 Ubar sum_k d'_k M_k
// (implicit derivative of the Fermi level through N(lambda_f) = N_e, Eq. Ne)
__global__ void k_adj_scalars(const double *coef, const double *coefd, const double *msum, const double *R, int K,
                              double inv_dV, double Ubar, double *alpha, double *beta, double *diag)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double *c = coef, *d = coef + (K + 1);
    const double *cp = coefd, *dp = coefd + (K + 1);
    double Np = 0.0, lr = 0.0, ld = 0.0;
    for (int k = 0; k <= K; k++) {
        Np += cp[k] * msum[k];
        lr += cp[k] * R[k];
        ld += dp[k] * msum[k];
    }
    Np *= 2.0;
    const double lambar = 2.0 * inv_dV * lr + 2.0 * Ubar * ld;
    for (int k = 0; k <= K; k++) {
        alpha[k] = 2.0 * c[k] * inv_dV;
        beta[k] = 2.0 * Ubar * d[k] - 2.0 * c[k] * lambar / Np;
    }
    diag[0] = Np;
    diag[1] = lambar;
}

template <typename T>
static sq_status density_vjp(sq_handle h, const double *d_rho_bar, double U_bar, int kc, double *d_vbar,
                             cudaStream_t stream)
{
    const int K = h->K, M = h->M;
    sq_status s;
    // scratch: c', d' coefficients, R, alpha, beta
    double *d_aux = nullptr;
    size_t aux_cap = 0;
    const size_t aux = sizeof(double) * (size_t)(5 * (K + 1) + 8);
    if ((s = ensure(&d_aux, &aux_cap, aux))) return s;
    double *coefd = d_aux, *R = coefd + 2 * (K + 1), *alpha = R + (K + 1), *beta = alpha + (K + 1),
           *diag = beta + (K + 1);
    double *lam = h->d_nodes, *f0 = h->d_nodes + 2 * M, *f1 = h->d_nodes + 3 * M;
    SQ_COUNT(2);
    k_node_deriv<<<grid_for(M, 256, h->num_sms), 256, 0, stream>>>(lam, M, h->lam_f, h->kT, f0, f1);
    k_coeffs<<<dim3(K + 1, 2), 256, 0, stream>>>(f0, f1, f1, M, K, coefd);
    dim3 g2(kSumBlocks, K + 1);
    SQ_COUNT(3);
    k_wsum_partial<T><<<g2, 256, 0, stream>>>(reinterpret_cast<const T *>(h->d_mu), d_rho_bar, h->N_d, K,
                                              h->d_msum_part);
    int *d_bad = reinterpret_cast<int *>(h->d_small) + 1;
    k_msum_final<<<1, 256, 0, stream>>>(h->d_msum_part, kSumBlocks, K, R, d_bad);
    k_adj_scalars<<<1, 32, 0, stream>>>(h->d_coef, coefd, h->d_msum, R, K, 1.0 / h->dV, U_bar, alpha, beta, diag);
    SQ_CUDA(cudaGetLastError());
    SQ_CUDA(cudaMemsetAsync(d_vbar, 0, sizeof(double) * h->N_d, stream));

    RecursionArgs<T> a;
    fill_args<T>(h, K, 0, a);
    a.adj_rho_bar = d_rho_bar;
    a.adj_alpha = alpha;
    a.adj_beta = beta;
    a.adj_vbar = d_vbar;
    a.adj_kc = kc;
    a.adj_inv_tau = 1.0 / h->tau;
    const int nsegs = (K + kc - 1) / kc;
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    if constexpr (sizeof(T) == 4) {
        // FP32 on 21^3 / 25^3 cubes with the 12th-order stencil: the slab mapping of the forward kernel
        if (h->natom > 0 && slab_supported(h->nc, h->p)) {
            int *d_cnt = reinterpret_cast<int *>(h->d_small) + 40;
            SQ_CUDA(cudaMemsetAsync(d_cnt, 0, 3 * sizeof(int), stream));
            SQ_COUNT(1);
            SQ_CUDA(slab_counts(a, d_cnt, h->num_sms, stream));
            int cnt[2];
            SQ_CUDA(cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, stream));
            SQ_CUDA(cudaStreamSynchronize(stream));
            const int amax = cnt[0] > 0 ? cnt[0] : 1;
            const size_t sm = slab_smem_bytes(h->nc[0], amax, 1);
            if (sm <= (size_t)dev_smem) {
                const long long sstride = (long long)(2 * nsegs + kc + 4) * slab_vector_floats(h->nc[0]);
                long long grid = h->num_sms;
                if (grid > h->N_d) grid = h->N_d;
                if ((s = ensure(&h->d_scratch, &h->scratch_cap, sizeof(T) * (size_t)sstride * grid))) {
                    cudaFree(d_aux);
                    return s;
                }
                a.scratch = reinterpret_cast<T *>(h->d_scratch);
                SQ_COUNT(1);
                cudaError_t e = launch_slab_adjoint(a, amax, (int)grid, sm, d_cnt + 2, sstride, stream);
                if (e != cudaSuccess) {
                    cudaFree(d_aux);
                    return fail(SQ_ERR_CUDA, "adjoint launch: %s", cudaGetErrorString(e));
                }
                int slab_err = 0;
                SQ_CUDA(cudaMemcpyAsync(&slab_err, d_cnt + 2, sizeof(int), cudaMemcpyDeviceToHost, stream));
                SQ_CUDA(cudaStreamSynchronize(stream));
                cudaFree(d_aux);
                if (slab_err) return fail(SQ_ERR_UNSUPPORTED, "a column exceeded the slab kernel's atom capacity (%d)", slab_err);
                return SQ_OK;
            }
        }
    }
    const long long stride = (long long)(2 + 2 * nsegs + kc + 1 + 3) * h->nc3;
    const size_t smem = recursion_smem_bytes<T>(h->natom, h->nc, 0);
    if (smem > (size_t)dev_smem) { cudaFree(d_aux); return fail(SQ_ERR_UNSUPPORTED, "too many atoms for shared memory"); }
    long long grid = 2LL * h->num_sms;
    if (grid > h->N_d) grid = h->N_d;
    if ((s = ensure(&h->d_scratch, &h->scratch_cap, sizeof(T) * (size_t)stride * grid))) { cudaFree(d_aux); return s; }
    a.scratch = reinterpret_cast<T *>(h->d_scratch);
    SQ_COUNT(1);
    cudaError_t e = launch_adjoint<T>(a, h->p, stride, (int)grid, smem, stream);
    if (e != cudaSuccess) { cudaFree(d_aux); return fail(SQ_ERR_CUDA, "adjoint launch: %s", cudaGetErrorString(e)); }
    SQ_CUDA(cudaStreamSynchronize(stream));
    cudaFree(d_aux);
    return SQ_OK;
}

extern "C" sq_status sq_density_vjp(sq_handle h, const double *d_rho_bar, double U_bar, int checkpoint_k,
                                    double *d_veff_bar, void *stream_)
{
    g_last_error[0] = 0;
    if (!h || !d_rho_bar || !d_veff_bar) return fail(SQ_ERR_ARG, "null argument");
    if (!h->have_density || h->q0 != 0 || h->q1 != h->N_d || h->gauss)
        return fail(SQ_ERR_STATE, "sq_density_vjp needs a whole-grid Chebyshev sq_density first");
    if (checkpoint_k < 1 || checkpoint_k > h->K) return fail(SQ_ERR_ARG, "checkpoint interval %d (K = %d)", checkpoint_k, h->K);
    if (!std::isfinite(U_bar)) return fail(SQ_ERR_NOT_FINITE, "U_bar");
    cudaStream_t stream = (cudaStream_t)stream_;
    return h->precision == SQ_FP64 ? density_vjp<double>(h, d_rho_bar, U_bar, checkpoint_k, d_veff_bar, stream)
                                   : density_vjp<float>(h, d_rho_bar, U_bar, checkpoint_k, d_veff_bar, stream);
}

// ------------------------------------------------------------------------------------------------
// Self-consistency pieces around the density (Sec. 2.1 LDA and Eq. Poisson; Sec. 3 "Electrostatic
// and effective potential"): V_xc, pseudocharges, the periodic FD Poisson solve, V_eff = V_xc + phi.

namespace {

int current_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// device buffer freed on every return path
struct DevBuf {
    double *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

sq_status check_grid(const int n[3], const double box[3])
{
    if (!n || !box) return fail(SQ_ERR_ARG, "null grid");
    for (int a = 0; a < 3; a++)
        if (n[a] < 1 || !(box[a] > 0) || !std::isfinite(box[a]))
            return fail(SQ_ERR_ARG, "axis %d: n = %d, box = %g", a, n[a], box[a]);
    return SQ_OK;
}

// a.b (sum of a when b is null) in a fixed order: per-block partial sums, added on the host in order
sq_status dot_fixed(long long N, const double *a, const double *b, double *d_part, cudaStream_t stream, double *out)
{
    double part[kDotBlocks];
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_dot_partial(N, a, b, d_part, stream));
    SQ_CUDA(cudaMemcpyAsync(part, d_part, sizeof(part), cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    double s = 0.0;
    for (int i = 0; i < kDotBlocks; i++) s += part[i];
    *out = s;
    return SQ_OK;
}

// -(1/4 pi) L_h phi = f - mean(f), mean(phi) = 0, by conjugate gradients on -L_h (symmetric positive
// definite on zero-mean grid functions); work: 3 N + kDotBlocks doubles.
sq_status poisson_cg(const int n[3], const double box[3], int fd_order, const double *d_f, double tol, int max_iter,
                     double *d_phi, double *work, int *iters, double *rel_res, cudaStream_t stream)
{
    const long long N = (long long)n[0] * n[1] * n[2];
    const int sms = current_sms();
    sq::LapWeights w;
    double c[kMaxHalfWidth + 1] = {0};
    fd_coefficients(fd_order, c);
    w.p = fd_order / 2;
    for (int a = 0; a < 3; a++) {
        const double ha = box[a] / n[a];
        for (int d = 0; d <= kMaxHalfWidth; d++) w.c[a][d] = d <= w.p ? c[d] / (ha * ha) : 0.0;
    }
    double *r = work, *p = work + N, *Ap = work + 2 * N, *part = work + 3 * N;
    const double four_pi = 4.0 * 3.14159265358979323846;
    sq_status s;
    double fsum = 0.0;
    if ((s = dot_fixed(N, d_f, nullptr, part, stream, &fsum))) return s;
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_affine(N, d_f, four_pi, -fsum / (double)N, r, sms, stream));
    SQ_CUDA(cudaMemsetAsync(d_phi, 0, sizeof(double) * N, stream));
    double rr = 0.0;
    if ((s = dot_fixed(N, r, r, part, stream, &rr))) return s;
    const double bnorm = std::sqrt(rr);
    *iters = 0;
    *rel_res = 0.0;
    if (!std::isfinite(bnorm)) return fail(SQ_ERR_NOT_FINITE, "Poisson right-hand side");
    if (bnorm == 0.0) return SQ_OK;
    SQ_CUDA(cudaMemcpyAsync(p, r, sizeof(double) * N, cudaMemcpyDeviceToDevice, stream));
    bool converged = false;
    int it = 0;
    while (it < max_iter) {
        it++;
        SQ_COUNT(1);
        SQ_CUDA(sq::launch_neg_laplacian(n, w, p, Ap, sms, stream));
        double pAp = 0.0;
        if ((s = dot_fixed(N, p, Ap, part, stream, &pAp))) return s;
        if (!(pAp > 0.0)) return fail(SQ_ERR_NOT_FINITE, "Poisson CG breakdown at iteration %d", it);
        const double alpha = rr / pAp;
        SQ_COUNT(1);
        SQ_CUDA(sq::launch_cg_step(N, alpha, p, Ap, d_phi, r, sms, stream));
        double rr_new = 0.0;
        if ((s = dot_fixed(N, r, r, part, stream, &rr_new))) return s;
        *rel_res = std::sqrt(rr_new) / bnorm;
        if (*rel_res <= tol) {
            converged = true;
            break;
        }
        SQ_COUNT(1);
        SQ_CUDA(sq::launch_cg_dir(N, rr_new / rr, r, p, sms, stream));
        rr = rr_new;
    }
    *iters = it;
    // rounding lets a constant creep in: restore the zero-mean gauge
    double psum = 0.0;
    if ((s = dot_fixed(N, d_phi, nullptr, part, stream, &psum))) return s;
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_affine(N, d_phi, 1.0, -psum / (double)N, d_phi, sms, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    if (!converged)
        return fail(SQ_ERR_TIMEOUT, "Poisson CG: relative residual %.3e after %d iterations", *rel_res, it);
    return SQ_OK;
}

}  // namespace

extern "C" sq_status sq_lda_pw92(long long n, const double *d_rho, double *d_exc, double *d_vxc, void *stream_)
{
    g_last_error[0] = 0;
    if (n < 1 || !d_rho || !d_exc || !d_vxc) return fail(SQ_ERR_ARG, "n = %lld or a null pointer", n);
    cudaStream_t stream = (cudaStream_t)stream_;
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_lda_pw92(n, d_rho, d_exc, d_vxc, current_sms(), stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    return SQ_OK;
}

extern "C" sq_status sq_pseudocharge(const int n[3], const double box[3], int natom, const double *R, const double *Z,
                                     double sigma_b, double *d_b, void *stream_)
{
    g_last_error[0] = 0;
    sq_status s;
    if ((s = check_grid(n, box))) return s;
    if (!d_b || natom < 0 || (natom > 0 && (!R || !Z))) return fail(SQ_ERR_ARG, "null argument or natom = %d", natom);
    if (!(sigma_b > 0) || !std::isfinite(sigma_b)) return fail(SQ_ERR_ARG, "sigma_b = %g", sigma_b);
    cudaStream_t stream = (cudaStream_t)stream_;
    std::vector<double> rz(4 * (size_t)std::max(natom, 1), 0.0);
    for (int J = 0; J < natom; J++) {
        for (int a = 0; a < 3; a++) rz[4 * J + a] = R[3 * J + a];
        rz[4 * J + 3] = Z[J];
        for (int a = 0; a < 4; a++)
            if (!std::isfinite(rz[4 * J + a])) return fail(SQ_ERR_NOT_FINITE, "atom %d", J);
    }
    DevBuf d_rz;
    SQ_CUDA(cudaMalloc(&d_rz.p, sizeof(double) * rz.size()));
    SQ_CUDA(cudaMemcpyAsync(d_rz.p, rz.data(), sizeof(double) * rz.size(), cudaMemcpyHostToDevice, stream));
    const double h[3] = {box[0] / n[0], box[1] / n[1], box[2] / n[2]};
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_pseudocharge(n, h, box, natom, d_rz.p, sigma_b, d_b, current_sms(), stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    return SQ_OK;
}

extern "C" sq_status sq_poisson_periodic(const int n[3], const double box[3], int fd_order, const double *d_f,
                                         double tol, int max_iter, double *d_phi, int *iters, double *rel_res,
                                         void *stream_)
{
    g_last_error[0] = 0;
    sq_status s;
    if ((s = check_grid(n, box))) return s;
    if (fd_order < 2 || fd_order > 2 * kMaxHalfWidth || fd_order % 2) return fail(SQ_ERR_ARG, "fd_order %d", fd_order);
    if (!d_f || !d_phi || !iters || !rel_res) return fail(SQ_ERR_ARG, "null argument");
    if (!(tol > 0) || max_iter < 1) return fail(SQ_ERR_ARG, "tol = %g, max_iter = %d", tol, max_iter);
    const long long N = (long long)n[0] * n[1] * n[2];
    DevBuf work;
    SQ_CUDA(cudaMalloc(&work.p, sizeof(double) * (3 * (size_t)N + kDotBlocks)));
    return poisson_cg(n, box, fd_order, d_f, tol, max_iter, d_phi, work.p, iters, rel_res, (cudaStream_t)stream_);
}

extern "C" sq_status sq_effective_potential(const int n[3], const double box[3], int fd_order, const double *d_rho,
                                            const double *d_b, double tol, int max_iter, double *d_phi,
                                            double *d_exc, double *d_vxc, double *d_veff, int *iters,
                                            double *rel_res, void *stream_)
{
    g_last_error[0] = 0;
    sq_status s;
    if ((s = check_grid(n, box))) return s;
    if (fd_order < 2 || fd_order > 2 * kMaxHalfWidth || fd_order % 2) return fail(SQ_ERR_ARG, "fd_order %d", fd_order);
    if (!d_rho || !d_b || !d_phi || !d_exc || !d_vxc || !d_veff || !iters || !rel_res)
        return fail(SQ_ERR_ARG, "null argument");
    if (!(tol > 0) || max_iter < 1) return fail(SQ_ERR_ARG, "tol = %g, max_iter = %d", tol, max_iter);
    cudaStream_t stream = (cudaStream_t)stream_;
    const long long N = (long long)n[0] * n[1] * n[2];
    const int sms = current_sms();
    DevBuf work;
    SQ_CUDA(cudaMalloc(&work.p, sizeof(double) * (4 * (size_t)N + kDotBlocks)));
    double *f = work.p + 3 * N + kDotBlocks;
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_add(N, d_rho, d_b, f, sms, stream));
    if ((s = poisson_cg(n, box, fd_order, f, tol, max_iter, d_phi, work.p, iters, rel_res, stream))) return s;
    SQ_COUNT(2);
    SQ_CUDA(sq::launch_lda_pw92(N, d_rho, d_exc, d_vxc, sms, stream));
    SQ_CUDA(sq::launch_add(N, d_vxc, d_phi, d_veff, sms, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    return SQ_OK;
}

// ------------------------------------------------------------------------------------------------
// Anderson mixing of the effective potential (Sec. 3: "In every SCF iteration, we mix the effective
// potential V_eff"): vectors stay on the device, the small least-squares system is solved on the host.

struct sq_mixer_s {
    long long n = 0;
    int m = 0;            // history length
    double beta = 0.0;    // mixing parameter
    int count = 0;        // differences held (<= m)
    int head = 0;         // slot of the next difference
    bool has_prev = false;
    double *buf = nullptr;   // [prev_v, prev_F, F, dV[m], dF[m], part]
    double *prev_v() const { return buf; }
    double *prev_F() const { return buf + n; }
    double *F() const { return buf + 2 * n; }
    double *dV(int j) const { return buf + (3 + (size_t)j) * n; }
    double *dF(int j) const { return buf + (3 + (size_t)m + j) * n; }
    double *part() const { return buf + (3 + 2 * (size_t)m) * n; }
};

extern "C" sq_status sq_mixer_create(long long n, int history, double beta, sq_mixer *out)
{
    g_last_error[0] = 0;
    if (!out || n < 1 || history < 0 || history > 32 || !(beta > 0) || !(beta <= 1))
        return fail(SQ_ERR_ARG, "n = %lld, history = %d, beta = %g", n, history, beta);
    *out = nullptr;
    sq_mixer_s *m = new sq_mixer_s();
    m->n = n;
    m->m = history;
    m->beta = beta;
    const size_t doubles = (3 + 2 * (size_t)history) * (size_t)n + kDotBlocks;
    if (cudaMalloc(&m->buf, sizeof(double) * doubles) != cudaSuccess) {
        delete m;
        cudaGetLastError();
        return fail(SQ_ERR_OOM, "mixer: %zu doubles", doubles);
    }
    *out = m;
    return SQ_OK;
}

extern "C" void sq_mixer_destroy(sq_mixer m)
{
    if (!m) return;
    if (m->buf) cudaFree(m->buf);
    delete m;
}

extern "C" sq_status sq_mixer_step(sq_mixer m, const double *d_vin, const double *d_vout, double *d_vnext,
                                   double *rel_err, void *stream_)
{
    g_last_error[0] = 0;
    if (!m || !d_vin || !d_vout || !d_vnext || !rel_err) return fail(SQ_ERR_ARG, "null argument");
    cudaStream_t stream = (cudaStream_t)stream_;
    const long long n = m->n;
    const int sms = current_sms();
    sq_status s;
    // F = V_out - V_in and its size relative to V_out
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_lincomb(n, 1.0, d_vout, -1.0, d_vin, m->F(), sms, stream));
    double ff = 0.0, oo = 0.0;
    if ((s = dot_fixed(n, m->F(), m->F(), m->part(), stream, &ff))) return s;
    if ((s = dot_fixed(n, d_vout, d_vout, m->part(), stream, &oo))) return s;
    if (!std::isfinite(ff) || !std::isfinite(oo)) return fail(SQ_ERR_NOT_FINITE, "mixer input");
    *rel_err = oo > 0.0 ? std::sqrt(ff / oo) : std::sqrt(ff);
    // the newest differences (dV, dF) = (V_in - V_in,prev, F - F_prev)
    if (m->has_prev && m->m > 0) {
        const int j = m->head;
        SQ_COUNT(2);
        SQ_CUDA(sq::launch_lincomb(n, 1.0, d_vin, -1.0, m->prev_v(), m->dV(j), sms, stream));
        SQ_CUDA(sq::launch_lincomb(n, 1.0, m->F(), -1.0, m->prev_F(), m->dF(j), sms, stream));
        m->head = (m->head + 1) % m->m;
        if (m->count < m->m) m->count++;
    }
    SQ_CUDA(cudaMemcpyAsync(m->prev_v(), d_vin, sizeof(double) * n, cudaMemcpyDeviceToDevice, stream));
    SQ_CUDA(cudaMemcpyAsync(m->prev_F(), m->F(), sizeof(double) * n, cudaMemcpyDeviceToDevice, stream));
    m->has_prev = true;
    // V_next = V_in + beta F - sum_j gamma_j (dV_j + beta dF_j), gamma minimising |F - sum_j gamma_j dF_j|
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_lincomb(n, 1.0, d_vin, m->beta, m->F(), d_vnext, sms, stream));
    const int k = m->count;
    if (k > 0) {
        double G[32 * 32], rhs[32], gam[32];
        for (int a = 0; a < k; a++) {
            for (int b = a; b < k; b++) {
                if ((s = dot_fixed(n, m->dF(a), m->dF(b), m->part(), stream, &G[a * k + b]))) return s;
                G[b * k + a] = G[a * k + b];
            }
            if ((s = dot_fixed(n, m->dF(a), m->F(), m->part(), stream, &rhs[a]))) return s;
        }
        double tr = 0.0;
        for (int a = 0; a < k; a++) tr += G[a * k + a];
        for (int a = 0; a < k; a++) G[a * k + a] += 1e-12 * tr / k;
        // Gaussian elimination with partial pivoting (k <= 32)
        for (int c = 0; c < k; c++) {
            int piv = c;
            for (int r = c + 1; r < k; r++)
                if (std::fabs(G[r * k + c]) > std::fabs(G[piv * k + c])) piv = r;
            if (!(std::fabs(G[piv * k + c]) > 0.0)) return fail(SQ_ERR_NOT_FINITE, "mixer: singular history");
            if (piv != c) {
                for (int q = 0; q < k; q++) std::swap(G[c * k + q], G[piv * k + q]);
                std::swap(rhs[c], rhs[piv]);
            }
            for (int r = c + 1; r < k; r++) {
                const double f = G[r * k + c] / G[c * k + c];
                for (int q = c; q < k; q++) G[r * k + q] -= f * G[c * k + q];
                rhs[r] -= f * rhs[c];
            }
        }
        for (int c = k - 1; c >= 0; c--) {
            double t = rhs[c];
            for (int q = c + 1; q < k; q++) t -= G[c * k + q] * gam[q];
            gam[c] = t / G[c * k + c];
        }
        for (int a = 0; a < k; a++) {
            SQ_COUNT(2);
            SQ_CUDA(sq::launch_lincomb(n, 1.0, d_vnext, -gam[a], m->dV(a), d_vnext, sms, stream));
            SQ_CUDA(sq::launch_lincomb(n, 1.0, d_vnext, -gam[a] * m->beta, m->dF(a), d_vnext, sms, stream));
        }
    }
    SQ_CUDA(cudaStreamSynchronize(stream));
    return SQ_OK;
}

// ------------------------------------------------------------------------------------------------
// Discrete free energy and local force (Sec. 3 "Free energy" and "Atomic forces")

namespace {

sq_status upload_atoms(int natom, const double *R, const double *Z, DevBuf &d_rz, cudaStream_t stream)
{
    std::vector<double> rz(4 * (size_t)std::max(natom, 1), 0.0);
    for (int J = 0; J < natom; J++) {
        for (int a = 0; a < 3; a++) rz[4 * J + a] = R[3 * J + a];
        rz[4 * J + 3] = Z[J];
        for (int a = 0; a < 4; a++)
            if (!std::isfinite(rz[4 * J + a])) return fail(SQ_ERR_NOT_FINITE, "atom %d", J);
    }
    SQ_CUDA(cudaMalloc(&d_rz.p, sizeof(double) * rz.size()));
    SQ_CUDA(cudaMemcpyAsync(d_rz.p, rz.data(), sizeof(double) * rz.size(), cudaMemcpyHostToDevice, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    return SQ_OK;
}

sq_status sum_partials(const double *d_part, cudaStream_t stream, double *out)
{
    double part[kDotBlocks];
    SQ_CUDA(cudaMemcpyAsync(part, d_part, sizeof(part), cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    double s = 0.0;
    for (int i = 0; i < kDotBlocks; i++) s += part[i];
    *out = s;
    return SQ_OK;
}

}  // namespace

extern "C" sq_status sq_self_energy(const int n[3], const double box[3], int natom, const double *R, const double *Z,
                                    double sigma_b, double *E_self, void *stream_)
{
    g_last_error[0] = 0;
    sq_status s;
    if ((s = check_grid(n, box))) return s;
    if (!E_self || natom < 0 || (natom > 0 && (!R || !Z))) return fail(SQ_ERR_ARG, "null argument or natom = %d", natom);
    if (!(sigma_b > 0) || !std::isfinite(sigma_b)) return fail(SQ_ERR_ARG, "sigma_b = %g", sigma_b);
    *E_self = 0.0;
    if (natom == 0) return SQ_OK;
    cudaStream_t stream = (cudaStream_t)stream_;
    DevBuf d_rz, part;
    if ((s = upload_atoms(natom, R, Z, d_rz, stream))) return s;
    SQ_CUDA(cudaMalloc(&part.p, sizeof(double) * kDotBlocks));
    const double h[3] = {box[0] / n[0], box[1] / n[1], box[2] / n[2]};
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_self_energy_partial(n, h, box, natom, d_rz.p, sigma_b, part.p, stream));
    double t = 0.0;
    if ((s = sum_partials(part.p, stream, &t))) return s;
    *E_self = -0.5 * h[0] * h[1] * h[2] * t;
    return SQ_OK;
}

extern "C" sq_status sq_free_energy(const int n[3], const double box[3], const double *d_rho, const double *d_b,
                                    const double *d_phi, const double *d_exc, const double *d_vxc, double F_band,
                                    double E_self, double *F, void *stream_)
{
    g_last_error[0] = 0;
    sq_status s;
    if ((s = check_grid(n, box))) return s;
    if (!d_rho || !d_b || !d_phi || !d_exc || !d_vxc || !F) return fail(SQ_ERR_ARG, "null argument");
    if (!std::isfinite(F_band) || !std::isfinite(E_self)) return fail(SQ_ERR_NOT_FINITE, "F_band or E_self");
    cudaStream_t stream = (cudaStream_t)stream_;
    const long long N = (long long)n[0] * n[1] * n[2];
    DevBuf part;
    SQ_CUDA(cudaMalloc(&part.p, sizeof(double) * kDotBlocks));
    SQ_COUNT(1);
    SQ_CUDA(sq::launch_free_energy_partial(N, d_rho, d_b, d_phi, d_exc, d_vxc, part.p, stream));
    double t = 0.0;
    if ((s = sum_partials(part.p, stream, &t))) return s;
    const double dV = (box[0] / n[0]) * (box[1] / n[1]) * (box[2] / n[2]);
    *F = F_band + dV * t + E_self;
    if (!std::isfinite(*F)) return fail(SQ_ERR_NOT_FINITE, "free energy");
    return SQ_OK;
}

extern "C" sq_status sq_local_force(const int n[3], const double box[3], int fd_order, int natom, const double *R,
                                    const double *Z, double sigma_b, const double *d_phi, double *force,
                                    void *stream_)
{
    g_last_error[0] = 0;
    sq_status s;
    if ((s = check_grid(n, box))) return s;
    if (fd_order < 2 || fd_order > 2 * kMaxHalfWidth || fd_order % 2) return fail(SQ_ERR_ARG, "fd_order %d", fd_order);
    if (!d_phi || !force || natom < 0 || (natom > 0 && (!R || !Z))) return fail(SQ_ERR_ARG, "null argument or natom");
    if (!(sigma_b > 0) || !std::isfinite(sigma_b)) return fail(SQ_ERR_ARG, "sigma_b = %g", sigma_b);
    if (natom == 0) return SQ_OK;
    cudaStream_t stream = (cudaStream_t)stream_;
    const long long N = (long long)n[0] * n[1] * n[2];
    const double h[3] = {box[0] / n[0], box[1] / n[1], box[2] / n[2]};
    sq::GradWeights gw;
    memset(&gw, 0, sizeof(gw));
    const Fd1Weights w1 = fd1_coefficients(fd_order);
    gw.p = w1.p;
    for (int a = 0; a < 3; a++)
        for (int d = 1; d <= w1.p; d++) gw.a[a][d] = w1.a[d] / h[a];
    DevBuf d_rz, g, d_f;
    if ((s = upload_atoms(natom, R, Z, d_rz, stream))) return s;
    SQ_CUDA(cudaMalloc(&g.p, sizeof(double) * 3 * (size_t)N));
    SQ_CUDA(cudaMalloc(&d_f.p, sizeof(double) * 3 * (size_t)natom));
    SQ_COUNT(2);
    SQ_CUDA(sq::launch_grad_h(n, gw, d_phi, g.p, current_sms(), stream));
    SQ_CUDA(sq::launch_local_force(n, h, box, natom, d_rz.p, sigma_b, h[0] * h[1] * h[2], g.p, d_f.p, stream));
    SQ_CUDA(cudaMemcpyAsync(force, d_f.p, sizeof(double) * 3 * (size_t)natom, cudaMemcpyDeviceToHost, stream));
    SQ_CUDA(cudaStreamSynchronize(stream));
    return SQ_OK;
}
