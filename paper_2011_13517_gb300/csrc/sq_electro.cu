// Self-consistency pieces around the SQ density (Sec. 2.1, Sec. 3 "Electrostatic and effective
// potential"), FP64, one thread per grid point:
//   k_lda_pw92        eps_xc and V_xc = d(rho eps_xc)/d rho of the LDA: Slater exchange and the
//                     spin-unpolarised Perdew-Wang correlation (published fit, p = 1);
//   k_pseudocharge    b(x) = sum_J -Z_J (2 pi s^2)^(-3/2) exp(-|x - R_J|^2 / (2 s^2)), minimum image;
//   k_neg_laplacian   -L_h v for the periodic finite-difference Laplacian of the kinetic term;
//   k_dot_partial     fixed-order per-block partial sums of a.b (the host adds the blocks in order);
//   k_cg_*            vector updates of the conjugate-gradient solve of -(1/4 pi) L_h phi = f (Eq. Poisson);
//   k_lincomb         alpha a + beta b, the vector steps of the Anderson mixing of V_eff (Sec. 3);
//   k_grad_h, k_local_force, k_self_energy_partial, k_free_energy_partial
//                     the discrete local force (Eq. DiscreteLocalForce), self energy (Eq.
//                     DiscreteSelfEnergy) and the density terms of the free energy (Eq. DiscreteEnergy).
#include <cuda_runtime.h>

#include <cmath>

#include "sq_internal.h"

namespace sq {
namespace {

constexpr int kEBlock = 256;

__global__ void k_lda_pw92(long long n, const double *rho, double *exc, double *vxc)
{
    // Perdew-Wang correlation (zeta = 0): A, alpha1, beta1..beta4
    const double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
    const double pi = 3.14159265358979323846;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double r = rho[i];
        double e = 0.0, v = 0.0;
        if (r > 0.0) {
            const double r13 = cbrt(r);
            const double cx = cbrt(3.0 / pi);
            const double ex = -0.75 * cx * r13;               // Slater exchange per electron
            const double rs = cbrt(3.0 / (4.0 * pi * r));     // Wigner-Seitz radius
            const double s = sqrt(rs);
            const double q0 = -2.0 * A * (1.0 + a1 * rs);
            const double q1 = 2.0 * A * (b1 * s + b2 * rs + b3 * rs * s + b4 * rs * rs);
            const double dq1 = A * (b1 / s + 2.0 * b2 + 3.0 * b3 * s + 4.0 * b4 * rs);
            const double lg = log1p(1.0 / q1);
            const double ec = q0 * lg;
            const double dec = -2.0 * A * a1 * lg - q0 * dq1 / (q1 * q1 + q1);
            e = ex + ec;
            v = 4.0 / 3.0 * ex + ec - rs / 3.0 * dec;
        }
        exc[i] = e;
        vxc[i] = v;
    }
}

__global__ void k_pseudocharge(int n0, int n1, int n2, double h0, double h1, double h2, double L0, double L1, double L2,
                               int natom, const double *RZ, double sigma, double *b)
{
    const long long N = (long long)n0 * n1 * n2;
    const double norm = pow(2.0 * 3.14159265358979323846 * sigma * sigma, -1.5);
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % n0), j = (int)((q / n0) % n1), k = (int)(q / ((long long)n0 * n1));
        const double x = i * h0, y = j * h1, z = k * h2;
        double s = 0.0;
        for (int J = 0; J < natom; J++) {
            double dx = x - RZ[4 * J], dy = y - RZ[4 * J + 1], dz = z - RZ[4 * J + 2];
            dx -= L0 * rint(dx / L0);
            dy -= L1 * rint(dy / L1);
            dz -= L2 * rint(dz / L2);
            s -= RZ[4 * J + 3] * exp(-(dx * dx + dy * dy + dz * dz) * inv2s2);
        }
        b[q] = norm * s;
    }
}

__global__ void k_neg_laplacian(int n0, int n1, int n2, LapWeights w, const double *v, double *out)
{
    const long long N = (long long)n0 * n1 * n2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % n0), j = (int)((q / n0) % n1), k = (int)(q / ((long long)n0 * n1));
        const long long row = q - i, plane = (long long)k * n0 * n1;
        double s = (w.c[0][0] + w.c[1][0] + w.c[2][0]) * v[q];
        for (int d = 1; d <= w.p; d++) {
            const int ip = (i + d) % n0, im = ((i - d) % n0 + n0) % n0;
            const int jp = (j + d) % n1, jm = ((j - d) % n1 + n1) % n1;
            const int kp = (k + d) % n2, km = ((k - d) % n2 + n2) % n2;
            s += w.c[0][d] * (v[row + ip] + v[row + im]);
            s += w.c[1][d] * (v[plane + (long long)jp * n0 + i] + v[plane + (long long)jm * n0 + i]);
            s += w.c[2][d] * (v[(long long)kp * n0 * n1 + (long long)j * n0 + i] + v[(long long)km * n0 * n1 + (long long)j * n0 + i]);
        }
        out[q] = -s;
    }
}

__global__ void k_dot_partial(long long n, const double *a, const double *b, double *part)
{
    __shared__ double red[kEBlock];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += b ? a[i] * b[i] : a[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kEBlock / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out = s (in + c)
__global__ void k_affine(long long n, const double *in, double s, double c, double *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = s * (in[i] + c);
}

// x += alpha p, r -= alpha Ap
__global__ void k_cg_step(long long n, double alpha, const double *p, const double *Ap, double *x, double *r)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * Ap[i];
    }
}

// p = r + beta p
__global__ void k_cg_dir(long long n, double beta, const double *r, double *p)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = r[i] + beta * p[i];
}

// out = a + b
__global__ void k_add(long long n, const double *a, const double *b, double *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

// out = alpha a + beta b (out may be a or b)
__global__ void k_lincomb(long long n, double alpha, const double *a, double beta, const double *b, double *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = alpha * a[i] + beta * b[i];
}

// gradient nabla_h of the order of the Laplacian, periodic: g_a = sum_j a_j (v(x + j e_a) - v(x - j e_a)) / h_a
__global__ void k_grad_h(int n0, int n1, int n2, GradWeights gw, const double *v, double *gx, double *gy, double *gz)
{
    const long long N = (long long)n0 * n1 * n2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % n0), j = (int)((q / n0) % n1), k = (int)(q / ((long long)n0 * n1));
        const long long row = q - i, plane = (long long)k * n0 * n1;
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int d = 1; d <= gw.p; d++) {
            const int ip = (i + d) % n0, im = ((i - d) % n0 + n0) % n0;
            const int jp = (j + d) % n1, jm = ((j - d) % n1 + n1) % n1;
            const int kp = (k + d) % n2, km = ((k - d) % n2 + n2) % n2;
            sx += gw.a[0][d] * (v[row + ip] - v[row + im]);
            sy += gw.a[1][d] * (v[plane + (long long)jp * n0 + i] - v[plane + (long long)jm * n0 + i]);
            sz += gw.a[2][d] * (v[(long long)kp * n0 * n1 + (long long)j * n0 + i] - v[(long long)km * n0 * n1 + (long long)j * n0 + i]);
        }
        gx[q] = sx;
        gy[q] = sy;
        gz[q] = sz;
    }
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = kEBlock / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// squared minimum-image distance from grid point (i, j, k) to atom J
__device__ __forceinline__ double min_image_r2(int i, int j, int k, double h0, double h1, double h2, double L0, double L1,
                                               double L2, const double *RZ, int J)
{
    double dx = i * h0 - RZ[4 * J], dy = j * h1 - RZ[4 * J + 1], dz = k * h2 - RZ[4 * J + 2];
    dx -= L0 * rint(dx / L0);
    dy -= L1 * rint(dy / L1);
    dz -= L2 * rint(dz / L2);
    return dx * dx + dy * dy + dz * dz;
}

// per-block sums of sum_I b_I V_I over the grid points, V_I = -Z_I erf(r / (sqrt 2 s)) / r
__global__ void k_self_energy_partial(int n0, int n1, int n2, double h0, double h1, double h2, double L0, double L1,
                                      double L2, int natom, const double *RZ, double sigma, double *part)
{
    __shared__ double red[kEBlock];
    const long long N = (long long)n0 * n1 * n2;
    const double pi = 3.14159265358979323846;
    const double norm = pow(2.0 * pi * sigma * sigma, -1.5), inv2s2 = 1.0 / (2.0 * sigma * sigma);
    const double rs2 = 1.0 / (sqrt(2.0) * sigma), v0 = sqrt(2.0 / pi) / sigma;
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % n0), j = (int)((q / n0) % n1), k = (int)(q / ((long long)n0 * n1));
        for (int J = 0; J < natom; J++) {
            const double Z = RZ[4 * J + 3];
            const double r2 = min_image_r2(i, j, k, h0, h1, h2, L0, L1, L2, RZ, J);
            const double r = sqrt(r2);
            const double V = r > 0.0 ? -Z * erf(r * rs2) / r : -Z * v0;
            acc += -Z * norm * exp(-r2 * inv2s2) * V;
        }
    }
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// per-block sums of (eps_xc - V_xc) rho + (b - rho) phi / 2
__global__ void k_free_energy_partial(long long n, const double *rho, const double *b, const double *phi, const double *exc,
                                      const double *vxc, double *part)
{
    __shared__ double red[kEBlock];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (exc[i] - vxc[i]) * rho[i] + 0.5 * (b[i] - rho[i]) * phi[i];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// one block per atom J: f_J = -dV sum_q b_J^q (nabla_h phi)^q, the summation-by-parts form of
// dV sum_q (nabla_h b_J)^q phi^q on the periodic grid
__global__ void k_local_force(int n0, int n1, int n2, double h0, double h1, double h2, double L0, double L1, double L2,
                              const double *RZ, double sigma, double dV, const double *gx, const double *gy,
                              const double *gz, double *force)
{
    __shared__ double red[kEBlock];
    const int J = blockIdx.x;
    const long long N = (long long)n0 * n1 * n2;
    const double norm = pow(2.0 * 3.14159265358979323846 * sigma * sigma, -1.5), inv2s2 = 1.0 / (2.0 * sigma * sigma);
    const double Z = RZ[4 * J + 3];
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (long long q = threadIdx.x; q < N; q += blockDim.x) {
        const int i = (int)(q % n0), j = (int)((q / n0) % n1), k = (int)(q / ((long long)n0 * n1));
        const double bj = -Z * norm * exp(-min_image_r2(i, j, k, h0, h1, h2, L0, L1, L2, RZ, J) * inv2s2);
        sx += bj * gx[q];
        sy += bj * gy[q];
        sz += bj * gz[q];
    }
    sx = block_sum(sx, red);
    sy = block_sum(sy, red);
    sz = block_sum(sz, red);
    if (threadIdx.x == 0) {
        force[3 * J] = -dV * sx;
        force[3 * J + 1] = -dV * sy;
        force[3 * J + 2] = -dV * sz;
    }
}

int grid_of(long long n, int num_sms)
{
    long long g = (n + kEBlock - 1) / kEBlock;
    const long long cap = (long long)num_sms * 8;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_lda_pw92(long long n, const double *rho, double *exc, double *vxc, int num_sms, cudaStream_t stream)
{
    k_lda_pw92<<<grid_of(n, num_sms), kEBlock, 0, stream>>>(n, rho, exc, vxc);
    return cudaGetLastError();
}

cudaError_t launch_pseudocharge(const int n[3], const double h[3], const double L[3], int natom, const double *d_RZ,
                                double sigma, double *b, int num_sms, cudaStream_t stream)
{
    const long long N = (long long)n[0] * n[1] * n[2];
    k_pseudocharge<<<grid_of(N, num_sms), kEBlock, 0, stream>>>(n[0], n[1], n[2], h[0], h[1], h[2], L[0], L[1], L[2],
                                                               natom, d_RZ, sigma, b);
    return cudaGetLastError();
}

cudaError_t launch_neg_laplacian(const int n[3], const LapWeights &w, const double *v, double *out, int num_sms,
                                 cudaStream_t stream)
{
    const long long N = (long long)n[0] * n[1] * n[2];
    k_neg_laplacian<<<grid_of(N, num_sms), kEBlock, 0, stream>>>(n[0], n[1], n[2], w, v, out);
    return cudaGetLastError();
}

cudaError_t launch_dot_partial(long long n, const double *a, const double *b, double *part, cudaStream_t stream)
{
    k_dot_partial<<<kDotBlocks, kEBlock, 0, stream>>>(n, a, b, part);
    return cudaGetLastError();
}

cudaError_t launch_affine(long long n, const double *in, double s, double c, double *out, int num_sms, cudaStream_t stream)
{
    k_affine<<<grid_of(n, num_sms), kEBlock, 0, stream>>>(n, in, s, c, out);
    return cudaGetLastError();
}

cudaError_t launch_cg_step(long long n, double alpha, const double *p, const double *Ap, double *x, double *r,
                           int num_sms, cudaStream_t stream)
{
    k_cg_step<<<grid_of(n, num_sms), kEBlock, 0, stream>>>(n, alpha, p, Ap, x, r);
    return cudaGetLastError();
}

cudaError_t launch_cg_dir(long long n, double beta, const double *r, double *p, int num_sms, cudaStream_t stream)
{
    k_cg_dir<<<grid_of(n, num_sms), kEBlock, 0, stream>>>(n, beta, r, p);
    return cudaGetLastError();
}

cudaError_t launch_lincomb(long long n, double alpha, const double *a, double beta, const double *b, double *out,
                           int num_sms, cudaStream_t stream)
{
    k_lincomb<<<grid_of(n, num_sms), kEBlock, 0, stream>>>(n, alpha, a, beta, b, out);
    return cudaGetLastError();
}

cudaError_t launch_add(long long n, const double *a, const double *b, double *out, int num_sms, cudaStream_t stream)
{
    k_add<<<grid_of(n, num_sms), kEBlock, 0, stream>>>(n, a, b, out);
    return cudaGetLastError();
}

}  // namespace sq

namespace sq {

cudaError_t launch_grad_h(const int n[3], const GradWeights &gw, const double *v, double *g, int num_sms,
                          cudaStream_t stream)
{
    const long long N = (long long)n[0] * n[1] * n[2];
    k_grad_h<<<grid_of(N, num_sms), kEBlock, 0, stream>>>(n[0], n[1], n[2], gw, v, g, g + N, g + 2 * N);
    return cudaGetLastError();
}

cudaError_t launch_self_energy_partial(const int n[3], const double h[3], const double L[3], int natom, const double *d_RZ,
                                       double sigma, double *part, cudaStream_t stream)
{
    k_self_energy_partial<<<kDotBlocks, kEBlock, 0, stream>>>(n[0], n[1], n[2], h[0], h[1], h[2], L[0], L[1], L[2], natom,
                                                              d_RZ, sigma, part);
    return cudaGetLastError();
}

cudaError_t launch_free_energy_partial(long long n, const double *rho, const double *b, const double *phi,
                                       const double *exc, const double *vxc, double *part, cudaStream_t stream)
{
    k_free_energy_partial<<<kDotBlocks, kEBlock, 0, stream>>>(n, rho, b, phi, exc, vxc, part);
    return cudaGetLastError();
}

cudaError_t launch_local_force(const int n[3], const double h[3], const double L[3], int natom, const double *d_RZ,
                               double sigma, double dV, const double *g, double *d_force, cudaStream_t stream)
{
    const long long N = (long long)n[0] * n[1] * n[2];
    k_local_force<<<natom, kEBlock, 0, stream>>>(n[0], n[1], n[2], h[0], h[1], h[2], L[0], L[1], L[2], d_RZ, sigma, dV, g,
                                                 g + N, g + 2 * N, d_force);
    return cudaGetLastError();
}

}  // namespace sq
