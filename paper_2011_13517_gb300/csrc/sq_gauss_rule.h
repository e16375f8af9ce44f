// Gauss rule of a symmetric tridiagonal Jacobi matrix, for host and device (internal to libsq).
//
// The Lanczos iteration of a column (Eq. Lanczos) gives the Jacobi matrix J_K = tridiag(b; a; b); the
// Gauss nodes are its eigenvalues and the weights the squared first components of its normalised
// eigenvectors (Sec. 2.2).  The eigendecomposition runs implicit symmetric QR sweeps with the
// Wilkinson shift (bulge chasing with Givens rotations, deflation of negligible off-diagonals) and
// carries only the first row of the accumulated rotations, which is all the weights need: O(K) memory
// and O(K^2) work per column.
#pragma once

#include <cmath>

namespace sq {

constexpr int kGaussMaxK = 256;   // largest polynomial order of the Gauss path

// On entry d[0..K-1] = a_1..a_K and e[0..K-1] = b_1..b_K (e[K-1] is not part of J_K).  The matrix is
// cut at the first b_k that is exactly zero (an exhausted Krylov space).  On exit d[0..n-1] hold the
// eigenvalues and z[0..n-1] the first components of the normalised eigenvectors (sum z^2 = 1).
// Returns n, or -n if the sweeps did not converge within 30 n + 30 of them.
__host__ __device__ inline int gauss_rule_inplace(double *d, double *e, double *z, int K)
{
    int n = K;
    for (int k = 0; k + 1 < K; k++)
        if (e[k] == 0.0) {
            n = k + 1;
            break;
        }
    double anorm = 0.0;
    for (int i = 0; i < n; i++) {
        z[i] = 0.0;
        const double r = fabs(d[i]) + (i + 1 < n ? fabs(e[i]) : 0.0);
        anorm = r > anorm ? r : anorm;
    }
    z[0] = 1.0;
    e[n - 1] = 0.0;
    const double eps = 2.220446049250313e-16;
    const double floor_abs = 1e-3 * eps * anorm;
    auto negligible = [&](int i) { return fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1])) + floor_abs; };
    int hi = n - 1, sweeps = 0;
    const int max_sweeps = 30 * n + 30;
    while (hi > 0) {
        if (negligible(hi - 1)) {
            e[hi - 1] = 0.0;
            hi--;
            continue;
        }
        if (++sweeps > max_sweeps) return -n;
        int lo = hi - 1;
        while (lo > 0 && !negligible(lo - 1)) lo--;
        // Wilkinson shift: the eigenvalue of the trailing 2x2 block nearer to d[hi]
        const double t = 0.5 * (d[hi - 1] - d[hi]);
        const double r = hypot(t, e[hi - 1]);
        const double mu = d[hi] - e[hi - 1] * e[hi - 1] / (t + (t >= 0.0 ? r : -r));
        // implicit QR sweep on rows lo..hi: the first rotation is set by the shifted first column,
        // the others chase the bulge it creates down the band
        double x = d[lo] - mu, y = e[lo];
        for (int k = lo; k < hi; k++) {
            const double rr = hypot(x, y);
            double c = 1.0, s = 0.0;
            if (rr != 0.0) {
                c = x / rr;
                s = y / rr;
            }
            if (k > lo) e[k - 1] = rr;
            const double dk = d[k], dk1 = d[k + 1], ek = e[k];
            d[k] = c * c * dk + 2.0 * c * s * ek + s * s * dk1;
            d[k + 1] = s * s * dk - 2.0 * c * s * ek + c * c * dk1;
            e[k] = c * s * (dk1 - dk) + (c * c - s * s) * ek;
            if (k < hi - 1) {
                x = e[k];
                y = s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            const double zk = z[k], zk1 = z[k + 1];
            z[k] = c * zk + s * zk1;
            z[k + 1] = -s * zk + c * zk1;
        }
    }
    return n;
}

}  // namespace sq
