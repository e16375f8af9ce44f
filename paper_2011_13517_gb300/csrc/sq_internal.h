// Internal declarations shared by the translation units of libsq (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sq.h"

namespace sq {

constexpr int kMaxHalfWidth = 8;   // FD order <= 16
constexpr int kNumFactors = 4;     // g, hp (p factor), g', hp' per atom and axis

// Adds n to the library's count of launched kernels (sq_kernel_launches).
void count_launches(long long n);

// Per-precision device data derived from the handle for one recursion launch.
template <typename T>
struct RecursionArgs {
    int n[3];            // grid points per axis
    int m[3];            // cube half-widths
    int nc[3];           // cube extents 2m+1
    int nc3;             // cube points
    long long N_d;       // grid points
    long long q0, q1;    // columns [q0, q1) of this launch (0 and N_d for the whole grid)
    const long long *cols;   // generic kernel only: when set, launch index i in [q0, q1) is column cols[i]
    int K;               // polynomial order
    int natom;
    int nproj;           // 1 (s) or 4 (s + p)
    int want_force;
    int kb_fma;          // cluster kernel: projector term on the CUDA cores instead of the tensor cores
    // scaled operator Hhat = (H - omega)/tau
    const T *dpad;       // Hhat diagonal on the periodically padded grid [n3+2m3][n2+2m2][n1+2m1]
    int pn[3];           // padded extents
    T w[3][kMaxHalfWidth];   // Hhat off-diagonal weights w[a][j-1] = -c_j / (2 h_a^2 tau)
    T kappa[2];          // c_l dV N^2 / tau for l = 0, 1
    // projector factor tables, doubled along each axis: element (J, a, f, i), i in [0, 2 n_a),
    // at J*fac_stride + fac_off[a] + f*2*n_a + i, equal to factor f of atom J on axis a at grid
    // index i mod n_a
    const T *fac;
    int fac_off[3];
    int fac_stride;
    const double *fac64; // FP64 tables [natom][3][4][n_a] (values of chi at the column centre)
    int fac64_off[3];
    int fac64_stride;
    const int *sup_start;   // [natom][3] first grid index of the support along each axis
    const int *sup_len;     // [natom][3] support length (n_a = whole axis)
    double Nnorm;        // projector normalisation N
    // outputs
    T *mu;               // [K+1][N_d]
    double *A;           // [K+1][natom][nproj][3] (accumulated with atomics) or null
    double *ab;          // Lanczos kernels: [2K][N_d], a_1..a_K then b_1..b_K of each column
    // vector storage
    T *scratch;          // [gridDim][2][nc3] when the vectors live in global memory
    int vec_in_smem;
    // reverse-mode pass (adjoint_kernel only): mubar_k = adj_alpha[k] adj_rho_bar[q] + adj_beta[k]
    const double *adj_rho_bar;
    const double *adj_alpha;
    const double *adj_beta;
    double *adj_vbar;    // accumulated with atomics
    int adj_kc;          // checkpoint interval
    double adj_inv_tau;
};

// Vector-Jacobian pass over all columns (scratch_stride elements of per-CTA scratch).
template <typename T>
cudaError_t launch_adjoint(const RecursionArgs<T> &args, int fd_half, long long scratch_stride, int grid,
                           size_t smem, cudaStream_t stream);

// One work item of a batched launch: columns [begin, end) of cell `cell`.
struct BatchItem {
    int cell;
    int pad;
    long long begin, end;
};

template <typename T>
struct BatchLaunch {
    const RecursionArgs<T> *cells;   // device [ncells]
    const BatchItem *items;          // device [nitems]
    int nitems;
    unsigned *counter;               // device, zero before the launch
    T *scratch;                      // per-CTA vectors when !vec_in_smem
    long long scratch_stride;        // elements per CTA
    int grid, block, vec_in_smem;
    size_t smem;
};

template <typename T>
cudaError_t launch_batch(const BatchLaunch<T> &b, int fd_half, cudaStream_t stream);
template <typename T>
int batch_blocks_per_sm(int fd_half, int block, size_t smem, int vec_in_smem);

// Lanczos iteration (Eq. Lanczos) of every column in [q0, q1) with the generic column machinery,
// writing args.ab; same launch configurations as launch_recursion.
template <typename T>
cudaError_t launch_lanczos(const RecursionArgs<T> &args, int fd_half, int grid, int block, size_t smem,
                           cudaStream_t stream);
template <typename T>
int lanczos_blocks_per_sm(int fd_half, int block, size_t smem, int vec_in_smem);

// Gauss nodes and weights of every column from its Lanczos coefficients (one thread per column):
// nodes[k][N_d] = tau lambda_hat_k + omega, weights[k][N_d]; *bad is set when a column's tridiagonal
// eigensolve did not converge.
cudaError_t launch_gauss_rule(const double *ab, long long N_d, long long q0, long long q1, int K, double omega,
                              double tau, double *nodes, double *weights, int *bad, int num_sms, cudaStream_t stream);

// Launch the per-column recursion for all N_d columns.  Returns cudaSuccess or the launch error.
template <typename T>
cudaError_t launch_recursion(const RecursionArgs<T> &args, int fd_half, int grid, int block,
                             size_t smem, cudaStream_t stream);

// Dynamic shared memory needed for one CTA of the recursion kernel.
template <typename T>
size_t recursion_smem_bytes(int natom, const int nc[3], int vec_in_smem);

// Occupancy helper: active CTAs per SM for the given configuration (block 256 with vectors in global
// scratch, or block 256/512 with vectors in shared memory).
template <typename T>
int recursion_blocks_per_sm(int fd_half, int block, size_t smem, int vec_in_smem);

// FP32 slab kernel (cubic cubes of 21 or 25 points, 12th-order FD): support test, shared memory
// for a given active/force atom capacity, the per-column capacity pre-pass (counts[0] = max active
// atoms, counts[1] = max force atoms; both must be zero-initialised) and the launch.  *err is set
// nonzero if a column exceeded the capacities.
bool slab_supported(const int nc[3], int fd_half);
size_t slab_smem_bytes(int nc, int amax, int fmax);
cudaError_t slab_counts(const RecursionArgs<float> &args, int *d_counts, int num_sms, cudaStream_t stream);
cudaError_t launch_slab(const RecursionArgs<float> &args, int amax, int fmax, int grid, size_t smem, int *err,
                        cudaStream_t stream);
// Reverse-mode pass with the slab mapping (args.adj_* set, args.want_force = 0): per-CTA scratch of
// scratch_stride floats = (2 nsegs + kc + 4) vectors of slab_vector_floats(nc) each; shared memory
// slab_smem_bytes(nc, amax, 1).
cudaError_t launch_slab_adjoint(const RecursionArgs<float> &args, int amax, int grid, size_t smem, int *err,
                                long long scratch_stride, cudaStream_t stream);
long long slab_vector_floats(int nc);

// FP32 cluster kernel (cubic 29^3 cubes, 12th-order FD): a cluster of two CTAs per column, each
// holding half of the cube's y-slabs.  Uses the slab kernel's capacity pre-pass (slab_counts).
// cluster_prepare gives the shared memory per CTA and how many clusters fit on the GPU at once; the
// launch needs args.scratch with cluster_scratch_floats(nc) floats per CTA (2 per cluster).
bool cluster_supported(const int nc[3], int fd_half);
long long cluster_scratch_floats(int nc);
cudaError_t cluster_prepare(int nc, int amax, int fmax, int kb_fma, size_t *smem, int *max_clusters);
cudaError_t launch_cluster(const RecursionArgs<float> &args, int amax, int fmax, int nclusters, size_t smem,
                           int *err, cudaStream_t stream);

// Self-consistency pieces (sq_electro.cu), FP64.  LapWeights: c[a][d] = FD weight c_d / h_a^2 of the
// kinetic term's Laplacian along axis a, d = 0..p.
struct LapWeights {
    int p;
    double c[3][kMaxHalfWidth + 1];
};
// GradWeights: a[a][d] = first-derivative FD weight a_d / h_a along axis a, d = 1..p.
struct GradWeights {
    int p;
    double a[3][kMaxHalfWidth + 1];
};
constexpr int kDotBlocks = 256;   // partial sums written by launch_dot_partial and the *_partial launchers
cudaError_t launch_lda_pw92(long long n, const double *rho, double *exc, double *vxc, int num_sms, cudaStream_t stream);
// d_RZ: device [natom][4] = (x, y, z, Z)
cudaError_t launch_pseudocharge(const int n[3], const double h[3], const double L[3], int natom, const double *d_RZ,
                                double sigma, double *b, int num_sms, cudaStream_t stream);
cudaError_t launch_neg_laplacian(const int n[3], const LapWeights &w, const double *v, double *out, int num_sms,
                                 cudaStream_t stream);
// part[kDotBlocks] = per-block sums of a.b (of a when b is null)
cudaError_t launch_dot_partial(long long n, const double *a, const double *b, double *part, cudaStream_t stream);
cudaError_t launch_affine(long long n, const double *in, double s, double c, double *out, int num_sms, cudaStream_t stream);
cudaError_t launch_cg_step(long long n, double alpha, const double *p, const double *Ap, double *x, double *r,
                           int num_sms, cudaStream_t stream);
cudaError_t launch_cg_dir(long long n, double beta, const double *r, double *p, int num_sms, cudaStream_t stream);
cudaError_t launch_add(long long n, const double *a, const double *b, double *out, int num_sms, cudaStream_t stream);
cudaError_t launch_lincomb(long long n, double alpha, const double *a, double beta, const double *b, double *out,
                           int num_sms, cudaStream_t stream);
// g: device [3][N] (x, y, z components)
cudaError_t launch_grad_h(const int n[3], const GradWeights &gw, const double *v, double *g, int num_sms,
                          cudaStream_t stream);
cudaError_t launch_self_energy_partial(const int n[3], const double h[3], const double L[3], int natom, const double *d_RZ,
                                       double sigma, double *part, cudaStream_t stream);
cudaError_t launch_free_energy_partial(long long n, const double *rho, const double *b, const double *phi,
                                       const double *exc, const double *vxc, double *part, cudaStream_t stream);
// one block per atom; d_force: device [natom][3]
cudaError_t launch_local_force(const int n[3], const double h[3], const double L[3], int natom, const double *d_RZ,
                               double sigma, double dV, const double *g, double *d_force, cudaStream_t stream);

}  // namespace sq
