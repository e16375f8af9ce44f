/*
 * sq.h -- C ABI of libsq: Clenshaw-Curtis (Chebyshev) spectral quadrature on one GB300 (sm_103a).
 *
 * The library evaluates, for a given local effective potential V_eff on a periodic finite-difference
 * grid and a set of atoms carrying Kleinman-Bylander projectors, the quantities of the linear-scaling
 * spectral quadrature (SQ) method of Ghosh & Bhattacharya, arXiv 2011.13517:
 *
 *   - for every grid point q, the Chebyshev recursion of the Hamiltonian H_q truncated to the cube of
 *     half-width R_cut around q (Sec. 3 "Hamiltonian at each grid point"; Eq. Chebyshev, Sec. 2.2),
 *     started from the unit vector e_q, and its moments mu_k^q = e_q^T T_k(Hhat_q) e_q;
 *   - the Fermi level from the electron-count constraint (Eq. Ne, Sec. 3), with the Chebyshev weights
 *     of the Fermi-Dirac function (Eq. ChebyshevWeights, Eq. FermiDirac);
 *   - the pointwise electron density (Eq. rhoq), the band energy U = 2 Tr(gamma H) and the electronic
 *     entropy S (Eqs. uq, sq, RSIntegrals);
 *   - the nonlocal atomic force from projector contractions of the same Chebyshev vectors
 *     (Eq. NLforceSQ and the discrete nonlocal force of Sec. 3 "Atomic forces").
 *
 * Conventions for every entry point:
 *   - Device buffers are caller-owned raw CUDA device pointers (allocated by e.g. PyTorch); host
 *     buffers are plain host pointers.  The library owns only the workspace behind a handle.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work is
 *     enqueued on that stream; entry points that return host scalars synchronise it.
 *   - Grid arrays are [n3][n2][n1] with x (axis 0) fastest; point index q = i1 + n1 (i2 + n2 i3).
 *   - Units: bohr and Hartree.  No exception or longjmp crosses the ABI.  A failing call returns a
 *     nonzero sq_status, leaves caller outputs untouched, and sets a message for sq_last_error().
 *   - One handle must not be used from two host threads at once.
 */
#ifndef SQ_H
#define SQ_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sq_handle_s *sq_handle;

typedef enum {
    SQ_OK = 0,
    SQ_ERR_ARG = 1,               /* invalid argument (null pointer, bad size, bad flag)          */
    SQ_ERR_CUBE_EXCEEDS_BOX = 2,  /* 2 round(R_cut/h_i) + 1 + n_o/2 > n_i on some axis            */
    SQ_ERR_NO_BRACKET = 3,        /* N(lambda_min) > N_e or N(lambda_max) < N_e                    */
    SQ_ERR_NOT_FINITE = 4,        /* V_eff, positions or a result is NaN/Inf                        */
    SQ_ERR_CUDA = 5,              /* a CUDA runtime call failed (see sq_last_error)                 */
    SQ_ERR_TIMEOUT = 6,           /* reserved: a bounded device wait gave up                        */
    SQ_ERR_OOM = 7,               /* device allocation failed                                       */
    SQ_ERR_STATE = 8,             /* call order: e.g. sq_energy before sq_density                   */
    SQ_ERR_UNSUPPORTED = 9        /* e.g. FD order above 16, or too many atoms touching one cube    */
} sq_status;

/* precision of the Chebyshev recursion (moments, stencil sweeps, projector contractions).
 * Moment sums, Chebyshev weights, the Fermi solve, rho, U, S and forces are always FP64. */
enum { SQ_FP64 = 0, SQ_FP32 = 1 };

/* flags of sq_density.
 * SQ_WANT_FORCE: also accumulate the force moments (Chebyshev path only).
 * SQ_GAUSS: Gauss quadrature (the paper's LSSGQ, Sec. 2.2 "Spectral Gauss quadrature") instead of the
 *   Chebyshev expansion for rho, U and S: per grid point K Lanczos steps (Eq. Lanczos) on the
 *   truncated operator from e_q, the Jacobi matrix's eigenvalues as nodes and squared first
 *   eigenvector components as weights, the Fermi level over all nodes (Eq. Ne), and rho^q, u^q, s^q
 *   (Eqs. rhoq, uq, sq).  K <= 256; not combinable with SQ_WANT_FORCE (the paper takes the force
 *   from the Clenshaw-Curtis path); sq_energy then reports the Gauss U and S.
 * SQ_KB_FMA: FP32 recursion on 29^3 cubes only (the two-CTA cluster kernel): take the projector term
 *   (chi^T v and the rank update) on the CUDA cores instead of the tensor cores.  By default that
 *   kernel runs both as warp-level TF32 MMAs with each operand split into two TF32 parts (three
 *   products, FP32 accumulation), which keep the products to about 2^-21 relative; the flag gives the
 *   plain FP32 FMA form of the same sums, for comparison.  No effect on other kernels. */
enum { SQ_WANT_FORCE = 1, SQ_GAUSS = 2, SQ_KB_FMA = 4 };

/* flags of sq_build_hamiltonian: the gradient of the projectors in the nonlocal force.
 * SQ_GRAD_ANALYTIC: the analytic gradient of chi.
 * SQ_GRAD_FD: the paper's discrete form (Sec. 3 "Atomic forces"), the central finite-difference
 *   gradient nabla_h of the same order as the Laplacian; the paper applies it to the density
 *   matrix columns, f_J = -4 sum_q e_q^T V_J nabla_h(gamma e_q), which on the periodic grid equals
 *   the same contraction with nabla_h chi in place of the analytic gradient (nabla_h^T = -nabla_h). */
enum { SQ_GRAD_ANALYTIC = 0, SQ_GRAD_FD = 1 };

/* Regular periodic grid (Sec. 3 "Discretization"): n_i points on [0, L_i), h_i = L_i / n_i, and the
 * central finite-difference Laplacian of even order fd_order = n_o in {2, 4, ..., 16}. */
typedef struct {
    int n[3];
    double L[3];
    int fd_order;
} sq_grid;

/* Atoms and their Kleinman-Bylander projectors (Sec. 2.1, nonlocal operator
 * V(x,x') = sum_J sum_lm c_Jl chi_Jlm(x) chi_Jlm(x')).  The projector shape is fixed by the library:
 * with w(t) = exp(-t^2/(2 sigma^2)) (1 - t^2/rc^2)^3 for |t| < rc (0 otherwise) and
 * N = (pi sigma^2)^(-3/4),
 *     chi_s(x)   = N prod_i g_i(x_i - R_i),      g(t) = sum over periodic images of w,
 *     chi_p_m(x) = sqrt(2)/sigma (x_m - R_m) chi_s(x)  (periodic-image sum of the same product),
 * i.e. separable windowed Gaussians (a synthetic stand-in for the paper's Troullier-Martins
 * projectors).  lmax = 0 uses chi_s only; lmax = 1 adds p_x, p_y, p_z.  The discrete operator is
 * sum_J sum_lm c_l dV chi chi^T (dV = h1 h2 h3). */
typedef struct {
    int natom;                 /* >= 0 */
    const double *R;           /* host [natom][3], bohr (any real values; wrapped periodically) */
    int lmax;                  /* 0 or 1 */
    double sigma;              /* > 0 */
    double rc;                 /* > 0, window half-width */
    const double *energy;      /* host [lmax+1] KB energies c_l (Ha) */
} sq_atoms;

/*
 * sq_build_hamiltonian -- set up the discrete Kohn-Sham Hamiltonian (Sec. 2.1 Hamiltonian
 * H = -1/2 Lap + V_eff + nonlocal; Sec. 3 "Discretization", "Hamiltonian at each grid point";
 * Sec. 2.2 scale and shift).
 *
 *   grid        periodic grid and FD order (host struct, read during the call)
 *   d_veff      device [N_d] FP64 V_eff, caller-owned; copied into the handle during the call
 *   atoms       atoms and projector parameters (host struct and arrays, read during the call)
 *   R_cut       half-width of the truncation cube (bohr); cube half-widths m_i = round(R_cut/h_i)
 *               (ties to even).  Requires 2 m_i + 1 + fd_order/2 <= n_i on every axis, so that no
 *               two cube points are stencil neighbours through the periodic wrap.
 *   flags       SQ_GRAD_ANALYTIC or SQ_GRAD_FD (gradient used by the force moments)
 *   lambda_min, lambda_max
 *               spectral bounds of H used for the scale and shift omega = (max+min)/2,
 *               tau = (max-min)/2.  Pass NaN for both to let the library compute the rigorous bound
 *               [min V + nl_lo, max kinetic eigenvalue + max V + nl_hi] (Weyl's inequality; the
 *               nonlocal interval from Gershgorin row sums of the weighted projector Gram matrix).
 *               Every truncated H_q is a principal submatrix of H, so the bound holds for all q.
 *   stream      cudaStream_t (void*)
 *   out         receives a new handle on success (free with sq_destroy)
 * Errors: SQ_ERR_ARG, SQ_ERR_CUBE_EXCEEDS_BOX, SQ_ERR_NOT_FINITE, SQ_ERR_UNSUPPORTED, SQ_ERR_OOM,
 * SQ_ERR_CUDA.  Synchronises `stream`.
 */
sq_status sq_build_hamiltonian(const sq_grid *grid, const double *d_veff, const sq_atoms *atoms,
                               double R_cut, int flags, double lambda_min, double lambda_max, void *stream,
                               sq_handle *out);

/*
 * sq_density -- the SQ hot path: per-point Chebyshev recursion (Eq. Chebyshev) of order K on the
 * truncated scaled Hamiltonian, moments mu_k^q (k = 0..K), moment sums M_k = sum_q mu_k^q, the Fermi
 * level (Eq. Ne) by bisection on [lambda_min, lambda_max], the Chebyshev weights c_k of the
 * Fermi-Dirac function (Eq. ChebyshevWeights, M-point Chebyshev-Gauss quadrature with
 * M = 2^ceil(log2 max(4(K+1), 16 tau/kT))), and the density rho(x_q) = 2 sum_k c_k mu_k^q / dV
 * (Eq. rhoq; electrons per bohr^3, so sum_q rho dV = N_e).  With flags & SQ_WANT_FORCE it also
 * accumulates the force moments A_k^{J,lm,d} = sum_q chi_Jlm(x_q) (d_d chi_Jlm)^T v_k^q used by
 * sq_nonlocal_force (Eq. NLforceSQ).
 *
 *   h           handle from sq_build_hamiltonian
 *   K           polynomial order, 1 <= K <= 4096
 *   kT          smearing k_B theta (Ha), > 0
 *   N_e         electron count, 0 < N_e < 2 N_d
 *   precision   SQ_FP64 or SQ_FP32 (recursion precision)
 *   flags       0 or SQ_WANT_FORCE, optionally with SQ_KB_FMA
 *   d_rho       device [N_d] FP64 output, caller-owned
 *   lambda_f    host double output (Fermi level, Ha)
 * Errors: SQ_ERR_ARG, SQ_ERR_NO_BRACKET, SQ_ERR_NOT_FINITE, SQ_ERR_OOM, SQ_ERR_CUDA.
 * Synchronises `stream`.
 */
sq_status sq_density(sq_handle h, int K, double kT, double N_e, int precision, int flags,
                     double *d_rho, double *lambda_f, void *stream);

/*
 * sq_fermi_level -- the Fermi level from moment sums (Eq. Ne, Sec. 3): solve
 *     N(lambda_f) = 2 sum_k c_k(lambda_f) M_k = N_e
 * on the host in FP64, where c_k(lambda_f) are the Chebyshev weights of the Fermi-Dirac function
 * (Eq. ChebyshevWeights, M-point Chebyshev-Gauss quadrature as in sq_density), by bisection on
 * [lambda_min, lambda_max]: mid = lo + (hi - lo)/2, lo = mid if N(mid) < N_e else hi = mid, until the
 * midpoint no longer separates the bracket (at most 200 steps).  A pure function: no handle, no GPU.
 * The paper does this with one global reduction of the moment sums over all processes; a caller that
 * splits the columns (sq_moments_range) sums the M_k itself and solves here.
 *   msum        host [K+1] moment sums M_k = sum_q mu_k^q over all grid points
 *   K           polynomial order, 1 <= K <= 4096
 *   omega, tau  scale and shift of the recursion (omega = (lambda_max+lambda_min)/2 and
 *               tau = (lambda_max-lambda_min)/2 of the bounds the moments were computed with)
 *   lambda_min, lambda_max   bisection bracket (normally the same spectral bounds)
 *   kT, N_e     smearing (Ha, > 0) and electron count (> 0)
 *   lambda_f    host output
 * Errors: SQ_ERR_ARG, SQ_ERR_NOT_FINITE (a moment sum), SQ_ERR_NO_BRACKET (N(lambda_min) > N_e or
 * N(lambda_max) < N_e), SQ_ERR_UNSUPPORTED (kT/tau needs more than 2^26 nodes).
 */
sq_status sq_fermi_level(const double *msum, int K, double omega, double tau, double lambda_min,
                         double lambda_max, double kT, double N_e, double *lambda_f);

/*
 * sq_fermi_weights -- the Chebyshev weights at a given Fermi level (Eq. ChebyshevWeights, FP64, host):
 * c_k of g(lam) (Eq. FermiDirac), d_k of lam g(lam) and e_k of s(g(lam)), k = 0..K, each a_k =
 * (2 - delta_k0)/M sum_j f(lam_j) cos(k theta_j) over the M Chebyshev-Gauss nodes of sq_density.
 * Then rho^q = 2 sum_k c_k mu_k^q, U = 2 sum_k d_k M_k and S = -2 sum_k e_k M_k (Eqs. rhoq, uq, sq).
 * Outputs are host [K+1] arrays; any may be NULL.  Errors: SQ_ERR_ARG, SQ_ERR_UNSUPPORTED.
 */
sq_status sq_fermi_weights(double lambda_f, int K, double omega, double tau, double kT, double *c, double *d,
                           double *e);

/*
 * sq_gauss_rule -- the Gauss rule of one grid point from its Lanczos coefficients (Sec. 2.2; host,
 * FP64, pure): the nodes are the eigenvalues of the Jacobi matrix tridiag(b_1..b_{K-1}; a_1..a_K;
 * b_1..b_{K-1}) mapped back to energies (lambda = tau lambda_hat + omega when a, b are those of the
 * scaled operator (H - omega)/tau; pass omega = 0, tau = 1 for unscaled coefficients), the weights
 * the squared first components of its normalised eigenvectors.  The matrix is cut at the first
 * b_k = 0 (k < K); the nodes past the cut get weight 0.  The same routine runs per column on the GPU
 * under SQ_GAUSS.
 *   a, b        host [K] coefficients a_1..a_K, b_1..b_K (b_K unused)
 *   nodes, weights  host [K] outputs
 * Errors: SQ_ERR_ARG (K outside 1..256, bad scale), SQ_ERR_NOT_FINITE (non-finite input, or the
 * eigensolve did not converge).
 */
sq_status sq_gauss_rule(const double *a, const double *b, int K, double omega, double tau, double *nodes,
                        double *weights);

/*
 * sq_fermi_resolve -- re-solve the electron-count equation (Eq. Ne) for a new kT / N_e from the
 * moment sums stored by the last whole-grid sq_density, on the device, and refresh the stored weights;
 * d_rho (may be NULL) receives the matching density.  Same bisection rule as sq_density.
 * Errors: SQ_ERR_STATE (no whole-grid sq_density yet), SQ_ERR_ARG, SQ_ERR_NO_BRACKET, SQ_ERR_CUDA.
 * Synchronises `stream`.
 */
sq_status sq_fermi_resolve(sq_handle h, double kT, double N_e, double *d_rho, double *lambda_f, void *stream);

/*
 * Column-range (sharded) form of sq_density.  The columns of the grid are independent given V_eff
 * (Sec. 3 "Hamiltonian at each grid point": each point's cube needs only V_eff around it), and the
 * Fermi level couples them through one global sum of moments (Eq. Ne).  A caller that splits the
 * grid over processes or GPUs runs, per shard:
 *     sq_moments_range  -> partial sums M_k (and force moments A) of its columns
 *     (caller)          -> sum M_k and A over the shards (e.g. one allreduce)
 *     sq_fermi_level    -> lambda_f (host, pure)
 *     sq_observables    -> rho of its columns; then sq_energy and sq_nonlocal_force as usual.
 *
 * sq_moments_range -- the recursion (Eq. Chebyshev) for the columns q in [q_begin, q_end) only.
 *   K, precision, flags   as sq_density (flags: 0 or SQ_WANT_FORCE, optionally with SQ_KB_FMA)
 *   q_begin, q_end        0 <= q_begin < q_end <= N_d
 *   msum        host [K+1] output: M_k summed over the range's columns (FP64)
 *   A           host [K+1][natom][nproj][3] output of the range's force moments
 *               (required with SQ_WANT_FORCE, else ignored)
 * Errors: SQ_ERR_ARG, SQ_ERR_NOT_FINITE, SQ_ERR_OOM, SQ_ERR_UNSUPPORTED, SQ_ERR_CUDA.  Synchronises
 * `stream`.
 *
 * sq_observables -- after sq_moments_range, take the global sums and the Fermi level: stores msum
 * (host [K+1] total M_k) and A (host total force moments, or NULL to skip forces), forms the weights
 * at lambda_f (as sq_fermi_weights) and writes d_rho (device [q_end - q_begin] FP64, the density of
 * the range's columns, rho(x_q) = 2 sum_k c_k mu_k^q / dV; may be NULL).  Afterwards sq_energy
 * reports U, S, F from the total sums, and sq_nonlocal_force the forces from the total A.
 * Errors: SQ_ERR_STATE (no sq_moments_range), SQ_ERR_ARG, SQ_ERR_NOT_FINITE, SQ_ERR_CUDA.
 * Synchronises `stream`.
 */
sq_status sq_moments_range(sq_handle h, int K, int precision, int flags, long long q_begin, long long q_end,
                           double *msum, double *A, void *stream);

/*
 * sq_moments_cols -- the recursion (Eq. Chebyshev) for a list of columns: the moments mu_k^q of the
 * grid points d_cols[0..ncols), written compactly to d_mu_out [K+1][ncols] (recursion precision, 8 or
 * 4 bytes per value, caller-owned device buffer).  For callers that need a few columns, e.g. the
 * columns whose cubes contain one grid point (those are the only ones a change of V_eff there can
 * move).  Runs the generic column kernel; no sums, no Fermi level; leaves the handle without a
 * density.  Indices must be distinct and in [0, N_d) (checked on the device before use).
 * Errors: SQ_ERR_ARG, SQ_ERR_OOM, SQ_ERR_UNSUPPORTED, SQ_ERR_CUDA.  Synchronises `stream`.
 */
sq_status sq_moments_cols(sq_handle h, int K, int precision, const long long *d_cols, long long ncols,
                          void *d_mu_out, void *stream);
sq_status sq_observables(sq_handle h, double lambda_f, double kT, double N_e, const double *msum, const double *A,
                         double *d_rho, void *stream);

/*
 * sq_energy -- band energy U = 2 Tr(gamma H) = 2 sum_k d_k M_k (d_k: Chebyshev weights of lam g),
 * entropy S = -2 Tr s(H) = -2 sum_k e_k M_k (units of k_B, S >= 0; s = g ln g + (1-g) ln(1-g),
 * Eq. FermiDirac and Eqs. uq, sq) and the band free energy F = U - kT S, at the Fermi level of the
 * last sq_density / sq_fermi_level.  Host outputs (any may be NULL).
 * Errors: SQ_ERR_STATE, SQ_ERR_CUDA.  Synchronises `stream`.
 */
sq_status sq_energy(sq_handle h, double *U, double *S, double *F, void *stream);

/*
 * sq_nonlocal_force -- nonlocal atomic forces f_J,d = 4 dV sum_lm c_l sum_k c_k A_k^{J,lm,d}
 * (Eq. AtomicForce nonlocal term, Eq. NLforceSQ): the physical force -dF/dR_J of the KB energy,
 * with the analytic gradient of the projectors.  Requires the last sq_density to have been called
 * with SQ_WANT_FORCE.
 *   d_force     device [natom][3] FP64 output, caller-owned
 * Errors: SQ_ERR_STATE, SQ_ERR_ARG, SQ_ERR_CUDA.  Asynchronous on `stream`.
 */
sq_status sq_nonlocal_force(sq_handle h, double *d_force, void *stream);

/* Spectral bounds in use (host outputs). */
sq_status sq_get_spectral_bounds(sq_handle h, double *lambda_min, double *lambda_max);

/*
 * Read-only views of the last sq_density's results (library-owned, valid until the next
 * sq_density or sq_destroy): d_mu is [K+1][N_d] in the recursion precision (float or double,
 * see *precision), d_msum is [K+1] FP64 moment sums M_k.  Any output pointer may be NULL.
 */
sq_status sq_get_moments(sq_handle h, int *K, int *precision, const void **d_mu,
                         const double **d_msum);

/*
 * sq_copy_moments -- copy the last sq_density's moments into caller-owned device buffers:
 * d_mu [K+1][N_d] in the recursion precision (8 or 4 bytes per value) and d_msum [K+1] FP64.
 * Either may be NULL.  Asynchronous on `stream`.
 * Errors: SQ_ERR_STATE, SQ_ERR_CUDA.
 */
sq_status sq_copy_moments(sq_handle h, void *d_mu, double *d_msum, void *stream);

/* Cube geometry in use: half-widths m[3] (grid points). */
sq_status sq_get_cube(sq_handle h, int m[3]);

/*
 * sq_get_timing -- device time of the last sq_density's kernels, measured with CUDA events recorded
 * on the caller's stream around them: the per-column recursion kernel alone, the moment sums, and
 * the Fermi solve with weights and density (milliseconds; any output may be NULL).
 */
sq_status sq_get_timing(sq_handle h, double *recursion_ms, double *msum_ms, double *fermi_ms);

/* Name of the recursion kernel the last sq_density ran (static string; "" before the first call). */
const char *sq_kernel_name(sq_handle h);

/* Total number of kernels this library has launched in this process (for launch accounting). */
long long sq_kernel_launches(void);

/*
 * sq_fma_throughput -- measured fused-multiply-add ceiling of the current GPU in the given precision
 * (SQ_FP32 or SQ_FP64): a probe kernel of independent FMA chains at full occupancy on every SM, timed
 * with CUDA events on `stream` (about 100 ms).  The recursion kernels are bound by these pipes, so
 * this is the denominator of their roofline fraction.  Outputs: TFLOP/s (2 FLOP per FMA) and the
 * timed launch's milliseconds (either may be NULL).  Errors: SQ_ERR_ARG, SQ_ERR_CUDA.
 */
sq_status sq_fma_throughput(int precision, double *tflops, double *ms, void *stream);

/*
 * sq_mma_throughput -- measured throughput of the warp-level tensor-core instruction (mma.sync) the
 * per-warp contractions of the projector term could use instead of FMAs: kind 0 TF32 m16n8k8, kind 1
 * BF16 m16n8k16, FP32 accumulation; 8 independent accumulator tiles per warp at full occupancy,
 * timed with CUDA events on `stream` (about 100 ms).  Outputs: TFLOP/s and the timed launch's
 * milliseconds (either may be NULL).  Errors: SQ_ERR_ARG, SQ_ERR_CUDA.
 */
sq_status sq_mma_throughput(int kind, double *tflops, double *ms, void *stream);

/*
 * sq_moments_noalloc -- the Chebyshev moments mu_k^q (k = 0..K, every grid point) of the handle's
 * Hamiltonian, computed without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot let the library allocate once their steady state has begun
 * (a fixed device-memory budget handed out up front, a latency-critical loop where cudaMalloc and
 * cudaFree would synchronise the device, or a GPU shared with other work whose footprint must not
 * grow).  Set-up calls such as sq_build_hamiltonian still allocate; this call does not.
 *
 * It runs the same recursion kernel as sq_density (without force moments), but keeps the kernel's
 * per-CTA cube vectors and the padded diagonal in one fixed 32 MiB device array that the library
 * defines at file scope.  Every GPU that loads the library holds that array until the process
 * exits, and all calls share it:
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 *     caches it; make that first call before any stream capture;
 *   - nothing in the array has to start at zero: each call rewrites every byte it reads, so it
 *     does not depend on what an earlier call left there;
 *   - calls whose kernels overlap on the GPU (other streams, other host threads) race on the array
 *     and give wrong results; serialise them.
 * Fewer CTAs run at once than in sq_density when a cube's two vectors are large, so it is slower.
 *
 *   h           handle from sq_build_hamiltonian, created on the current device
 *   K           polynomial order, 1 <= K <= 4096
 *   precision   SQ_FP64 or SQ_FP32
 *   d_mu        device [K+1][N_d] output in the chosen precision (8 or 4 bytes per value),
 *               caller-owned; the same values sq_density computes
 * Errors: SQ_ERR_ARG; SQ_ERR_UNSUPPORTED when the padded diagonal plus one cube's two vectors do not
 * fit in the 32 MiB array (or the device ordinal is >= 64); SQ_ERR_CUDA.  Asynchronous on `stream`;
 * calls no allocating routine.
 */
sq_status sq_moments_noalloc(sq_handle h, int K, int precision, void *d_mu, void *stream);

/*
 * sq_density_vjp -- vector-Jacobian product of the last sq_density: for the scalar
 * L = sum_q rho_bar(x_q) rho(x_q) + U_bar U, writes d_veff_bar(x) = dL/dV_eff(x) on every grid point.
 * The derivative includes the implicit change of the Fermi level (N(lambda_f) = N_e, Eq. Ne) and holds
 * the scale and shift omega, tau fixed.  It runs the reverse (adjoint) Chebyshev recursion of every
 * column -- a_K = mubar_K e_q, a_k = 2 Hhat_q a_{k+1} - a_{k+2} + mubar_k e_q (reverse Clenshaw) --
 * with the forward vectors stored as checkpoint pairs every checkpoint_k steps and recomputed segment
 * by segment (Eq. Chebyshev run backwards; the paper needs this derivative only implicitly, through
 * the SCF mixing of V_eff, Sec. 3).  Same recursion precision as the last sq_density; in SQ_FP32 on
 * cubic 21^3 / 25^3 cubes with the 12th-order stencil it runs on the FP32 slab kernel's mapping.
 *   d_rho_bar    device [N_d] FP64 cotangent of rho (per bohr^3 density, as returned by sq_density)
 *   U_bar        cotangent of the band energy U
 *   checkpoint_k 1 <= checkpoint_k <= K (1: every vector kept; larger: less memory, more recompute)
 *   d_veff_bar   device [N_d] FP64 output (overwritten)
 * Column contributions are summed with FP64 atomics, so results may differ in the last bits between
 * runs.  Errors: SQ_ERR_STATE (no sq_density), SQ_ERR_ARG, SQ_ERR_OOM, SQ_ERR_UNSUPPORTED (a cube
 * holds more atoms than shared memory allows), SQ_ERR_CUDA.  Synchronises `stream`.
 */
sq_status sq_density_vjp(sq_handle h, const double *d_rho_bar, double U_bar, int checkpoint_k,
                         double *d_veff_bar, void *stream);

/*
 * Batched evaluation of many independent cells (the paper's method applied to a set of defect cells,
 * Sec. 3 per cell): every cell's per-point recursion runs in ONE persistent kernel launch whose CTAs
 * take (cell, column-range) work items from a queue, followed by each cell's moment sums, Fermi
 * level, weights and density -- the whole sequence captured once into a CUDA graph and replayed.
 * In SQ_FP32, cells with cubic 21^3, 25^3 or 29^3 cubes and the 12th-order stencil leave the queue and
 * run as one launch each of the kernel sq_density uses for them (the FP32 slab kernel for 21^3 and
 * 25^3, the two-CTA cluster kernel for 29^3), captured in the same graph.
 *
 * sq_batch_create -- group built handles (cells may differ in grid, cube, atoms, K, kT, N_e; they must
 * share the FD order and the device).  Allocates every buffer the graph will use.
 *   cells[ncells]   handles from sq_build_hamiltonian (owned by the caller; keep them alive)
 *   K, kT, N_e      host [ncells] per-cell polynomial order, smearing and electron count
 *   precision       SQ_FP64 or SQ_FP32;  flags: 0 or SQ_WANT_FORCE, optionally with SQ_KB_FMA (as
 *                   sq_density; a 29^3 cell whose atom lists exceed the tensor-core path then needs it)
 * Errors: SQ_ERR_ARG, SQ_ERR_UNSUPPORTED, SQ_ERR_OOM, SQ_ERR_CUDA.
 */
typedef struct sq_batch_s *sq_batch;
sq_status sq_batch_create(const sq_handle *cells, int ncells, const int *K, const double *kT, const double *N_e,
                          int precision, int flags, sq_batch *out);

/*
 * sq_batch_density -- run the batch.  The first call autotunes the recursion launch of the work queue
 * (vectors in shared memory with 512 or 256 threads, or in global scratch; work items of 32 or 128
 * columns), timed on a prefix of the queue (256 columns per SM; skipped when every cell has its own
 * launch), then captures the graph; later calls with the same d_rho pointers replay it (new pointers
 * trigger a new capture).  The Fermi level of each cell is solved inside the graph by a fixed number
 * of bisection launches (2 bracket checks and 94 halvings, enough to reach the last bit of any
 * bracket within the spectral bounds' range of 2^94 ulps); a cell whose bisection has not closed by
 * then is re-solved on the host-driven path of sq_density after the replay.  Afterwards each handle
 * holds its cell's results as after sq_density, so sq_energy and sq_nonlocal_force apply per cell.
 *   d_rho[ncells]   device FP64 density outputs, one per cell (caller-owned)
 *   lambda_f        host [ncells] Fermi levels (may be NULL)
 * Errors: SQ_ERR_ARG, SQ_ERR_NO_BRACKET, SQ_ERR_NOT_FINITE, SQ_ERR_UNSUPPORTED, SQ_ERR_CUDA.
 * Synchronises `stream`.
 */
sq_status sq_batch_density(sq_batch b, double *const *d_rho, double *lambda_f, void *stream);

/* Tuning and graph facts of a batch: chosen configuration (0: shared-memory vectors with 512
 * threads, 1: with 256 threads, 2: global-scratch vectors), columns per work item, CTAs in the
 * persistent launch, tuned probe time (ms) and number of graph nodes.  Any output may be NULL. */
sq_status sq_batch_info(sq_batch b, int *config, int *chunk, int *grid, double *tuned_ms, long long *graph_nodes);

/* Release a batch (NULL is ignored; the cell handles are not touched). */
void sq_batch_destroy(sq_batch b);

/*
 * Self-consistency pieces around the density (Sec. 2.1: LDA exchange-correlation, Eq. Poisson;
 * Sec. 3 "Electrostatic and effective potential": V_eff^q = V_xc(rho^q) + phi^q).  All FP64 device
 * arrays of one periodic grid [n3][n2][n1] (x fastest), caller-owned; each call synchronises `stream`.
 *
 * sq_lda_pw92 -- local exchange-correlation energy per electron eps_xc(rho) and potential
 *   V_xc = d(rho eps_xc)/d rho: Slater exchange and the spin-unpolarised Perdew-Wang correlation
 *   (published fit, p = 1); zero where rho <= 0.  n >= 1 points.  Errors: SQ_ERR_ARG, SQ_ERR_CUDA.
 *
 * sq_pseudocharge -- total pseudocharge of the nuclei on the grid of `box` (bohr) with n points per
 *   axis: b(x) = sum_J -Z_J (2 pi sigma_b^2)^(-3/2) exp(-|x - R_J|^2 / (2 sigma_b^2)), minimum-image
 *   distances (valid for boxes at least 12 sigma_b wide).  R: host [natom][3] bohr, Z: host [natom]
 *   valence charges; natom >= 0.  Errors: SQ_ERR_ARG, SQ_ERR_NOT_FINITE, SQ_ERR_OOM, SQ_ERR_CUDA.
 *
 * sq_poisson_periodic -- phi with -(1/4 pi) L_h phi = f - mean(f) and mean(phi) = 0, L_h the periodic
 *   finite-difference Laplacian of order fd_order (the kinetic term's stencil), by conjugate
 *   gradients on -L_h until the residual is tol times that of phi = 0 (at most max_iter iterations).
 *   The mean of f (a periodic cell's net charge) is removed: the periodic problem has no solution
 *   otherwise.  Outputs the iteration count and the final relative residual.  Errors: SQ_ERR_ARG,
 *   SQ_ERR_NOT_FINITE, SQ_ERR_TIMEOUT (not converged; phi holds the last iterate), SQ_ERR_OOM,
 *   SQ_ERR_CUDA.  Allocates and frees its own work space (3 N + 256 doubles).
 *
 * sq_effective_potential -- the step from a density to the next effective potential: phi of
 *   rho + b (as sq_poisson_periodic), eps_xc and V_xc of rho (as sq_lda_pw92) and V_eff = V_xc + phi.
 *   Errors as sq_poisson_periodic.
 */
sq_status sq_lda_pw92(long long n, const double *d_rho, double *d_exc, double *d_vxc, void *stream);
sq_status sq_pseudocharge(const int n[3], const double box[3], int natom, const double *R, const double *Z,
                          double sigma_b, double *d_b, void *stream);
sq_status sq_poisson_periodic(const int n[3], const double box[3], int fd_order, const double *d_f, double tol,
                              int max_iter, double *d_phi, int *iters, double *rel_res, void *stream);
sq_status sq_effective_potential(const int n[3], const double box[3], int fd_order, const double *d_rho,
                                 const double *d_b, double tol, int max_iter, double *d_phi, double *d_exc,
                                 double *d_vxc, double *d_veff, int *iters, double *rel_res, void *stream);

/*
 * Anderson mixing of the effective potential between SCF iterations (Sec. 3: the SCF iteration mixes
 * V_eff and stops on the normalised error of V_eff).  A mixer holds, on the device, the previous
 * input potential and residual and the differences of the last `history` steps.
 *
 * sq_mixer_create -- n grid points, history 0..32 (0: linear mixing), 0 < beta <= 1.  Allocates
 *   (3 + 2 history) n + 256 doubles.  Errors: SQ_ERR_ARG, SQ_ERR_OOM.
 * sq_mixer_step -- with F = V_out - V_in: rel_err = |F| / |V_out|; gamma minimises
 *   |F - sum_j gamma_j dF_j| over the held differences (dV_j, dF_j) of V_in and F (normal equations,
 *   regularised by 1e-12 of their mean diagonal); V_next = V_in + beta F - sum_j gamma_j (dV_j + beta dF_j).
 *   d_vin, d_vout: device [n] inputs; d_vnext: device [n] output (may be d_vin).  Synchronises
 *   `stream`.  Errors: SQ_ERR_ARG, SQ_ERR_NOT_FINITE, SQ_ERR_CUDA.
 * sq_mixer_destroy -- release (NULL is ignored).
 */
typedef struct sq_mixer_s *sq_mixer;
sq_status sq_mixer_create(long long n, int history, double beta, sq_mixer *out);
sq_status sq_mixer_step(sq_mixer m, const double *d_vin, const double *d_vout, double *d_vnext, double *rel_err,
                        void *stream);
void sq_mixer_destroy(sq_mixer m);

/*
 * Discrete free energy and local force (Sec. 3 "Free energy", "Atomic forces"), FP64 on the grid of
 * the self-consistency calls above; host outputs; each call synchronises `stream`.
 *
 * sq_self_energy -- E_self^h = -(1/2) h1 h2 h3 sum_q sum_I b_I^q V_I^q (Eq. DiscreteSelfEnergy) for the
 *   Gaussian pseudocharges of sq_pseudocharge, V_I = -Z_I erf(r / (sqrt(2) sigma_b)) / r their
 *   free-space potentials (minimum image).  Errors: SQ_ERR_ARG, SQ_ERR_NOT_FINITE, SQ_ERR_OOM, SQ_ERR_CUDA.
 * sq_free_energy -- F^h = F_band + h1 h2 h3 sum_q [(eps_xc - V_xc) rho + (1/2)(b - rho) phi] + E_self
 *   (Eq. DiscreteEnergy), with F_band = U - kT S of sq_energy (its sum over q of u^q - 2 theta s^q),
 *   phi, eps_xc, V_xc of rho from sq_effective_potential and E_self from sq_self_energy.
 *   Errors: SQ_ERR_ARG, SQ_ERR_NOT_FINITE, SQ_ERR_OOM, SQ_ERR_CUDA.
 * sq_local_force -- f_J = h1 h2 h3 sum_q (nabla_h b_J)^q phi^q (Eq. DiscreteLocalForce), nabla_h the
 *   central first difference of order fd_order, evaluated as -h1 h2 h3 sum_q b_J^q (nabla_h phi)^q
 *   (the same sum on the periodic grid).  force: host [natom][3] output (Ha/bohr).  Errors as above.
 */
sq_status sq_self_energy(const int n[3], const double box[3], int natom, const double *R, const double *Z,
                         double sigma_b, double *E_self, void *stream);
sq_status sq_free_energy(const int n[3], const double box[3], const double *d_rho, const double *d_b,
                         const double *d_phi, const double *d_exc, const double *d_vxc, double F_band, double E_self,
                         double *F, void *stream);
sq_status sq_local_force(const int n[3], const double box[3], int fd_order, int natom, const double *R, const double *Z,
                         double sigma_b, const double *d_phi, double *force, void *stream);

/* Release a handle and its device workspace (NULL is ignored).  Synchronises the device. */
void sq_destroy(sq_handle h);

/* Static description of a status code. */
const char *sq_status_string(sq_status s);

/* Message of the last failing call on this host thread ("" if none). */
const char *sq_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SQ_H */
