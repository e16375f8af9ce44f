/*
 * sq_oracle.c -- plain, slow, FP64 CPU oracle of the Clenshaw-Curtis spectral-quadrature (SQ)
 * recursion.  TEST INFRASTRUCTURE ONLY: it exists so the CUDA library can be checked against an
 * independent implementation.  Only tests/, the package smoke check and bench.py's CPU-baseline
 * leg may load it; the product path never does.  It shares no code, header or table with the
 * CUDA library.
 *
 * What it computes (paper: Ghosh & Bhattacharya, "Spectral quadrature for the first principles
 * study of crystal defects: Application to magnesium", arXiv 2011.13517):
 *
 *  - the Kohn-Sham Hamiltonian H = -1/2 Lap_h + V_eff + sum_J sum_lm c_Jl dV chi_Jlm chi_Jlm^T
 *    on a regular periodic grid (Sec. 2.1 Hamiltonian and nonlocal operator; Sec. 3
 *    "Discretization", "Hamiltonian at each grid point"), with the central finite-difference
 *    Laplacian of even order n_o;
 *  - its restriction H_q to the cube of half-width m_i = round(R_cut/h_i) around grid point q
 *    ("region of influence", Sec. 3), with zero values outside the cube;
 *  - the scaled operator Hhat = (H - omega)/tau (Sec. 2.2, scale and shift);
 *  - the Chebyshev three-term recursion v_0 = e_q, v_1 = Hhat v_0, v_{k+1} = 2 Hhat v_k - v_{k-1}
 *    (Eq. Chebyshev, Sec. 2.2), its moments mu_k^q = v_k(q);
 *  - the nonlocal-force moments A_k^{J,lm,d} = sum_q chi_Jlm(x_q) sum_x d_d chi_Jlm(x) v_k^q(x)
 *    (Eq. NLforceSQ and the discrete nonlocal force of Sec. 3 "Atomic forces");
 *  - the Lanczos coefficients a_k, b_k of the same truncated operator started from e_q (Eq. Lanczos,
 *    Sec. 2.2), whose Jacobi matrices give the Gauss quadrature nodes and weights (oracle.py).
 *
 * Readings where the paper is silent or ambiguous:
 *  - the recursion starts from the Euclidean unit vector e_q, so mu_0 = 1;
 *  - the discrete KB term carries dV, because chi^T v approximates the integral of chi f;
 *  - projectors are separable windowed Gaussians (below), summed over periodic images;
 *  - the gradient in the force is the analytic gradient of chi; with grad_fd set it is instead
 *    the central finite-difference gradient D_h chi of the same order n_o as the Laplacian, the
 *    discrete form of Sec. 3 "Atomic forces" (the paper applies nabla_h to gamma e_q; on the
 *    periodic grid chi^T D_h v = -(D_h chi)^T v, so the force keeps its form with D_h chi in place
 *    of the analytic gradient).
 *
 * Projectors.  With w(t) = exp(-t^2/(2 sigma^2)) (1 - t^2/rc^2)^3 for |t| < rc (0 otherwise),
 *   chi_s(x)   = N gx(x1-R1) gy(x2-R2) gz(x3-R3),          N = (pi sigma^2)^(-3/4),
 *   chi_p_m(x) = sqrt(2)/sigma (x_m - R_m) chi_s(x)        (m = x, y, z),
 * where g(t) = sum_images w(t - n L) and the p factor hp(t) = sum_images sqrt(2)/sigma (t-nL) w(t-nL).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n[3];              /* grid points per axis */
    double L[3];           /* periodic box (bohr) */
    int fd_order;          /* even FD order n_o */
    const double *veff;    /* [n3][n2][n1], x fastest */
    int natom;
    const double *R;       /* [natom][3] */
    int lmax;              /* 0: s only, 1: s + p */
    double sigma, rc;      /* projector width and window half-width */
    const double *cl;      /* [lmax+1] KB energies */
    int m[3];              /* cube half-widths (grid points) */
    int full;              /* 1: no truncation, the "cube" is the whole periodic box */
    int grad_fd;           /* 1: force moments with the FD gradient D_h chi instead of the analytic one */
} sq_oracle_problem;

enum { F_G = 0, F_HP = 1, F_GD = 2, F_HD = 3, NFACT = 4 };

/* Central second-derivative weights c_0..c_p of order n_o = 2p:
 *   c_j = 2 (-1)^(j+1) (p!)^2 / (j^2 (p-j)! (p+j)!),  c_0 = -2 sum_{j>=1} c_j.
 * (Textbook Fornberg weights; Sec. 3 "Discretization" uses an FD Laplacian of unstated order.) */
int sq_oracle_fd_coeffs(int order, double *c)
{
    if (order < 2 || order % 2 || order > 32) return -1;
    int p = order / 2;
    double sum = 0.0;
    for (int j = 1; j <= p; j++) {
        double num = 2.0 * ((j % 2) ? 1.0 : -1.0);
        /* (p!)^2 / ((p-j)! (p+j)!) = prod_{i=1..j} (p-j+i)/(p+i) */
        double r = 1.0;
        for (int i = 1; i <= j; i++) r *= (double)(p - j + i) / (double)(p + i);
        c[j] = num * r / ((double)j * (double)j);
        sum += c[j];
    }
    c[0] = -2.0 * sum;
    return p;
}

/* Central first-derivative weights a_1..a_p of order n_o = 2p (df/dx ~ sum_j a_j (f_{+j} - f_{-j})/h):
 *   a_j = (-1)^(j+1) (p!)^2 / (j (p-j)! (p+j)!).
 * (Textbook Fornberg weights, the first-derivative companion of the Laplacian's.) */
int sq_oracle_fd1_coeffs(int order, double *a)
{
    if (order < 2 || order % 2 || order > 32) return -1;
    int p = order / 2;
    a[0] = 0.0;
    for (int j = 1; j <= p; j++) {
        double r = 1.0;
        for (int i = 1; i <= j; i++) r *= (double)(p - j + i) / (double)(p + i);
        a[j] = ((j % 2) ? 1.0 : -1.0) * r / (double)j;
    }
    return p;
}

/* One-dimensional periodized projector factors on the n_a grid points of one axis. */
void sq_oracle_axis_factors(double R_a, double L_a, int n_a, double sigma, double rc,
                            double *g, double *hp, double *gd, double *hd)
{
    const double h = L_a / n_a;
    const double pf = sqrt(2.0) / sigma;
    for (int i = 0; i < n_a; i++) {
        double x = i * h;
        double sg = 0.0, sh = 0.0, sgd = 0.0, shd = 0.0;
        int lo = (int)floor((x - R_a - rc) / L_a) - 1;
        int hi = (int)ceil((x - R_a + rc) / L_a) + 1;
        for (int im = lo; im <= hi; im++) {
            double t = x - R_a - im * L_a;
            if (fabs(t) >= rc) continue;
            double u = 1.0 - t * t / (rc * rc);
            double e = exp(-t * t / (2.0 * sigma * sigma));
            double w = e * u * u * u;
            /* dw/dt = e * [ -t/sigma^2 u^3 + 3 u^2 (-2 t / rc^2) ] */
            double wd = e * (-t / (sigma * sigma) * u * u * u - 6.0 * t / (rc * rc) * u * u);
            sg += w;
            sgd += wd;
            sh += pf * t * w;
            shd += pf * (w + t * wd);
        }
        g[i] = sg;
        hp[i] = sh;
        gd[i] = sgd;
        hd[i] = shd;
    }
}

/* ---------------------------------------------------------------------------------------- */

typedef struct {
    const sq_oracle_problem *P;
    int nc[3];             /* cube extent per axis */
    long nc3;
    int p;                 /* stencil half-width */
    double w[3][17];       /* off-diagonal kinetic weights -c_j/(2 h_i^2) */
    double kdiag;          /* sum_i -c_0/(2 h_i^2) */
    double dV;
    int nproj;             /* 1 or 4 projectors per atom */
    double N;              /* Gaussian normalisation */
    double *fac;           /* [natom][3][NFACT][n_axis] full-axis factor tables */
    int fac_off[3];        /* offset of axis a inside one atom's block */
    int fac_stride;        /* doubles per atom */
    /* nbr[a][i*(2p)+2(j-1)+{0,1}]: local index of the +j / -j neighbour of local index i along
     * axis a, or -1 when that grid point lies outside the cube */
    int *nbr[3];
} oracle_ctx;

static int ctx_init(oracle_ctx *C, const sq_oracle_problem *P)
{
    memset(C, 0, sizeof(*C));
    C->P = P;
    double c[17];
    int p = sq_oracle_fd_coeffs(P->fd_order, c);
    if (p < 0) return -1;
    C->p = p;
    C->kdiag = 0.0;
    for (int a = 0; a < 3; a++) {
        double h = P->L[a] / P->n[a];
        for (int j = 1; j <= p; j++) C->w[a][j] = -c[j] / (2.0 * h * h);
        C->kdiag += -c[0] / (2.0 * h * h);
        if (P->full) {
            C->nc[a] = P->n[a];
        } else {
            C->nc[a] = 2 * P->m[a] + 1;
            if (C->nc[a] > P->n[a]) return -2;
        }
    }
    C->nc3 = (long)C->nc[0] * C->nc[1] * C->nc[2];
    /* The cube operator is the principal submatrix P_q H P_q of the periodic H: the neighbour at
     * local offset i +- j is the global point (q - m + i +- j) mod n, whose local index is
     * (i +- j) mod n; it belongs to the cube iff that index is < n_c.  With n_c = n (no
     * truncation) this is the plain periodic stencil. */
    for (int a = 0; a < 3; a++) {
        int nb = P->n[a], ncl = C->nc[a];
        C->nbr[a] = (int *)malloc(sizeof(int) * (size_t)ncl * 2 * p);
        if (!C->nbr[a]) return -3;
        for (int i = 0; i < ncl; i++)
            for (int j = 1; j <= p; j++) {
                int lp = (i + j) % nb;
                int lm = ((i - j) % nb + nb) % nb;
                C->nbr[a][i * 2 * p + 2 * (j - 1)] = lp < ncl ? lp : -1;
                C->nbr[a][i * 2 * p + 2 * (j - 1) + 1] = lm < ncl ? lm : -1;
            }
    }
    C->dV = (P->L[0] / P->n[0]) * (P->L[1] / P->n[1]) * (P->L[2] / P->n[2]);
    C->nproj = P->lmax == 0 ? 1 : 4;
    C->N = pow(M_PI * P->sigma * P->sigma, -0.75);
    C->fac_off[0] = 0;
    C->fac_off[1] = NFACT * P->n[0];
    C->fac_off[2] = NFACT * (P->n[0] + P->n[1]);
    C->fac_stride = NFACT * (P->n[0] + P->n[1] + P->n[2]);
    C->fac = (double *)malloc(sizeof(double) * (size_t)C->fac_stride * (P->natom > 0 ? P->natom : 1));
    if (!C->fac) return -3;
    for (int J = 0; J < P->natom; J++) {
        for (int a = 0; a < 3; a++) {
            double *base = C->fac + (size_t)J * C->fac_stride + C->fac_off[a];
            int na = P->n[a];
            sq_oracle_axis_factors(P->R[3 * J + a], P->L[a], na, P->sigma, P->rc,
                                   base + F_G * na, base + F_HP * na, base + F_GD * na,
                                   base + F_HD * na);
            if (P->grad_fd) {
                /* D_h of the separable factors: chi's FD gradient along axis a differentiates only
                 * its axis-a factor, periodically on the n_a points */
                double a1[17];
                int p1 = sq_oracle_fd1_coeffs(P->fd_order, a1);
                double h = P->L[a] / na;
                for (int i = 0; i < na; i++) {
                    double sg = 0.0, sh = 0.0;
                    for (int j = 1; j <= p1; j++) {
                        int ip = (i + j) % na, im = ((i - j) % na + na) % na;
                        sg += a1[j] * (base[F_G * na + ip] - base[F_G * na + im]);
                        sh += a1[j] * (base[F_HP * na + ip] - base[F_HP * na + im]);
                    }
                    base[F_GD * na + i] = sg / h;
                    base[F_HD * na + i] = sh / h;
                }
            }
        }
    }
    return 0;
}

static void ctx_free(oracle_ctx *C)
{
    free(C->fac);
    for (int a = 0; a < 3; a++) free(C->nbr[a]);
}

static inline const double *factor(const oracle_ctx *C, int J, int a, int which)
{
    return C->fac + (size_t)J * C->fac_stride + C->fac_off[a] + which * C->P->n[a];
}

/* Factor type per axis for projector lm (0 = s, 1..3 = p_x..p_z), optionally differentiated
 * along axis d (d < 0: no derivative). */
static void proj_factor_types(int lm, int d, int type[3])
{
    for (int a = 0; a < 3; a++) type[a] = (lm == 1 + a) ? F_HP : F_G;
    if (d >= 0) type[d] = (type[d] == F_HP) ? F_HD : F_GD;
}

/* Global grid index along axis a of local cube index i for column centre qa. */
static inline int glob(const oracle_ctx *C, int a, int qa, int i)
{
    int n = C->P->n[a];
    int m = C->P->full ? C->P->n[a] / 2 : C->P->m[a];
    int g = (qa - m + i) % n;
    return g < 0 ? g + n : g;
}

/* Per-column list of the local indices where an atom's axis factor is nonzero, and the list the
 * force moments contract over (the same, or with grad_fd the indices within p points of the
 * support, where D_h g can be nonzero). */
typedef struct {
    int cnt[3];
    int *idx[3];           /* local indices */
    int *gi[3];            /* matching global indices */
    int cntd[3];
    int *idxd[3];
    int *gid[3];
} atom_window;

typedef struct {
    int nact;
    int *atom;             /* active atom ids */
    atom_window *win;      /* per active atom */
    int *store;            /* backing storage */
} column_atoms;

static int column_atoms_build(const oracle_ctx *C, const int q3[3], column_atoms *ca)
{
    const sq_oracle_problem *P = C->P;
    int per = 4 * (C->nc[0] + C->nc[1] + C->nc[2]);
    ca->atom = (int *)malloc(sizeof(int) * (P->natom > 0 ? P->natom : 1));
    ca->win = (atom_window *)malloc(sizeof(atom_window) * (P->natom > 0 ? P->natom : 1));
    ca->store = (int *)malloc(sizeof(int) * (size_t)per * (P->natom > 0 ? P->natom : 1));
    if (!ca->atom || !ca->win || !ca->store) return -1;
    ca->nact = 0;
    for (int J = 0; J < P->natom; J++) {
        atom_window *wv = &ca->win[ca->nact];
        int *s = ca->store + (size_t)per * ca->nact;
        int ok = 1;
        for (int a = 0; a < 3; a++) {
            const double *g = factor(C, J, a, F_G);
            wv->idx[a] = s;
            s += C->nc[a];
            wv->gi[a] = s;
            s += C->nc[a];
            wv->cnt[a] = 0;
            for (int i = 0; i < C->nc[a]; i++) {
                int gi = glob(C, a, q3[a], i);
                if (g[gi] != 0.0) {
                    wv->idx[a][wv->cnt[a]] = i;
                    wv->gi[a][wv->cnt[a]] = gi;
                    wv->cnt[a]++;
                }
            }
            if (wv->cnt[a] == 0) ok = 0;
            wv->idxd[a] = s;
            s += C->nc[a];
            wv->gid[a] = s;
            s += C->nc[a];
            wv->cntd[a] = 0;
            int reach = P->grad_fd ? C->p : 0;
            for (int i = 0; i < C->nc[a]; i++) {
                int gi = glob(C, a, q3[a], i);
                int near = 0;
                for (int j = -reach; j <= reach && !near; j++) {
                    int gj = ((gi + j) % P->n[a] + P->n[a]) % P->n[a];
                    near = g[gj] != 0.0;
                }
                if (near) {
                    wv->idxd[a][wv->cntd[a]] = i;
                    wv->gid[a][wv->cntd[a]] = gi;
                    wv->cntd[a]++;
                }
            }
        }
        if (ok) ca->atom[ca->nact++] = J;
    }
    return 0;
}

static void column_atoms_free(column_atoms *ca)
{
    free(ca->atom);
    free(ca->win);
    free(ca->store);
}

/* out = Hhat_q v on the cube (local indices, x fastest). */
static void apply_hhat(const oracle_ctx *C, const int q3[3], const column_atoms *ca, double omega,
                       double tau, const double *v, double *out)
{
    const sq_oracle_problem *P = C->P;
    const int n0 = C->nc[0], n1 = C->nc[1], n2 = C->nc[2];
    const int p = C->p;
    /* kinetic + local potential: -1/2 Lap_h v + V_eff v (stencil neighbours from C->nbr) */
    for (int c = 0; c < n2; c++) {
        int gz = glob(C, 2, q3[2], c);
        for (int b = 0; b < n1; b++) {
            int gy = glob(C, 1, q3[1], b);
            for (int a = 0; a < n0; a++) {
                int gx = glob(C, 0, q3[0], a);
                long lc = a + (long)n0 * (b + (long)n1 * c);
                double V = P->veff[gx + (long)P->n[0] * (gy + (long)P->n[1] * gz)];
                double s = (C->kdiag + V) * v[lc];
                const int *nx = C->nbr[0] + a * 2 * p;
                const int *ny = C->nbr[1] + b * 2 * p;
                const int *nz = C->nbr[2] + c * 2 * p;
                for (int j = 1; j <= p; j++) {
                    int ip = nx[2 * (j - 1)], im = nx[2 * (j - 1) + 1];
                    double vp = ip >= 0 ? v[ip + (long)n0 * (b + (long)n1 * c)] : 0.0;
                    double vm = im >= 0 ? v[im + (long)n0 * (b + (long)n1 * c)] : 0.0;
                    s += C->w[0][j] * (vp + vm);
                    ip = ny[2 * (j - 1)];
                    im = ny[2 * (j - 1) + 1];
                    vp = ip >= 0 ? v[a + (long)n0 * (ip + (long)n1 * c)] : 0.0;
                    vm = im >= 0 ? v[a + (long)n0 * (im + (long)n1 * c)] : 0.0;
                    s += C->w[1][j] * (vp + vm);
                    ip = nz[2 * (j - 1)];
                    im = nz[2 * (j - 1) + 1];
                    vp = ip >= 0 ? v[a + (long)n0 * (b + (long)n1 * ip)] : 0.0;
                    vm = im >= 0 ? v[a + (long)n0 * (b + (long)n1 * im)] : 0.0;
                    s += C->w[2][j] * (vp + vm);
                }
                out[lc] = s;
            }
        }
    }
    /* nonlocal: sum_J sum_lm c_l dV chi (chi^T v), both restricted to the cube */
    for (int t = 0; t < ca->nact; t++) {
        int J = ca->atom[t];
        const atom_window *wv = &ca->win[t];
        for (int lm = 0; lm < C->nproj; lm++) {
            int ty[3];
            proj_factor_types(lm, -1, ty);
            const double *fx = factor(C, J, 0, ty[0]);
            const double *fy = factor(C, J, 1, ty[1]);
            const double *fz = factor(C, J, 2, ty[2]);
            double dot = 0.0;
            for (int kc = 0; kc < wv->cnt[2]; kc++)
                for (int kb = 0; kb < wv->cnt[1]; kb++)
                    for (int ka = 0; ka < wv->cnt[0]; ka++) {
                        long lc = wv->idx[0][ka] +
                                  (long)n0 * (wv->idx[1][kb] + (long)n1 * wv->idx[2][kc]);
                        double chi = C->N * fx[wv->gi[0][ka]] * fy[wv->gi[1][kb]] * fz[wv->gi[2][kc]];
                        dot += chi * v[lc];
                    }
            double coef = P->cl[lm == 0 ? 0 : 1] * C->dV * dot;
            for (int kc = 0; kc < wv->cnt[2]; kc++)
                for (int kb = 0; kb < wv->cnt[1]; kb++)
                    for (int ka = 0; ka < wv->cnt[0]; ka++) {
                        long lc = wv->idx[0][ka] +
                                  (long)n0 * (wv->idx[1][kb] + (long)n1 * wv->idx[2][kc]);
                        double chi = C->N * fx[wv->gi[0][ka]] * fy[wv->gi[1][kb]] * fz[wv->gi[2][kc]];
                        out[lc] += coef * chi;
                    }
        }
    }
    /* scale and shift: Hhat = (H - omega)/tau */
    for (long i = 0; i < C->nc3; i++) out[i] = (out[i] - omega * v[i]) / tau;
}

static long centre_local(const oracle_ctx *C)
{
    int c[3];
    for (int a = 0; a < 3; a++) c[a] = C->P->full ? C->P->n[a] / 2 : C->P->m[a];
    return c[0] + (long)C->nc[0] * (c[1] + (long)C->nc[1] * c[2]);
}

static void unravel(const sq_oracle_problem *P, long q, int q3[3])
{
    q3[0] = (int)(q % P->n[0]);
    q3[1] = (int)((q / P->n[0]) % P->n[1]);
    q3[2] = (int)(q / ((long)P->n[0] * P->n[1]));
}

/* Apply Hhat_q to one local cube vector (used by the tests to pin the operator). */
int sq_oracle_apply(const sq_oracle_problem *P, long q, double omega, double tau, const double *v,
                    double *out)
{
    oracle_ctx C;
    int rc = ctx_init(&C, P);
    if (rc) return rc;
    int q3[3];
    unravel(P, q, q3);
    column_atoms ca;
    if (column_atoms_build(&C, q3, &ca)) { ctx_free(&C); return -3; }
    apply_hhat(&C, q3, &ca, omega, tau, v, out);
    column_atoms_free(&ca);
    ctx_free(&C);
    return 0;
}

/* Global grid index of every local cube point of column q (tests use it to build dense H_q). */
int sq_oracle_cube_indices(const sq_oracle_problem *P, long q, long *gidx)
{
    oracle_ctx C;
    int rc = ctx_init(&C, P);
    if (rc) return rc;
    int q3[3];
    unravel(P, q, q3);
    for (int c = 0; c < C.nc[2]; c++)
        for (int b = 0; b < C.nc[1]; b++)
            for (int a = 0; a < C.nc[0]; a++) {
                long lc = a + (long)C.nc[0] * (b + (long)C.nc[1] * c);
                gidx[lc] = glob(&C, 0, q3[0], a) +
                           (long)P->n[0] * (glob(&C, 1, q3[1], b) + (long)P->n[1] * glob(&C, 2, q3[2], c));
            }
    ctx_free(&C);
    return 0;
}

/*
 * Chebyshev moments of a set of columns.
 *   mu   [ncols][K+1]  : mu_k^q = v_k(q)
 *   A    [K+1][natom][nproj][3] (may be NULL): accumulated force moments over the given columns
 * Returns 0 on success.
 */
int sq_oracle_moments(const sq_oracle_problem *P, double omega, double tau, int K, long ncols,
                      const long *cols, double *mu, double *A, int nthreads)
{
    oracle_ctx C;
    int rc = ctx_init(&C, P);
    if (rc) return rc;
    const int nproj = C.nproj;
    const long asz = (long)(K + 1) * P->natom * nproj * 3;
    if (A) memset(A, 0, sizeof(double) * asz);
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *va = (double *)malloc(sizeof(double) * C.nc3);
        double *vb = (double *)malloc(sizeof(double) * C.nc3);
        double *tmp = (double *)malloc(sizeof(double) * C.nc3);
        double *Aloc = A ? (double *)calloc(asz, sizeof(double)) : NULL;
        if (!va || !vb || !tmp || (A && !Aloc)) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (long ic = 0; ic < ncols; ic++) {
                long q = cols[ic];
                int q3[3];
                unravel(P, q, q3);
                column_atoms ca;
                if (column_atoms_build(&C, q3, &ca)) {
#pragma omp atomic write
                    err = 1;
                    continue;
                }
                const long cen = centre_local(&C);
                double *vprev = va, *vcur = vb;
                double *mq = mu + ic * (K + 1);
                /* v_0 = e_q */
                memset(vcur, 0, sizeof(double) * C.nc3);
                vcur[cen] = 1.0;
                memset(vprev, 0, sizeof(double) * C.nc3);
                for (int k = 0; k <= K; k++) {
                    mq[k] = vcur[cen];
                    /* force moments of v_k: for atoms whose projectors are nonzero at x_q */
                    if (A) {
                        for (int t = 0; t < ca.nact; t++) {
                            int J = ca.atom[t];
                            double gq[3];
                            for (int a = 0; a < 3; a++) gq[a] = factor(&C, J, a, F_G)[q3[a]];
                            if (gq[0] == 0.0 || gq[1] == 0.0 || gq[2] == 0.0) continue;
                            const atom_window *wv = &ca.win[t];
                            for (int lm = 0; lm < nproj; lm++) {
                                int ty[3];
                                proj_factor_types(lm, -1, ty);
                                double chi_q = C.N;
                                for (int a = 0; a < 3; a++)
                                    chi_q *= factor(&C, J, a, ty[a])[q3[a]];
                                for (int d = 0; d < 3; d++) {
                                    int td[3];
                                    proj_factor_types(lm, d, td);
                                    const double *fx = factor(&C, J, 0, td[0]);
                                    const double *fy = factor(&C, J, 1, td[1]);
                                    const double *fz = factor(&C, J, 2, td[2]);
                                    double dot = 0.0;
                                    for (int kc = 0; kc < wv->cntd[2]; kc++)
                                        for (int kb = 0; kb < wv->cntd[1]; kb++)
                                            for (int ka = 0; ka < wv->cntd[0]; ka++) {
                                                long lc = wv->idxd[0][ka] + (long)C.nc[0] * (wv->idxd[1][kb] + (long)C.nc[1] * wv->idxd[2][kc]);
                                                dot += C.N * fx[wv->gid[0][ka]] * fy[wv->gid[1][kb]] * fz[wv->gid[2][kc]] * vcur[lc];
                                            }
                                    Aloc[(((long)k * P->natom + J) * nproj + lm) * 3 + d] += chi_q * dot;
                                }
                            }
                        }
                    }
                    if (k == K) break;
                    apply_hhat(&C, q3, &ca, omega, tau, vcur, tmp);
                    if (k == 0) {
                        /* v_1 = Hhat v_0 */
                        for (long i = 0; i < C.nc3; i++) vprev[i] = tmp[i];
                    } else {
                        /* v_{k+1} = 2 Hhat v_k - v_{k-1} */
                        for (long i = 0; i < C.nc3; i++) vprev[i] = 2.0 * tmp[i] - vprev[i];
                    }
                    double *sw = vprev;
                    vprev = vcur;
                    vcur = sw;
                }
                column_atoms_free(&ca);
            }
        }
        if (A && Aloc) {
#pragma omp critical
            for (long i = 0; i < asz; i++) A[i] += Aloc[i];
        }
        free(va);
        free(vb);
        free(tmp);
        free(Aloc);
    }
    ctx_free(&C);
    return err ? -4 : 0;
}

/* Maximum number of OpenMP threads the oracle would use. */
int sq_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Forward-mode tangent of the moments along a potential perturbation dV (full grid, FP64):
 * differentiating Eq. Chebyshev with Hhat_q depending on V_eff through its diagonal,
 *   dv_0 = 0,  dv_1 = dH v_0,  dv_{k+1} = 2 Hhat dv_k + 2 dH v_k - dv_{k-1},
 * with dH = diag(dV restricted to the cube) / tau, and dmu_k^q = dv_k(q).  omega and tau are held
 * fixed.  dmu is [ncols][K+1].
 */
int sq_oracle_tangent(const sq_oracle_problem *P, double omega, double tau, int K, const double *dV, long ncols,
                      const long *cols, double *dmu, int nthreads)
{
    oracle_ctx C;
    int rc = ctx_init(&C, P);
    if (rc) return rc;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *v0 = (double *)malloc(sizeof(double) * C.nc3), *v1 = (double *)malloc(sizeof(double) * C.nc3);
        double *d0 = (double *)malloc(sizeof(double) * C.nc3), *d1 = (double *)malloc(sizeof(double) * C.nc3);
        double *t1 = (double *)malloc(sizeof(double) * C.nc3), *t2 = (double *)malloc(sizeof(double) * C.nc3);
        double *dloc = (double *)malloc(sizeof(double) * C.nc3);
        if (!v0 || !v1 || !d0 || !d1 || !t1 || !t2 || !dloc) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (long ic = 0; ic < ncols; ic++) {
                long q = cols[ic];
                int q3[3];
                unravel(P, q, q3);
                column_atoms ca;
                if (column_atoms_build(&C, q3, &ca)) {
#pragma omp atomic write
                    err = 1;
                    continue;
                }
                for (int c = 0; c < C.nc[2]; c++)
                    for (int b = 0; b < C.nc[1]; b++)
                        for (int a = 0; a < C.nc[0]; a++) {
                            long lc = a + (long)C.nc[0] * (b + (long)C.nc[1] * c);
                            long g = glob(&C, 0, q3[0], a) +
                                     (long)P->n[0] * (glob(&C, 1, q3[1], b) + (long)P->n[1] * glob(&C, 2, q3[2], c));
                            dloc[lc] = dV[g] / tau;
                        }
                const long cen = centre_local(&C);
                double *vprev = v0, *vcur = v1, *dprev = d0, *dcur = d1;
                double *mq = dmu + ic * (K + 1);
                memset(vcur, 0, sizeof(double) * C.nc3);
                vcur[cen] = 1.0;
                memset(vprev, 0, sizeof(double) * C.nc3);
                memset(dcur, 0, sizeof(double) * C.nc3);
                memset(dprev, 0, sizeof(double) * C.nc3);
                mq[0] = 0.0;
                for (int k = 0; k < K; k++) {
                    apply_hhat(&C, q3, &ca, omega, tau, vcur, t1);
                    apply_hhat(&C, q3, &ca, omega, tau, dcur, t2);
                    if (k == 0) {
                        for (long i = 0; i < C.nc3; i++) {
                            dprev[i] = t2[i] + dloc[i] * vcur[i];
                            vprev[i] = t1[i];
                        }
                    } else {
                        for (long i = 0; i < C.nc3; i++) {
                            dprev[i] = 2.0 * t2[i] + 2.0 * dloc[i] * vcur[i] - dprev[i];
                            vprev[i] = 2.0 * t1[i] - vprev[i];
                        }
                    }
                    double *sw = vprev;
                    vprev = vcur;
                    vcur = sw;
                    sw = dprev;
                    dprev = dcur;
                    dcur = sw;
                    mq[k + 1] = dcur[cen];
                }
                column_atoms_free(&ca);
            }
        }
        free(v0); free(v1); free(d0); free(d1); free(t1); free(t2); free(dloc);
    }
    ctx_free(&C);
    return err ? -4 : 0;
}

/*
 * Lanczos iteration of Sec. 2.2 (Eq. Lanczos) on the truncated scaled operator Hhat_q of each given
 * column, started from the unit vector at the column's own point (eta_q = e_q):
 *     v_{-1} = 0, v_0 = e_q, b_0 v_{-1} = 0,
 *     a_{k+1} = (Hhat v_k, v_k),
 *     b_{k+1} v_{k+1} = (Hhat - a_{k+1}) v_k - b_k v_{k-1},   b_{k+1} = || that vector ||,
 * for k = 0 .. K-1, without reorthogonalisation (the paper states none).  The Jacobi matrix of the
 * column is tridiag(b_1..b_{K-1}; a_1..a_K; b_1..b_{K-1}); the Gauss nodes and weights follow from
 * its eigendecomposition (oracle.py).  When b_{k+1} = 0 the Krylov space is exhausted: the remaining
 * a and b are written as 0 and the caller truncates the Jacobi matrix there.
 *   a, b   [ncols][K]: a_1..a_K and b_1..b_K of the scaled operator (Hhat = (H - omega)/tau)
 */
int sq_oracle_lanczos(const sq_oracle_problem *P, double omega, double tau, int K, long ncols, const long *cols,
                      double *a, double *b, int nthreads)
{
    oracle_ctx C;
    int rc = ctx_init(&C, P);
    if (rc) return rc;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *vm = (double *)malloc(sizeof(double) * C.nc3), *v = (double *)malloc(sizeof(double) * C.nc3);
        double *w = (double *)malloc(sizeof(double) * C.nc3);
        if (!vm || !v || !w) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (long ic = 0; ic < ncols; ic++) {
                long q = cols[ic];
                int q3[3];
                unravel(P, q, q3);
                column_atoms ca;
                if (column_atoms_build(&C, q3, &ca)) {
#pragma omp atomic write
                    err = 1;
                    continue;
                }
                double *ak = a + ic * K, *bk = b + ic * K;
                memset(vm, 0, sizeof(double) * C.nc3);
                memset(v, 0, sizeof(double) * C.nc3);
                v[centre_local(&C)] = 1.0;
                double bprev = 0.0;
                int done = 0;
                for (int k = 0; k < K; k++) {
                    if (done) {
                        ak[k] = 0.0;
                        bk[k] = 0.0;
                        continue;
                    }
                    apply_hhat(&C, q3, &ca, omega, tau, v, w);
                    double alpha = 0.0;
                    for (long i = 0; i < C.nc3; i++) alpha += w[i] * v[i];
                    double nrm = 0.0;
                    for (long i = 0; i < C.nc3; i++) {
                        w[i] = w[i] - alpha * v[i] - bprev * vm[i];
                        nrm += w[i] * w[i];
                    }
                    double beta = sqrt(nrm);
                    ak[k] = alpha;
                    bk[k] = beta;
                    if (beta == 0.0) {
                        done = 1;
                        continue;
                    }
                    for (long i = 0; i < C.nc3; i++) {
                        vm[i] = v[i];
                        v[i] = w[i] / beta;
                    }
                    bprev = beta;
                }
                column_atoms_free(&ca);
            }
        }
        free(vm);
        free(v);
        free(w);
    }
    ctx_free(&C);
    return err ? -4 : 0;
}
