"""FP64 CPU oracle of the Clenshaw-Curtis spectral-quadrature (SQ) hot path.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA library is checked
against; only tests/, the package smoke check and bench.py's CPU-baseline leg may import it.  It
shares no code with the CUDA path: the per-column recursion is plain C (sq_oracle.c, OpenMP over
grid points); the steps after it (moment sums, Chebyshev coefficients, Fermi level, density,
energy, force) are plain numpy below, each written from the paper's definition.  The Gauss
(Lanczos) quadrature path for rho, U and S (lanczos, gauss_rule, gauss_fermi_level, gauss_solve) is
the paper's own density method; its Jacobi eigendecomposition uses scipy's tridiagonal eigensolver.

Paper: Ghosh & Bhattacharya, arXiv 2011.13517.  Sections cited below:
  Sec. 2.1  density-operator KS-DFT, Fermi-Dirac fixed point (Eq. FixedPoint), free energy,
            band energy U = 2 Tr(gamma H), entropy S, atomic force (Eq. AtomicForce)
  Sec. 2.2  spectral quadrature: pointwise u^q, s^q, rho^q (Eqs. RSIntegrals, uq, sq, rhoq),
            Fermi function and entropy density (Eq. FermiDirac), scale/shift, Chebyshev weights
            (Eq. ChebyshevWeights), Chebyshev recursion (Eq. Chebyshev), NL force (Eq. NLforceSQ)
  Sec. 3    discretisation, region of influence, Fermi level from the electron count (Eq. Ne),
            discrete nonlocal force.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sq_oracle.c")
_LIB = os.path.join(_HERE, "libsq_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags; runs on x86_64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("L", ctypes.c_double * 3),
        ("fd_order", ctypes.c_int),
        ("veff", ctypes.POINTER(ctypes.c_double)),
        ("natom", ctypes.c_int),
        ("R", ctypes.POINTER(ctypes.c_double)),
        ("lmax", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("cl", ctypes.POINTER(ctypes.c_double)),
        ("m", ctypes.c_int * 3),
        ("full", ctypes.c_int),
        ("grad_fd", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        _lib.sq_oracle_fd_coeffs.argtypes = [ctypes.c_int, dp]
        _lib.sq_oracle_fd1_coeffs.argtypes = [ctypes.c_int, dp]
        _lib.sq_oracle_axis_factors.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
        _lib.sq_oracle_apply.argtypes = [ctypes.POINTER(_Problem), ctypes.c_long, ctypes.c_double,
                                         ctypes.c_double, dp, dp]
        _lib.sq_oracle_cube_indices.argtypes = [ctypes.POINTER(_Problem), ctypes.c_long, lp]
        _lib.sq_oracle_moments.argtypes = [ctypes.POINTER(_Problem), ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_long, lp, dp, dp, ctypes.c_int]
        _lib.sq_oracle_max_threads.restype = ctypes.c_int
        _lib.sq_oracle_lanczos.argtypes = [ctypes.POINTER(_Problem), ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_long, lp, dp, dp, ctypes.c_int]
        _lib.sq_oracle_tangent.argtypes = [ctypes.POINTER(_Problem), ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           dp, ctypes.c_long, lp, dp, ctypes.c_int]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


class Problem:
    """ctypes view of a Cell (keeps the arrays alive)."""

    def __init__(self, cell, full: bool = False, m=None, grad_fd: bool = False):
        self.cell = cell
        self.veff = np.ascontiguousarray(cell.veff, dtype=np.float64)
        self.R = np.ascontiguousarray(cell.R, dtype=np.float64).reshape(-1)
        self.cl = np.ascontiguousarray(cell.proj_energy, dtype=np.float64)
        st = _Problem()
        for a in range(3):
            st.n[a] = int(cell.n[a])
            st.L[a] = float(cell.box[a])
            st.m[a] = int(cell.m[a] if m is None else m[a])
        st.fd_order = int(cell.fd_order)
        st.veff = _dp(self.veff)
        st.natom = int(cell.natom)
        st.R = _dp(self.R) if cell.natom else ctypes.POINTER(ctypes.c_double)()
        st.lmax = int(cell.lmax)
        st.sigma = float(cell.proj_sigma)
        st.rc = float(cell.proj_rc)
        st.cl = _dp(self.cl)
        st.full = 1 if full else 0
        st.grad_fd = 1 if grad_fd else 0
        self.st = st
        self.full = full
        self.nc = cell.n.copy() if full else 2 * np.array([st.m[0], st.m[1], st.m[2]]) + 1


# --------------------------------------------------------------------------------------------
# Hamiltonian pieces (Sec. 2.1, Sec. 3)

def fd_coeffs(order: int) -> np.ndarray:
    """Central 2nd-derivative FD weights c_0..c_p (Sec. 3 'Discretization'; order unstated)."""
    c = np.zeros(17)
    p = lib().sq_oracle_fd_coeffs(order, _dp(c))
    if p < 0:
        raise ValueError("bad FD order")
    return c[: p + 1].copy()


def fd1_coeffs(order: int) -> np.ndarray:
    """Central 1st-derivative FD weights a_0..a_p (a_0 = 0) of the gradient nabla_h (Sec. 3, local and
    nonlocal forces; same order as the Laplacian)."""
    a = np.zeros(17)
    p = lib().sq_oracle_fd1_coeffs(order, _dp(a))
    if p < 0:
        raise ValueError("bad FD order")
    return a[: p + 1].copy()


def axis_factors(R_a, L_a, n_a, sigma, rc):
    """1D periodised projector factors (g, hp, g', hp') on the n_a grid points of one axis."""
    out = [np.zeros(n_a) for _ in range(4)]
    lib().sq_oracle_axis_factors(float(R_a), float(L_a), int(n_a), float(sigma), float(rc),
                                 *[_dp(o) for o in out])
    return out


def projector_norm_const(sigma):
    return (math.pi * sigma * sigma) ** -0.75


def projectors(cell, grad: bool = False):
    """Projectors chi_Jlm on the full grid, shape [natom, nproj, N_d] (and their analytic
    gradients [natom, nproj, 3, N_d] when grad).  Dense: tiny cells only."""
    nproj = 1 if cell.lmax == 0 else 4
    N = projector_norm_const(cell.proj_sigma)
    chi = np.zeros((cell.natom, nproj, cell.N_d))
    dchi = np.zeros((cell.natom, nproj, 3, cell.N_d)) if grad else None
    for J in range(cell.natom):
        f = [axis_factors(cell.R[J, a], cell.box[a], cell.n[a], cell.proj_sigma, cell.proj_rc)
             for a in range(3)]
        for lm in range(nproj):
            for d in ([-1] + ([0, 1, 2] if grad else [])):
                ty = [1 if lm == 1 + a else 0 for a in range(3)]
                if d >= 0:
                    ty[d] += 2
                v = N * np.einsum("k,j,i->kji", f[2][ty[2]], f[1][ty[1]], f[0][ty[0]]).reshape(-1)
                if d < 0:
                    chi[J, lm] = v
                else:
                    dchi[J, lm, d] = v
    return (chi, dchi) if grad else chi


def kinetic_symbol_max(cell) -> float:
    """Largest eigenvalue of -1/2 Lap_h on the periodic grid: the Laplacian is a Kronecker sum of
    circulant matrices, so its eigenvalues are sum_i s_i(2 pi k_i / n_i) with
    s_i(theta) = -(c_0 + 2 sum_j c_j cos(j theta)) / (2 h_i^2)."""
    c = fd_coeffs(cell.fd_order)
    tot = 0.0
    for a in range(3):
        h = cell.box[a] / cell.n[a]
        th = 2.0 * math.pi * np.arange(cell.n[a]) / cell.n[a]
        s = c[0] + 2.0 * sum(c[j] * np.cos(j * th) for j in range(1, len(c)))
        tot += float(np.max(-s / (2.0 * h * h)))
    return tot


def nonlocal_bound(cell):
    """Interval holding the spectrum of the KB term sum_P c_P dV chi_P chi_P^T.  Its nonzero
    eigenvalues are those of the weighted Gram matrix C^1/2 G C^1/2 dV (G_PP' = <chi_P, chi_P'>),
    bounded by Gershgorin row sums.  The Gram entries factor over the three axes."""
    nproj = 1 if cell.lmax == 0 else 4
    if cell.natom == 0:
        return 0.0, 0.0
    N = projector_norm_const(cell.proj_sigma)
    dV = float(np.prod(cell.box / cell.n))
    f = [[axis_factors(cell.R[J, a], cell.box[a], cell.n[a], cell.proj_sigma, cell.proj_rc)
          for a in range(3)] for J in range(cell.natom)]
    P = cell.natom * nproj
    cP = np.array([cell.proj_energy[0 if lm == 0 else 1] for J in range(cell.natom) for lm in range(nproj)])
    G = np.ones((P, P))
    for a in range(3):
        F = np.zeros((P, cell.n[a]))
        for J in range(cell.natom):
            for lm in range(nproj):
                F[J * nproj + lm] = f[J][a][1 if lm == 1 + a else 0]
        G *= F @ F.T
    G *= N * N
    W = np.sqrt(np.abs(cP))[:, None] * np.abs(G) * np.sqrt(np.abs(cP))[None, :] * dV
    B = float(np.max(W.sum(axis=1)))
    lo = 0.0 if np.all(cP >= 0) else -B
    hi = 0.0 if np.all(cP <= 0) else B
    return lo, hi


def spectral_bounds(cell):
    """Rigorous [lambda_min, lambda_max] of the full periodic H (Sec. 2.2 needs the extreme
    eigenvalues for the scale and shift; how they are obtained is not stated).  Weyl's inequality
    on H = kinetic + diag(V_eff) + KB term: kinetic in [0, max symbol], potential in
    [min V, max V], KB term in nonlocal_bound().  Every truncated H_q is a principal submatrix of
    H, so by Cauchy interlacing its spectrum lies in the same interval."""
    klo, khi = 0.0, kinetic_symbol_max(cell)
    nlo, nhi = nonlocal_bound(cell)
    return klo + float(cell.veff.min()) + nlo, khi + float(cell.veff.max()) + nhi


def scale_shift(lmin, lmax):
    """omega = (lmax + lmin)/2, tau = (lmax - lmin)/2 (Sec. 2.2)."""
    return 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)


# --------------------------------------------------------------------------------------------
# Per-column recursion (Eq. Chebyshev) via the C oracle

def apply_hhat(cell, q, omega, tau, v, full=False, m=None):
    prob = Problem(cell, full=full, m=m)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    rc = lib().sq_oracle_apply(ctypes.byref(prob.st), int(q), float(omega), float(tau), _dp(v), _dp(out))
    if rc:
        raise RuntimeError(f"sq_oracle_apply failed ({rc})")
    return out


def cube_indices(cell, q, full=False, m=None):
    prob = Problem(cell, full=full, m=m)
    out = np.zeros(int(np.prod(prob.nc)), dtype=np.int64)
    rc = lib().sq_oracle_cube_indices(ctypes.byref(prob.st), int(q), _lp(out))
    if rc:
        raise RuntimeError(f"sq_oracle_cube_indices failed ({rc})")
    return out


def moments(cell, omega, tau, K=None, cols=None, force=False, nthreads=0, full=False, m=None, grad_fd=False):
    """mu [ncols, K+1] with mu_k^q = (T_k(Hhat_q))_qq, and (if force) the force moments
    A [K+1, natom, nproj, 3] summed over the given columns (grad_fd: with the FD gradient D_h chi)."""
    K = cell.K if K is None else K
    cols = np.arange(cell.N_d, dtype=np.int64) if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
    prob = Problem(cell, full=full, m=m, grad_fd=grad_fd)
    mu = np.zeros((cols.size, K + 1))
    nproj = 1 if cell.lmax == 0 else 4
    A = np.zeros((K + 1, cell.natom, nproj, 3)) if force else None
    rc = lib().sq_oracle_moments(ctypes.byref(prob.st), float(omega), float(tau), int(K), int(cols.size),
                                 _lp(cols), _dp(mu), _dp(A) if force else ctypes.POINTER(ctypes.c_double)(),
                                 int(nthreads))
    if rc:
        raise RuntimeError(f"sq_oracle_moments failed ({rc})")
    return (mu, A) if force else mu


def max_threads() -> int:
    return int(lib().sq_oracle_max_threads())


# --------------------------------------------------------------------------------------------
# Fermi-Dirac function and entropy density (Eq. FermiDirac, Sec. 2.2)

def fermi(lam, lam_f, kT):
    """g = 1/(1 + exp((lam - lam_f)/kT)), written as (1 - tanh(y/2))/2 (no overflow)."""
    return 0.5 * (1.0 - np.tanh((lam - lam_f) / (2.0 * kT)))


def entropy_density(lam, lam_f, kT):
    """s = g ln g + (1-g) ln(1-g) <= 0, evaluated as -[log1p(e^-|y|) + |y| g(|y|)],
    y = (lam - lam_f)/kT (s is even in y)."""
    y = np.abs((lam - lam_f) / kT)
    return -(np.log1p(np.exp(-y)) + y * fermi(y, 0.0, 1.0))


# --------------------------------------------------------------------------------------------
# Chebyshev coefficients (Eq. ChebyshevWeights)

def n_nodes(K, kT, tau):
    """Chebyshev-Gauss node count M = 2^ceil(log2 max(4(K+1), 16 tau/kT)) (reading: the paper does
    not say how the weight integral is evaluated)."""
    need = max(4 * (K + 1), 16.0 * tau / kT)
    return 1 << int(math.ceil(math.log2(need)))


def cheb_nodes(M):
    theta = math.pi * (np.arange(M) + 0.5) / M
    return theta, np.cos(theta)


def cheb_coeffs(fvals, theta, K):
    """a_k = (2 - delta_k0)/M sum_j f(x_j) cos(k theta_j): M-point Chebyshev-Gauss quadrature of
    (2/pi) int f T_k / sqrt(1 - x^2) dx, with the 1/2 of the k = 0 term folded in, so that
    f ~ sum_{k=0}^K a_k T_k."""
    M = theta.size
    a = np.array([np.dot(fvals, np.cos(k * theta)) for k in range(K + 1)]) * (2.0 / M)
    a[0] *= 0.5
    return a


def fermi_coeffs(lam_f, omega, tau, kT, K, M):
    """Chebyshev coefficients of g (c_k), of lam g (d_k, lam = tau x + omega), and of the entropy
    density s (e_k), all in the scaled variable x of Hhat."""
    theta, x = cheb_nodes(M)
    lam = tau * x + omega
    g = fermi(lam, lam_f, kT)
    return (cheb_coeffs(g, theta, K), cheb_coeffs(lam * g, theta, K),
            cheb_coeffs(entropy_density(lam, lam_f, kT), theta, K))


def electron_count(lam_f, Msum, omega, tau, kT, M):
    """N(lam_f) = 2 sum_k c_k(lam_f) M_k  (Eq. Ne with the CC quadrature)."""
    K = Msum.size - 1
    theta, x = cheb_nodes(M)
    c = cheb_coeffs(fermi(tau * x + omega, lam_f, kT), theta, K)
    return 2.0 * float(np.dot(c, Msum))


class NoBracket(ValueError):
    pass


def fermi_level(Msum, omega, tau, kT, N_e, lmin, lmax, M):
    """Solve N(lam_f) = N_e by bisection on [lmin, lmax] (Sec. 3 'Spectral weights ...' uses
    Brent; bisection is used here so that two implementations pick the same root even where the
    truncated N(lam) is not monotone).  Stops when the midpoint no longer separates the bracket."""
    lo, hi = float(lmin), float(lmax)
    if electron_count(lo, Msum, omega, tau, kT, M) > N_e or electron_count(hi, Msum, omega, tau, kT, M) < N_e:
        raise NoBracket("electron count not bracketed by the spectral bounds")
    for _ in range(200):
        mid = lo + 0.5 * (hi - lo)
        if mid <= lo or mid >= hi:
            break
        if electron_count(mid, Msum, omega, tau, kT, M) < N_e:
            lo = mid
        else:
            hi = mid
    return lo + 0.5 * (hi - lo)


# --------------------------------------------------------------------------------------------
# Observables (Eqs. uq, sq, rhoq, RSIntegrals; Sec. 3 free energy and nonlocal force)

def density(mu, c, dV):
    """rho(x_q) = rho^q / dV with rho^q = 2 sum_k c_k mu_k^q (electrons at point q)."""
    return 2.0 * (mu @ c) / dV


def band_energy(Msum, d):
    """U = 2 Tr(gamma H) = 2 sum_k d_k M_k."""
    return 2.0 * float(np.dot(d, Msum))


def entropy(Msum, e):
    """S = -2 Tr s(H) = -2 sum_k e_k M_k (units of k_B; S >= 0)."""
    return -2.0 * float(np.dot(e, Msum))


def nonlocal_force(A, c, cl, dV):
    """f_J,d = 4 dV sum_lm c_Jl sum_k c_k A_k^{J,lm,d}: the physical force -dF/dR_J of the KB term
    (Eq. AtomicForce and the discrete nonlocal force; sign reading: the printed expression is
    -dF/dR, checked by finite differences in the tests)."""
    nproj = A.shape[2]
    cl_lm = np.array([cl[0 if lm == 0 else 1] for lm in range(nproj)])
    return 4.0 * dV * np.einsum("k,kJld,l->Jd", c, A, cl_lm)


def sq_solve(cell, force=True, bounds=None, nthreads=0, full=False, K=None, cols_mu=None, grad_fd=False):
    """The whole SQ evaluation for one cell, oracle side.  Returns a dict with the spectral bounds,
    omega, tau, M, moment sums, Fermi level, density rho (per bohr^3), U, S, F_band = U - kT S and
    the nonlocal forces [natom, 3]."""
    K = cell.K if K is None else K
    lmin, lmax = spectral_bounds(cell) if bounds is None else bounds
    omega, tau = scale_shift(lmin, lmax)
    M = n_nodes(K, cell.kT, tau)
    dV = float(np.prod(cell.box / cell.n))
    res = moments(cell, omega, tau, K=K, force=force, nthreads=nthreads, full=full, grad_fd=grad_fd)
    mu, A = res if force else (res, None)
    Msum = mu.sum(axis=0)
    lam_f = fermi_level(Msum, omega, tau, cell.kT, cell.N_e, lmin, lmax, M)
    c, d, e = fermi_coeffs(lam_f, omega, tau, cell.kT, K, M)
    rho = density(mu, c, dV)
    U = band_energy(Msum, d)
    S = entropy(Msum, e)
    out = dict(lmin=lmin, lmax=lmax, omega=omega, tau=tau, M=M, K=K, mu=mu, Msum=Msum, lam_f=lam_f,
               c=c, d=d, e=e, rho=rho, U=U, S=S, F=U - cell.kT * S, dV=dV)
    if force:
        out["A"] = A
        out["force"] = nonlocal_force(A, c, cell.proj_energy, dV)
    return out


# --------------------------------------------------------------------------------------------
# Forward-mode derivative (tangent) of rho and U along a potential perturbation

def moment_tangent(cell, omega, tau, dV, K=None, cols=None, nthreads=0):
    """dmu [ncols, K+1]: derivative of the moments along dV (full grid), omega and tau fixed."""
    K = cell.K if K is None else K
    cols = np.arange(cell.N_d, dtype=np.int64) if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
    prob = Problem(cell)
    dVa = np.ascontiguousarray(np.asarray(dV, dtype=np.float64).reshape(-1))
    dmu = np.zeros((cols.size, K + 1))
    rc = lib().sq_oracle_tangent(ctypes.byref(prob.st), float(omega), float(tau), int(K), _dp(dVa),
                                 int(cols.size), _lp(cols), _dp(dmu), int(nthreads))
    if rc:
        raise RuntimeError(f"sq_oracle_tangent failed ({rc})")
    return dmu


def sq_tangent(cell, dV, bounds=None, K=None):
    """(d rho [N_d], d U, d lambda_f) along dV: the moment tangent pushed through the weights with the
    implicit derivative of the Fermi level, d lambda_f = -dN / N'(lambda_f), N = 2 sum_k c_k M_k
    (Eq. Ne), N' = 2 sum_k c'_k M_k where c'_k are the Chebyshev weights of dg/dlambda_f."""
    r = sq_solve(cell, force=False, bounds=bounds, K=K)
    K = r["K"]
    dmu = moment_tangent(cell, r["omega"], r["tau"], dV, K=K)
    dM = dmu.sum(axis=0)
    theta, x = cheb_nodes(r["M"])
    lam = r["tau"] * x + r["omega"]
    g = fermi(lam, r["lam_f"], cell.kT)
    gp = g * (1.0 - g) / cell.kT
    cp = cheb_coeffs(gp, theta, K)
    dp = cheb_coeffs(lam * gp, theta, K)
    Np = 2.0 * float(np.dot(cp, r["Msum"]))
    dN = 2.0 * float(np.dot(r["c"], dM))
    dlam = -dN / Np
    drho = 2.0 * (dmu @ r["c"] + dlam * (r["mu"] @ cp)) / r["dV"]
    dU = 2.0 * (float(np.dot(r["d"], dM)) + dlam * float(np.dot(dp, r["Msum"])))
    return drho, dU, dlam, r


# --------------------------------------------------------------------------------------------
# Gauss (Lanczos) spectral quadrature for rho, U and S (Sec. 2.2 "Spectral Gauss quadrature",
# Eq. Lanczos; Sec. 3 Eq. Ne and "Spectral weights, nodes and electronic fields")

def lanczos(cell, omega, tau, K=None, cols=None, nthreads=0, full=False, m=None):
    """Lanczos coefficients (a [ncols, K], b [ncols, K]) of the scaled truncated operator of each
    column, started from e_q (Eq. Lanczos): a_{k+1} = (Hhat v_k, v_k), b_{k+1} = ||(Hhat - a_{k+1}) v_k
    - b_k v_{k-1}||.  Zeros after an exact breakdown (b = 0)."""
    K = cell.K if K is None else K
    cols = np.arange(cell.N_d, dtype=np.int64) if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
    prob = Problem(cell, full=full, m=m)
    a = np.zeros((cols.size, K))
    b = np.zeros((cols.size, K))
    rc = lib().sq_oracle_lanczos(ctypes.byref(prob.st), float(omega), float(tau), int(K), int(cols.size), _lp(cols),
                                 _dp(a), _dp(b), int(nthreads))
    if rc:
        raise RuntimeError(f"sq_oracle_lanczos failed ({rc})")
    return a, b


def gauss_rule(a, b, omega, tau):
    """Spectral nodes and weights of each column from its Jacobi matrix J_K = tridiag(b; a; b): the
    nodes are the eigenvalues, the weights the squared first components of the normalised
    eigenvectors (Sec. 2.2; the printed sentence swaps the two symbols).  Nodes are returned in the
    unscaled energy, lambda = tau lambda_hat + omega.  A column whose b_k vanishes (exhausted Krylov
    space) uses the leading k x k block; its other nodes get weight 0.
    Returns (nodes [ncols, K], weights [ncols, K])."""
    from scipy.linalg import eigh_tridiagonal
    ncols, K = a.shape
    nodes = np.zeros((ncols, K))
    weights = np.zeros((ncols, K))
    for i in range(ncols):
        n = K
        for k in range(K - 1):
            if b[i, k] == 0.0:
                n = k + 1
                break
        lam, vec = eigh_tridiagonal(a[i, :n], b[i, :n - 1])
        nodes[i, :n] = tau * lam + omega
        nodes[i, n:] = omega
        weights[i, :n] = vec[0, :] ** 2
    return nodes, weights


def gauss_electron_count(lam_f, nodes, weights, kT):
    """N(lambda_f) = 2 sum_q sum_k w_k^q g(lambda_k^q, lambda_f) (Eq. Ne)."""
    return 2.0 * float(np.sum(weights * fermi(nodes, lam_f, kT)))


def gauss_fermi_level(nodes, weights, kT, N_e, lmin, lmax):
    """Root of N(lambda_f) = N_e by bisection on [lmin, lmax] (the paper uses Brent's method; the
    same deterministic rule as the Chebyshev path: mid = lo + (hi - lo)/2, lo = mid if N(mid) < N_e
    else hi = mid, until the midpoint no longer separates the bracket, at most 200 steps)."""
    lo, hi = lmin, lmax
    if gauss_electron_count(lo, nodes, weights, kT) > N_e or gauss_electron_count(hi, nodes, weights, kT) < N_e:
        raise ValueError("electron count not bracketed")
    x = lo + 0.5 * (hi - lo)
    for _ in range(200):
        if gauss_electron_count(x, nodes, weights, kT) < N_e:
            lo = x
        else:
            hi = x
        x = lo + 0.5 * (hi - lo)
        if x <= lo or x >= hi:
            break
    return x


def gauss_solve(cell, bounds=None, nthreads=0, full=False, K=None):
    """Gauss (Lanczos) SQ for one cell: spectral nodes and weights at every grid point, the Fermi
    level (Eq. Ne), and rho^q = 2 sum_k w_k g(lambda_k) (Eq. rhoq, electrons per point; rho = rho^q/dV
    per bohr^3), U = sum_q u^q with u^q = 2 sum_k w_k lambda_k g(lambda_k) (Eq. uq; the printed
    approximation drops the integral's factor 2), S = sum_q s^q with s^q = -2 sum_k w_k s(lambda_k)
    (Eq. sq, units of k_B), F = U - kT S."""
    K = cell.K if K is None else K
    lmin, lmax = spectral_bounds(cell) if bounds is None else bounds
    omega, tau = scale_shift(lmin, lmax)
    dV = float(np.prod(cell.box / cell.n))
    a, b = lanczos(cell, omega, tau, K=K, nthreads=nthreads, full=full)
    nodes, weights = gauss_rule(a, b, omega, tau)
    lam_f = gauss_fermi_level(nodes, weights, cell.kT, cell.N_e, lmin, lmax)
    g = fermi(nodes, lam_f, cell.kT)
    rho_q = 2.0 * np.sum(weights * g, axis=1)
    U = 2.0 * float(np.sum(weights * nodes * g))
    S = -2.0 * float(np.sum(weights * entropy_density(nodes, lam_f, cell.kT)))
    return dict(lmin=lmin, lmax=lmax, omega=omega, tau=tau, K=K, a=a, b=b, nodes=nodes, weights=weights,
                lam_f=lam_f, rho=rho_q / dV, U=U, S=S, F=U - cell.kT * S, dV=dV)
