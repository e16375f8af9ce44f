"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the mathematics, not by the
oracle itself: textbook FD weights, the plane-wave symbol of the periodic FD Laplacian, Cauchy
restriction of an independently assembled dense H, Chebyshev moments from an eigendecomposition,
quadrature of the Chebyshev weight integral, the full-band special case, the electron-count sum
rule, the separable free-electron cube, convergence to the exact dense finite-temperature solution,
Hellmann-Feynman identities for dF/dV_eff and the nonlocal force, and exact lattice symmetries.
"""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle import dense, oracle
from paper_2011_13517_gb300 import cells


def pin_cell(lmax=1, m=2, noise=0.02, natoms_reps=(1, 1, 1), h=0.9, fd=6, K=30, kT=0.01, seed=3):
    """Small periodic hcp cell (4 atoms, 7x12x11 grid) whose dense H fits in memory."""
    c = cells.make_cell("pin", natoms_reps, h, fd, lmax, 0.0, K, kT, seed=seed, noise_amp=noise)
    c.R_cut = m * float(np.min(c.h)) + 1e-9
    # choose R_cut so that round(R_cut/h_i) == m on every axis
    c.R_cut = float(m * np.mean(c.h))
    assert np.all(c.m == m), (c.m, c.h)
    return c


# --- finite differences (Sec. 3 "Discretization") -----------------------------------------

@pytest.mark.parametrize("order,expected", [
    (2, [-2.0, 1.0]),
    (4, [-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0]),
    (6, [-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0]),
    (8, [-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0]),
])
def test_fd_coeffs_textbook(order, expected):
    np.testing.assert_allclose(oracle.fd_coeffs(order), expected, rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
def test_fd_coeffs_exact_on_polynomials(order):
    """sum_j c_|j| j^s equals s(s-1) 0^(s-2): exact second derivative of x^s at 0, s <= order+1."""
    c = oracle.fd_coeffs(order)
    p = order // 2
    for s in range(order + 2):
        val = sum(c[abs(j)] * float(j) ** s for j in range(-p, p + 1))
        exact = 2.0 if s == 2 else 0.0
        assert abs(val - exact) < 1e-9 * max(1.0, p ** s), (s, val)


def test_kinetic_plane_wave_symbol():
    """On the periodic grid a plane wave is an eigenvector of -1/2 Lap_h with eigenvalue
    sum_i -(c_0 + 2 sum_j c_j cos(j theta_i)) / (2 h_i^2)."""
    c = cells.make_cell("free", (1, 1, 1), 0.8, 8, 0, 1.0, 10, 0.01, noise_amp=0.0)
    c.veff = np.zeros_like(c.veff)
    c.R = np.zeros((0, 3))
    c.species = np.zeros(0, dtype=int)
    coef = oracle.fd_coeffs(c.fd_order)
    h = c.h
    n1, n2, n3 = c.n
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    for kvec in [(1, 0, 0), (0, 2, 0), (0, 0, 3), (2, 1, 1), (3, 5, 4)]:
        th = [2 * math.pi * kvec[a] / c.n[a] for a in range(3)]
        wave = np.cos(th[0] * i1 + th[1] * i2 + th[2] * i3 + 0.3).reshape(-1)
        sym = sum(-(coef[0] + 2 * sum(coef[j] * math.cos(j * th[a]) for j in range(1, len(coef))))
                  / (2 * h[a] ** 2) for a in range(3))
        q = 37
        gidx = oracle.cube_indices(c, q, full=True)
        v = wave[gidx]
        out = oracle.apply_hhat(c, q, 0.0, 1.0, v, full=True)
        np.testing.assert_allclose(out, sym * v, rtol=0, atol=1e-11)


# --- projectors (Sec. 2.1 nonlocal operator) -------------------------------------------------

def test_projector_norms_match_continuum():
    """On a fine grid, ||chi||^2 dV equals the continuum integral N^2 (int w^2)^3 (s) and
    N^2 (int 2 t^2/sigma^2 w^2)(int w^2)^2 (p); the sum over a periodic grid of a smooth
    compactly supported function converges spectrally."""
    sigma, rc = 1.0, 5.0
    c = cells.make_cell("norm", (2, 1, 1), 0.25, 2, 1, 1.0, 4, 0.01, noise_amp=0.0)
    c.R = np.array([[6.1, 5.2, 4.9]])
    c.species = np.zeros(1, dtype=int)
    chi = oracle.projectors(c)
    dV = float(np.prod(c.h))
    N = (math.pi * sigma ** 2) ** -0.75
    w = lambda t: math.exp(-t * t / (2 * sigma ** 2)) * (1 - t * t / rc ** 2) ** 3
    I0 = scipy.integrate.quad(lambda t: w(t) ** 2, -rc, rc, epsabs=1e-15, epsrel=1e-14)[0]
    I1 = scipy.integrate.quad(lambda t: 2 * t * t / sigma ** 2 * w(t) ** 2, -rc, rc,
                              epsabs=1e-15, epsrel=1e-14)[0]
    np.testing.assert_allclose(np.sum(chi[0, 0] ** 2) * dV, N ** 2 * I0 ** 3, rtol=1e-9)
    for m in range(3):
        np.testing.assert_allclose(np.sum(chi[0, 1 + m] ** 2) * dV, N ** 2 * I1 * I0 ** 2, rtol=1e-9)
    # s and p are orthogonal by parity
    for m in range(3):
        assert abs(np.sum(chi[0, 0] * chi[0, 1 + m]) * dV) < 1e-9


def test_projector_gradient_matches_finite_difference():
    """grad_x chi(x; R) = -d chi/dR: analytic gradient vs central differences in the atom position
    (including periodic images: the cell is smaller than the projector support)."""
    c = pin_cell()
    chi, dchi = oracle.projectors(c, grad=True)
    delta = 1e-5
    for J in (0, 2):
        for d in range(3):
            cp, cm = pin_cell(), pin_cell()
            cp.R = c.R.copy()
            cm.R = c.R.copy()
            cp.R[J, d] += delta
            cm.R[J, d] -= delta
            fd = -(oracle.projectors(cp)[J] - oracle.projectors(cm)[J]) / (2 * delta)
            np.testing.assert_allclose(dchi[J, :, d], fd, rtol=0, atol=2e-8)


def test_projector_lattice_translation():
    """Moving an atom by a box vector leaves its periodised projector unchanged."""
    c = pin_cell()
    chi = oracle.projectors(c)
    c2 = pin_cell()
    c2.R = c.R + c.box * np.array([1, -2, 3])
    np.testing.assert_allclose(oracle.projectors(c2), chi, rtol=0, atol=1e-13)


# --- the truncated Hamiltonian (Sec. 3 "Hamiltonian at each grid point") ---------------------

@pytest.mark.parametrize("lmax,m", [(0, 2), (1, 3)])
def test_cube_operator_is_principal_submatrix(lmax, m):
    """Hhat_q v from the matrix-free oracle equals (P_q H P_q - omega)/tau applied to v, with H
    assembled independently as a Kronecker sum of circulant FD matrices plus diag(V) plus the KB
    outer products."""
    c = pin_cell(lmax=lmax, m=m)
    H = dense.hamiltonian(c)
    rng = np.random.default_rng(5)
    omega, tau = 1.3, 7.5
    for q in [0, 17, c.N_d // 2, c.N_d - 1]:
        gidx = oracle.cube_indices(c, q)
        assert len(set(gidx.tolist())) == gidx.size
        assert gidx[(gidx.size - 1) // 2] == q
        v = rng.standard_normal(gidx.size)
        ref = (H[np.ix_(gidx, gidx)] @ v - omega * v) / tau
        np.testing.assert_allclose(oracle.apply_hhat(c, q, omega, tau, v), ref, rtol=0, atol=1e-12)


def test_full_mode_is_full_hamiltonian():
    c = pin_cell(lmax=1)
    H = dense.hamiltonian(c)
    rng = np.random.default_rng(6)
    q = 123
    gidx = oracle.cube_indices(c, q, full=True)
    v = rng.standard_normal(c.N_d)
    ref = H[np.ix_(gidx, gidx)] @ v
    np.testing.assert_allclose(oracle.apply_hhat(c, q, 0.0, 1.0, v, full=True), ref, rtol=0, atol=1e-12)


def test_spectral_bounds_contain_spectrum():
    c = pin_cell(lmax=1)
    ev = np.linalg.eigvalsh(dense.hamiltonian(c))
    lo, hi = oracle.spectral_bounds(c)
    assert lo <= ev[0] and ev[-1] <= hi
    # and they are not absurdly loose: within the nonlocal and potential ranges
    assert hi - ev[-1] < 1.0 and ev[0] - lo < 1.5


# --- Chebyshev recursion (Eq. Chebyshev) -----------------------------------------------------

@pytest.mark.parametrize("lmax,m", [(0, 2), (1, 3)])
def test_moments_match_eigendecomposition(lmax, m):
    """mu_k^q = e_q^T T_k(Hhat_q) e_q = sum_i U_qi^2 cos(k arccos lambda_i)."""
    c = pin_cell(lmax=lmax, m=m)
    lo, hi = oracle.spectral_bounds(c)
    omega, tau = oracle.scale_shift(lo, hi)
    K = 40
    cols = np.array([0, 5, 300, c.N_d - 1])
    mu = oracle.moments(c, omega, tau, K=K, cols=cols)
    for i, q in enumerate(cols):
        ref, lam = dense.cube_moments(c, int(q), omega, tau, K)
        assert lam.min() >= -1 and lam.max() <= 1
        np.testing.assert_allclose(mu[i], ref, rtol=0, atol=1e-12)


def test_free_electron_cube_is_separable():
    """V = 0, no projectors, 12th-order FD, 25^3 cube (the vacancy cell's truncation): the cube
    operator is a Kronecker sum of three 1D Toeplitz blocks, so mu_k = sum_abc u_a^2 u_b^2 u_c^2
    T_k((l_a + l_b + l_c - omega)/tau) from three small eigendecompositions."""
    c = cells.make_cell("free", (4, 2, 3), 0.5, 12, 0, 6.0, 60, 0.005, noise_amp=0.0)
    c.veff = np.zeros_like(c.veff)
    c.R = np.zeros((0, 3))
    c.species = np.zeros(0, dtype=int)
    assert np.all(c.n_c == 25)
    lo, hi = oracle.spectral_bounds(c)
    omega, tau = oracle.scale_shift(lo, hi)
    coef = oracle.fd_coeffs(12)
    lams, weights = [], []
    for a in range(3):
        nc = int(c.n_c[a])
        T = np.zeros((nc, nc))
        for i in range(nc):
            for j in range(nc):
                d = abs(i - j)
                if d < len(coef):
                    T[i, j] = -coef[d] / (2 * c.h[a] ** 2)
        l, U = np.linalg.eigh(T)
        lams.append(l)
        weights.append(U[nc // 2] ** 2)
    L = (lams[2][:, None, None] + lams[1][None, :, None] + lams[0][None, None, :] - omega) / tau
    W = weights[2][:, None, None] * weights[1][None, :, None] * weights[0][None, None, :]
    ac = np.arccos(np.clip(L, -1, 1)).reshape(-1)
    ref = np.array([np.dot(W.reshape(-1), np.cos(k * ac)) for k in range(c.K + 1)])
    cols = np.array([0, 12345, c.N_d - 1])
    mu = oracle.moments(c, omega, tau, cols=cols)
    for i in range(cols.size):
        np.testing.assert_allclose(mu[i], ref, rtol=0, atol=1e-12)


# --- Chebyshev weights, Fermi level and observables (Eqs. ChebyshevWeights, Ne, rhoq) -------

@pytest.mark.parametrize("lam_f,kT", [(0.3, 0.05), (-4.0, 0.2), (2.0, 0.02)])
def test_chebyshev_coefficients_match_quadrature(lam_f, kT):
    """c_k = (2/pi) int_{-1}^{1} g T_k / sqrt(1-x^2) dx (k = 0 halved), computed in theta-space
    by adaptive quadrature."""
    omega, tau, K = 1.0, 9.0, 30
    M = oracle.n_nodes(K, kT, tau)
    c, d, e = oracle.fermi_coeffs(lam_f, omega, tau, kT, K, M)
    tf = math.acos(max(-1.0, min(1.0, (lam_f - omega) / tau)))
    for k in range(K + 1):
        for coef, f in ((c, lambda lam: oracle.fermi(lam, lam_f, kT)),
                        (d, lambda lam: lam * oracle.fermi(lam, lam_f, kT)),
                        (e, lambda lam: oracle.entropy_density(lam, lam_f, kT))):
            integrand = lambda th: float(f(tau * math.cos(th) + omega)) * math.cos(k * th)
            val = scipy.integrate.quad(integrand, 0, math.pi, points=[tf], limit=1000,
                                       epsabs=1e-14, epsrel=1e-13)[0] * 2 / math.pi
            if k == 0:
                val *= 0.5
            assert abs(coef[k] - val) < 1e-12 * max(1.0, abs(omega) + tau), (k, coef[k], val)


def test_entropy_density_definition():
    lam = np.linspace(-3, 3, 101)
    g = oracle.fermi(lam, 0.2, 0.3)
    ref = g * np.log(g) + (1 - g) * np.log(1 - g)
    np.testing.assert_allclose(oracle.entropy_density(lam, 0.2, 0.3), ref, rtol=1e-12, atol=1e-15)


def test_full_band_special_case():
    """Fermi level far above the spectrum: g = 1 on [-1, 1], so c_0 = 1, c_k = 0 and
    rho^q = 2 mu_0 = 2 electrons at every point."""
    c = pin_cell()
    lo, hi = oracle.spectral_bounds(c)
    omega, tau = oracle.scale_shift(lo, hi)
    M = oracle.n_nodes(c.K, c.kT, tau)
    coef, _, _ = oracle.fermi_coeffs(hi + 200 * c.kT, omega, tau, c.kT, c.K, M)
    assert abs(coef[0] - 1.0) < 1e-14 and np.max(np.abs(coef[1:])) < 1e-14
    mu = oracle.moments(c, omega, tau, cols=np.arange(40))
    np.testing.assert_allclose(oracle.density(mu, coef, 1.0), 2.0, rtol=0, atol=1e-13)


def test_sum_rule_tiny_cell():
    """sum_q rho(x_q) dV = N_e after the Fermi-level solve (Eq. RSIntegrals / Eq. Ne)."""
    c = cells.tiny_cell()
    r = oracle.sq_solve(c, force=False)
    assert abs(r["rho"].sum() * r["dV"] - c.N_e) < 1e-11 * c.N_e
    assert r["S"] >= 0.0


# --- convergence to the exact dense solution and Hellmann-Feynman identities ------------------

@pytest.mark.slow
def test_untruncated_sq_converges_to_dense():
    """With no truncation (the cube is the whole periodic box) and K large enough for the
    Chebyshev series of g to converge, SQ gives the exact finite-temperature rho, U, S, lambda_f and
    nonlocal force of the dense eigendecomposition."""
    c = pin_cell(lmax=1, kT=0.1)
    ref = dense.solve(c)
    lo, hi = oracle.spectral_bounds(c)
    r = oracle.sq_solve(c, force=True, bounds=(lo, hi), full=True, K=700)
    assert abs(r["lam_f"] - ref["lam_f"]) < 1e-9
    np.testing.assert_allclose(r["rho"], ref["rho"], rtol=0, atol=1e-9 * np.max(ref["rho"]))
    assert abs(r["U"] - ref["U"]) < 1e-9 * max(1, abs(ref["U"]))
    assert abs(r["S"] - ref["S"]) < 1e-9 * max(1, abs(ref["S"]))
    np.testing.assert_allclose(r["force"], ref["force"], rtol=0, atol=1e-9)


def test_sq_error_decays_with_polynomial_order():
    """Untruncated SQ vs dense: the error envelope decays with K (exponential convergence of the
    Chebyshev series, Sec. 4 Table 1's Error ~ A exp(-beta K) shape)."""
    c = pin_cell(lmax=0, kT=0.1)
    ref = dense.solve(c, force=False)
    lo, hi = oracle.spectral_bounds(c)
    errs = []
    for K in (40, 80, 160, 320):
        r = oracle.sq_solve(c, force=False, bounds=(lo, hi), full=True, K=K)
        errs.append(np.max(np.abs(r["rho"] - ref["rho"])))
    assert errs[-1] < 1e-6 * np.max(ref["rho"])
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_truncated_sq_converges_with_cube_size():
    """Truncation error against R_cut (Sec. 4, the convergence of the energy with the truncation
    radius): on the 8-atom cell at a fixed K, the truncated SQ density, Fermi level, band energy and
    forces approach the untruncated SQ values at the same K as the cube grows (m = 3..6, cubes
    7^3..13^3), with the error falling by more than two decades over that range."""
    c = cells.tiny_cell()
    lo, hi = oracle.spectral_bounds(c)
    ref = oracle.sq_solve(c, force=True, bounds=(lo, hi), full=True)
    errs = []
    for m in (3, 4, 5, 6):
        c.R_cut = float(m * np.mean(c.h))
        assert np.all(c.m == m)
        r = oracle.sq_solve(c, force=True, bounds=(lo, hi))
        errs.append((np.max(np.abs(r["rho"] - ref["rho"])) / np.max(ref["rho"]), abs(r["lam_f"] - ref["lam_f"]),
                     abs(r["U"] - ref["U"]), np.max(np.abs(r["force"] - ref["force"]))))
    errs = np.array(errs)
    assert np.all(np.diff(errs, axis=0) < 0), errs
    assert np.all(errs[-1] < 1e-2 * errs[0]), errs


def test_hellmann_feynman_density():
    """dF/dV_eff(x_p) = rho(x_p) dV for F = U - kT S at fixed N_e (dense, exact)."""
    c = pin_cell(lmax=1, kT=0.05)
    ref = dense.solve(c, force=False)
    step = 1e-4
    for p in [0, 77, 400]:
        fp, fm = pin_cell(lmax=1, kT=0.05), pin_cell(lmax=1, kT=0.05)
        fp.veff = c.veff.copy()
        fm.veff = c.veff.copy()
        fp.veff.reshape(-1)[p] += step
        fm.veff.reshape(-1)[p] -= step
        dF = (dense.solve(fp, force=False)["F"] - dense.solve(fm, force=False)["F"]) / (2 * step)
        assert abs(dF - ref["rho"][p] * ref["dV"]) < 1e-7 * max(1e-3, abs(dF)), (p, dF)


def test_hellmann_feynman_force():
    """The nonlocal force equals -dF/dR_J when only atom J's projectors move (V_eff fixed)."""
    c = pin_cell(lmax=1, kT=0.05)
    ref = dense.solve(c, force=True)
    delta = 1e-4
    for J, d in [(0, 0), (1, 1), (3, 2)]:
        cp, cm = pin_cell(lmax=1, kT=0.05), pin_cell(lmax=1, kT=0.05)
        for cc in (cp, cm):
            cc.veff = c.veff.copy()
            cc.R = c.R.copy()
        cp.R[J, d] += delta
        cm.R[J, d] -= delta
        dF = (dense.solve(cp, force=False)["F"] - dense.solve(cm, force=False)["F"]) / (2 * delta)
        assert abs(-dF - ref["force"][J, d]) < 1e-7 * max(1e-3, abs(dF)), (J, d, -dF, ref["force"][J, d])


def test_hcp_symmetry_of_truncated_density():
    """Ideal hcp (no displacement, no noise) on a lattice-commensurate 16x16x14 grid: the SQ
    density is invariant under the lattice translations (a,0,0), (a/2, a sqrt3/2, 0) and the
    mirrors x -> -x, z -> -z (all map grid, atoms, V_eff, projectors and cubes to themselves)."""
    c = cells.make_cell("sym", (2, 1, 1), 0.7, 6, 1, 3.5, 20, 0.01, displace=0.0, noise_amp=0.0,
                        grid=(16, 16, 14))
    assert np.all(c.m == 5)
    r = oracle.sq_solve(c, force=False)
    rho = r["rho"].reshape(c.n[2], c.n[1], c.n[0])
    scale = np.max(np.abs(rho))
    tests = {
        "tx": np.roll(rho, 8, axis=2),
        "txy": np.roll(np.roll(rho, 4, axis=2), 8, axis=1),
        "mx": np.roll(rho[:, :, ::-1], 1, axis=2),
        "mz": np.roll(rho[::-1, :, :], 1, axis=0),
    }
    for name, t in tests.items():
        assert np.max(np.abs(t - rho)) < 1e-12 * scale, name


# --- the finite-difference gradient of the nonlocal force (Sec. 3 "Atomic forces") --------------

@pytest.mark.parametrize("order,expected", [
    (2, [0.0, 1.0 / 2.0]),
    (4, [0.0, 2.0 / 3.0, -1.0 / 12.0]),
    (6, [0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0]),
    (8, [0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0]),
])
def test_fd1_coeffs_textbook(order, expected):
    np.testing.assert_allclose(oracle.fd1_coeffs(order), expected, rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
def test_fd1_coeffs_exact_on_polynomials(order):
    """sum_j a_j (j^s - (-j)^s) is the exact first derivative of x^s at 0 (1 for s = 1, else 0) for
    every s <= order."""
    a = oracle.fd1_coeffs(order)
    p = order // 2
    for s in range(order + 1):
        val = sum(a[j] * (float(j) ** s - float(-j) ** s) for j in range(1, p + 1))
        exact = 1.0 if s == 1 else 0.0
        assert abs(val - exact) < 1e-9 * max(1.0, p ** s), (s, val)


def _periodic_fd_gradient(f3, h, a):
    """D_h f on the full periodic grid, f3 indexed [z][y][x]: plain np.roll differences per axis."""
    out = []
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        g = np.zeros_like(f3)
        for j in range(1, len(a)):
            g += a[j] * (np.roll(f3, -j, axis=ax) - np.roll(f3, j, axis=ax))
        out.append(g / h[d])
    return out


def test_fd_gradient_force_moments_match_dense_cube_eigendecomposition():
    """The oracle's force moments with the FD gradient (separable D_h tables) against an independent
    route: D_h chi by 3D np.roll differences of the dense projectors, and T_k(Hhat_q) e_q from the
    eigendecomposition of each dense cube operator; A_k = sum_q chi(x_q) (D_h chi)_{C_q}^T v_k^q."""
    c = pin_cell(lmax=1, m=2, K=6)
    lo, hi = oracle.spectral_bounds(c)
    omega, tau = oracle.scale_shift(lo, hi)
    _, A = oracle.moments(c, omega, tau, K=c.K, force=True, grad_fd=True)
    chi = oracle.projectors(c)
    a = oracle.fd1_coeffs(c.fd_order)
    H = dense.hamiltonian(c, chi)
    shape = (int(c.n[2]), int(c.n[1]), int(c.n[0]))
    Dchi = np.zeros((c.natom, chi.shape[1], 3, c.N_d))
    for J in range(c.natom):
        for lm in range(chi.shape[1]):
            for d, g in enumerate(_periodic_fd_gradient(chi[J, lm].reshape(shape), c.h, a)):
                Dchi[J, lm, d] = g.reshape(-1)
    ref = np.zeros_like(A)
    for q in range(c.N_d):
        gidx = oracle.cube_indices(c, q)
        Hq = (H[np.ix_(gidx, gidx)] - omega * np.eye(gidx.size)) / tau
        lam, U = np.linalg.eigh(Hq)
        lam = np.clip(lam, -1.0, 1.0)
        centre = int(np.flatnonzero(gidx == q)[0])
        for k in range(c.K + 1):
            vk = U @ (np.cos(k * np.arccos(lam)) * U[centre])
            ref[k] += np.einsum("jl,jldx,x->jld", chi[:, :, q], Dchi[:, :, :, gidx], vk)
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_fd_gradient_force_approaches_analytic_as_h_shrinks():
    """D_h chi -> grad chi at order n_o in h: the FD-gradient force approaches the analytic-gradient
    force of the same truncated SQ as the grid is refined (h = 0.9, 0.7, 0.55 bohr, 6th order)."""
    diffs = []
    for h in (0.9, 0.7, 0.55):
        c = cells.make_cell("gfd", (1, 1, 1), h, 6, 1, 0.0, 8, 0.01, seed=3)
        c.R_cut = float(2 * np.mean(c.h))
        assert np.all(c.m == 2)
        lo, hi = oracle.spectral_bounds(c)
        fa = oracle.sq_solve(c, force=True, bounds=(lo, hi))["force"]
        ff = oracle.sq_solve(c, force=True, bounds=(lo, hi), grad_fd=True)["force"]
        diffs.append(float(np.max(np.abs(ff - fa))) / float(np.max(np.abs(fa))))
    assert diffs[0] > 2.0 * diffs[1] > 4.0 * diffs[2], diffs
    assert diffs[2] < 1e-2, diffs


# --- Gauss (Lanczos) spectral quadrature (Sec. 2.2 "Spectral Gauss quadrature", Eq. Lanczos) -------

def _dense_cube(c, q, omega, tau):
    H = dense.hamiltonian(c, oracle.projectors(c) if c.natom else None)
    gidx = oracle.cube_indices(c, q)
    Hq = (H[np.ix_(gidx, gidx)] - omega * np.eye(gidx.size)) / tau
    lam, U = np.linalg.eigh(Hq)
    centre = int(np.flatnonzero(gidx == q)[0])
    return lam, U[centre] ** 2


def test_gauss_rule_integrates_polynomials_exactly():
    """A K-node Gauss rule of the spectral measure of e_q is exact for polynomials of degree 2K-1:
    sum_k w_k lam_k^j = (Hhat_q^j)_qq for j <= 2K - 1, with the right side from the eigendecomposition
    of the dense cube operator.  The weights sum to 1 (||e_q|| = 1)."""
    c = pin_cell(lmax=1, m=2, K=7)
    lo, hi = oracle.spectral_bounds(c)
    omega, tau = oracle.scale_shift(lo, hi)
    cols = np.array([0, 17, 400, c.N_d - 1])
    a, b = oracle.lanczos(c, omega, tau, K=c.K, cols=cols)
    nodes, w = oracle.gauss_rule(a, b, 0.0, 1.0)          # scaled nodes
    for i, q in enumerate(cols):
        lam, wq = _dense_cube(c, q, omega, tau)
        assert abs(w[i].sum() - 1.0) < 1e-13
        for j in range(2 * c.K):
            exact = float(np.dot(wq, lam ** j))
            assert abs(float(np.dot(w[i], nodes[i] ** j)) - exact) < 1e-12, (q, j)
    # and not beyond: degree 2K differs
    lam, wq = _dense_cube(c, cols[0], omega, tau)
    assert abs(float(np.dot(w[0], nodes[0] ** (2 * c.K))) - float(np.dot(wq, lam ** (2 * c.K)))) > 1e-12


def test_gauss_rule_with_the_whole_krylov_space_is_exact():
    """With K equal to the cube's dimension (m = 1: 27 points) the Krylov space of e_q is the whole
    cube, so the Gauss rule reproduces the spectral measure itself: rho^q = 2 g(H_q)_qq for any
    Fermi level, from the dense cube eigendecomposition."""
    c = pin_cell(lmax=1, m=1, K=27)
    lo, hi = oracle.spectral_bounds(c)
    omega, tau = oracle.scale_shift(lo, hi)
    cols = np.array([5, 300, 777])
    a, b = oracle.lanczos(c, omega, tau, K=c.K, cols=cols)
    nodes, w = oracle.gauss_rule(a, b, omega, tau)
    for lam_f in (-0.3, 0.2, 0.9):
        for i, q in enumerate(cols):
            lam, wq = _dense_cube(c, q, omega, tau)
            exact = 2.0 * float(np.dot(wq, oracle.fermi(tau * lam + omega, lam_f, c.kT)))
            got = 2.0 * float(np.dot(w[i], oracle.fermi(nodes[i], lam_f, c.kT)))
            assert abs(got - exact) < 1e-10, (q, lam_f, got, exact)


def test_gauss_sum_rule_and_entropy_sign():
    c = cells.tiny_cell()
    r = oracle.gauss_solve(c)
    assert abs(r["rho"].sum() * r["dV"] - c.N_e) < 1e-11 * c.N_e
    assert r["S"] >= 0.0
    np.testing.assert_allclose(r["weights"].sum(axis=1), 1.0, rtol=0, atol=1e-12)


@pytest.mark.slow
def test_untruncated_gauss_converges_faster_than_chebyshev():
    """No truncation (the cube is the whole box): Gauss quadrature converges to the exact dense
    finite-temperature density as K grows, and at the same K it is more accurate than the
    Clenshaw-Curtis (Chebyshev) expansion (the paper's observation in Sec. 4, Table 1)."""
    c = pin_cell(lmax=0, kT=0.1)
    ref = dense.solve(c, force=False)
    lo, hi = oracle.spectral_bounds(c)
    eg, ec = [], []
    for K in (10, 20, 40):
        g = oracle.gauss_solve(c, bounds=(lo, hi), full=True, K=K)
        ch = oracle.sq_solve(c, force=False, bounds=(lo, hi), full=True, K=K)
        eg.append(float(np.max(np.abs(g["rho"] - ref["rho"]))))
        ec.append(float(np.max(np.abs(ch["rho"] - ref["rho"]))))
    assert eg[0] > eg[1] > eg[2] and eg[2] < 1e-6 * np.max(ref["rho"]), eg
    assert all(x < y for x, y in zip(eg, ec)), (eg, ec)
    g20 = oracle.gauss_solve(c, bounds=(lo, hi), full=True, K=20)
    g40 = oracle.gauss_solve(c, bounds=(lo, hi), full=True, K=40)
    assert abs(g40["U"] - ref["U"]) < abs(g20["U"] - ref["U"]) and abs(g40["U"] - ref["U"]) < 1e-5
    assert abs(g40["lam_f"] - ref["lam_f"]) < 1e-6
