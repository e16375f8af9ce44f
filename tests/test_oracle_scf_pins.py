"""Pins of the oracle's self-consistency pieces (oracle/electrostatics.py) against what mathematics and
physics fix independently of its code: the Slater exchange in another closed form, V_xc as the
derivative of rho eps_xc, the exact high-density coefficient of the correlation energy, the Poisson
solution checked by applying the finite-difference Laplacian in real space and on a plane wave, the
pseudocharge normalisation, and the self energy of a Gaussian charge."""
import math

import numpy as np
from scipy.special import erf

from oracle import electrostatics as es
from paper_2011_13517_gb300 import cells


def test_slater_exchange_closed_form():
    rho = np.array([1e-5, 1e-3, 0.01, 0.1, 1.0, 3.0])
    ex, vx = es.lda_exchange(rho)
    kf = (3.0 * math.pi ** 2 * rho) ** (1.0 / 3.0)          # Fermi wave number of the uniform gas
    np.testing.assert_allclose(ex, -3.0 * kf / (4.0 * math.pi), rtol=1e-14)
    np.testing.assert_allclose(vx, -kf / math.pi, rtol=1e-14)


def test_vxc_is_the_derivative_of_rho_exc():
    for rho in (1e-5, 3e-4, 0.01, 0.07, 0.5, 2.0):
        e = 1e-6 * rho
        f = lambda r: r * es.lda_pw92(np.array([r]))[0][0]
        num = (f(rho + e) - f(rho - e)) / (2 * e)
        v = es.lda_pw92(np.array([rho]))[1][0]
        assert abs(num - v) < 1e-8 * abs(v), (rho, num, v)


def test_pw92_high_density_coefficient_is_exact():
    # the correlation energy per electron of the uniform gas grows as c0 ln r_s for r_s -> 0 with
    # c0 = (1 - ln 2) / pi^2 (random-phase approximation, exact in that limit)
    c0 = (1.0 - math.log(2.0)) / math.pi ** 2
    assert abs(es.PW92_A - c0) < 1e-5 * c0
    ec1, _ = es.pw92_correlation(np.array([1e-7]))
    ec2, _ = es.pw92_correlation(np.array([1e-8]))
    slope = (ec1[0] - ec2[0]) / math.log(10.0)
    assert abs(slope - c0) < 2e-3 * c0
    # the correlation energy is negative and increases monotonically toward zero with r_s
    rs = np.geomspace(1e-3, 100.0, 50)
    ec, dec = es.pw92_correlation(rs)
    assert np.all(ec < 0) and np.all(np.diff(ec) > 0) and np.all(dec > 0)


def test_lda_zero_density():
    exc, vxc = es.lda_pw92(np.array([0.0, -1e-12]))
    assert np.all(exc == 0) and np.all(vxc == 0)


def test_poisson_residual_in_real_space():
    c = cells.tiny_cell()
    rng = np.random.default_rng(3)
    f = rng.standard_normal(c.N_d)
    phi = es.poisson_periodic(f, c)
    shape = (int(c.n[2]), int(c.n[1]), int(c.n[0]))
    lap = es.laplacian_apply(phi.reshape(shape), c).reshape(-1)
    res = -lap / (4.0 * math.pi) - (f - f.mean())
    assert np.max(np.abs(res)) < 1e-11 * np.max(np.abs(f))
    assert abs(phi.mean()) < 1e-13 * np.max(np.abs(phi))


def test_poisson_plane_wave():
    c = cells.vacancy_cell()
    n = [int(v) for v in c.n]
    x = np.arange(n[0]) * c.h[0]
    k = 2.0 * math.pi * 3 / c.box[0]
    f3 = np.broadcast_to(np.cos(k * x)[None, None, :], (n[2], n[1], n[0]))
    lam = es.laplacian_symbol(c)[0, 0, 3]
    phi = es.poisson_periodic(f3.reshape(-1), c)
    np.testing.assert_allclose(phi, (-4.0 * math.pi / lam * f3).reshape(-1), rtol=0, atol=1e-12)
    # the FD symbol approaches the continuum -k^2 on a smooth wave (12th order)
    assert abs(lam + k * k) < 1e-9 * k * k


def test_pseudocharge_normalisation_and_self_energy():
    c = cells.vacancy_cell()
    sig = 1.0
    Z = es.valence_charges(c)
    b = es.pseudocharge(c, sig)
    dV = float(np.prod(c.h))
    assert abs(b.sum() * dV + Z.sum()) < 1e-8 * Z.sum()
    assert np.all(b <= 0)
    # discrete self energy of one nucleus against the continuum value -Z^2 / (2 sqrt(pi) sigma)
    J = 0
    bJ = es.pseudocharge(c, sig, Z=np.where(np.arange(c.natom) == J, Z, 0.0))
    n = [int(v) for v in c.n]
    d2 = 0.0
    for a, npax in ((0, 2), (1, 1), (2, 0)):
        t = np.arange(n[a]) * c.h[a] - c.R[J, a]
        t = t - c.box[a] * np.round(t / c.box[a])
        shp = [1, 1, 1]
        shp[npax] = n[a]
        d2 = d2 + (t * t).reshape(shp)
    r = np.sqrt(d2).reshape(-1)
    arg = r / (math.sqrt(2.0) * sig)
    VJ = -Z[J] * np.where(r > 0, erf(arg) / np.where(r > 0, r, 1.0), math.sqrt(2.0 / math.pi) / sig)
    e_disc = -0.5 * dV * float(np.sum(bJ * VJ))
    e_cont = es.self_energy_continuum([Z[J]], sig)
    assert abs(e_disc - e_cont) < 1e-6 * abs(e_cont), (e_disc, e_cont)


def test_anderson_without_history_is_linear_mixing():
    rng = np.random.default_rng(4)
    hist = {}
    v0, o0 = rng.standard_normal(50), rng.standard_normal(50)
    v1, _ = es.anderson_next(v0, o0, hist, 0.3, 0)
    np.testing.assert_allclose(v1, v0 + 0.3 * (o0 - v0), rtol=0, atol=1e-15)
    o1 = rng.standard_normal(50)
    v2, _ = es.anderson_next(v1, o1, hist, 0.3, 0)
    np.testing.assert_allclose(v2, v1 + 0.3 * (o1 - v1), rtol=0, atol=1e-15)


def test_anderson_finds_the_fixed_point_of_an_affine_map():
    # V_out = A V + c with a contraction A: the fixed point solves (I - A) V = c; Anderson mixing with
    # enough history reaches it in far fewer steps than linear mixing
    rng = np.random.default_rng(8)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(rng.uniform(-0.9, 0.9, n)) @ Q.T
    c = rng.standard_normal(n)
    exact = np.linalg.solve(np.eye(n) - A, c)
    v, hist = np.zeros(n), {}
    for it in range(200):
        v_next, err = es.anderson_next(v, A @ v + c, hist, 0.5, 10)
        if err < 1e-12:
            break
        v = v_next
    assert it < 60
    np.testing.assert_allclose(v, exact, rtol=0, atol=1e-10 * np.abs(exact).max())


def test_scf_fixed_point_is_self_consistent_and_independent_of_the_mixing():
    c = cells.tiny_cell()
    r1 = es.scf(c, 1.0, beta=0.3, m=5, tol=1e-10, max_iter=80)
    r2 = es.scf(c, 1.0, beta=0.5, m=3, tol=1e-10, max_iter=80)
    assert r1["iters"] < 80 and r2["iters"] < 80
    scale = np.abs(r1["veff"]).max()
    assert np.max(np.abs(r1["veff"] - r2["veff"])) < 1e-8 * scale
    vout, _, _, _ = es.effective_potential(r1["rho"], c, 1.0)
    assert np.linalg.norm(vout - r1["veff"]) <= 1e-10 * np.linalg.norm(vout)
    assert abs(r1["rho"].sum() * float(np.prod(c.h)) - c.N_e) < 1e-9 * c.N_e


def test_local_force_is_minus_the_derivative_of_the_electrostatic_energy():
    """At a fixed density the local force f_J = dV sum (nabla_h b_J) phi (Eq. DiscreteLocalForce) is
    -dE/dR_J of the discrete electrostatic energy E = dV/2 sum (rho + b) phi + E_self^h (phi of rho + b),
    the pseudocharge b_J moving with its nucleus: central differences in R_J (95-atom cell, where the
    Gaussians are far inside the minimum image)."""
    import copy
    c = cells.vacancy_cell()
    sig = 1.0
    rho = np.exp(-c.veff.reshape(-1))
    rho *= c.N_e / (rho.sum() * float(np.prod(c.h)))
    dV = float(np.prod(c.h))

    def energy(cc):
        b = es.pseudocharge(cc, sig)
        phi = es.poisson_periodic(rho + b, cc)
        return 0.5 * dV * float(np.sum((rho + b) * phi)) + es.self_energy_discrete(cc, sig), phi

    _, phi = energy(c)
    f = es.local_force(c, sig, phi)
    J, e = 7, 1e-3
    for d in range(3):
        cp, cm = copy.deepcopy(c), copy.deepcopy(c)
        cp.R[J, d] += e
        cm.R[J, d] -= e
        fd = -(energy(cp)[0] - energy(cm)[0]) / (2 * e)
        assert abs(f[J, d] - fd) < 1e-6 * np.abs(f).max(), (d, f[J, d], fd)
    # summation by parts on the periodic grid: sum (D b_J) phi = -sum b_J (D phi)
    shape = (int(c.n[2]), int(c.n[1]), int(c.n[0]))
    g = es.grad_h(phi.reshape(shape), c)
    Z = es.valence_charges(c)
    bJ = es.pseudocharge_one(c, sig, J, Z[J])
    sbp = np.array([-dV * float(np.sum(bJ * g[d])) for d in range(3)])
    np.testing.assert_allclose(f[J], sbp, rtol=0, atol=1e-13 * np.abs(f).max())


def test_discrete_self_energy_of_the_cell():
    c = cells.vacancy_cell()
    Z = es.valence_charges(c)
    e = es.self_energy_discrete(c, 1.0)
    assert abs(e - es.self_energy_continuum(Z, 1.0)) < 1e-6 * abs(e)
