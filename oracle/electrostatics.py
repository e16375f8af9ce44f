"""FP64 CPU oracle of the self-consistency pieces around the SQ density: local exchange-correlation,
nuclear pseudocharges and the periodic finite-difference Poisson problem.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only tests/, the package smoke check and
bench.py's CPU legs may import it, and it shares no code with the CUDA path.

Paper: Ghosh & Bhattacharya, arXiv 2011.13517.
  Sec. 2.1  E_xc in the LDA with the Perdew-Wang parametrisation of the correlation energy;
            V_xc = dE_xc/drho; the electrostatic potential phi solves -(1/4 pi) lap phi = rho + b
            (Eq. Poisson) with b the total pseudocharge of the nuclei; V_eff = V_xc + phi.
  Sec. 3    "Electrostatic and effective potential": phi on the grid, V_eff^q = V_xc(rho^q) + phi^q.

Readings (the paper is silent on them):
  - The Perdew-Wang correlation is the spin-unpolarised fit with p = 1 and the published parameters
    A, alpha1, beta1..beta4 of its zeta = 0 column; exchange is the Slater (Dirac) form.
  - The pseudocharges are synthetic (the Troullier-Martins pseudopotentials are not available):
    b_J(x) = -Z_J (2 pi sigma_b^2)^(-3/2) exp(-|x - R_J|^2 / (2 sigma_b^2)) with minimum-image
    distances (the cells are at least 12 sigma_b wide), Z_J the valence charge (2 for Mg, 3 for Al).
  - The cells are periodic, so the Poisson problem is the periodic one with the same finite-
    difference Laplacian as the kinetic term; it is solvable for a zero-mean right-hand side, so
    the mean of rho + b (the grid's small normalisation error of the Gaussians; zero for a neutral
    cell in the continuum) is removed, and phi is taken with zero mean.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle

# Perdew-Wang correlation, spin-unpolarised (published fit parameters)
PW92_A = 0.031091
PW92_ALPHA1 = 0.21370
PW92_BETA = (7.5957, 3.5876, 1.6382, 0.49294)


def lda_exchange(rho):
    """Slater exchange per electron eps_x = -(3/4)(3/pi)^(1/3) rho^(1/3) and V_x = (4/3) eps_x."""
    rho = np.asarray(rho, dtype=np.float64)
    r13 = np.cbrt(np.maximum(rho, 0.0))
    ex = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * r13
    return ex, 4.0 / 3.0 * ex


def pw92_correlation(rs):
    """Perdew-Wang correlation per electron eps_c(r_s) and d eps_c / d r_s (spin-unpolarised, p = 1):
    eps_c = -2A (1 + alpha1 r_s) ln(1 + 1 / (2A (beta1 r_s^(1/2) + beta2 r_s + beta3 r_s^(3/2) + beta4 r_s^2)))."""
    rs = np.asarray(rs, dtype=np.float64)
    A, a1 = PW92_A, PW92_ALPHA1
    b1, b2, b3, b4 = PW92_BETA
    sq = np.sqrt(rs)
    q0 = -2.0 * A * (1.0 + a1 * rs)
    q1 = 2.0 * A * (b1 * sq + b2 * rs + b3 * rs * sq + b4 * rs * rs)
    dq1 = A * (b1 / sq + 2.0 * b2 + 3.0 * b3 * sq + 4.0 * b4 * rs)
    lg = np.log1p(1.0 / q1)
    ec = q0 * lg
    dec = -2.0 * A * a1 * lg - q0 * dq1 / (q1 * q1 + q1)
    return ec, dec


def lda_pw92(rho):
    """LDA exchange-correlation energy per electron eps_xc(rho) and potential V_xc = d(rho eps_xc)/d rho
    (Sec. 2.1); zero where rho <= 0."""
    rho = np.asarray(rho, dtype=np.float64)
    pos = rho > 0.0
    r = np.where(pos, rho, 1.0)
    ex, vx = lda_exchange(r)
    rs = np.cbrt(3.0 / (4.0 * math.pi * r))
    ec, dec = pw92_correlation(rs)
    vc = ec - rs / 3.0 * dec
    exc = np.where(pos, ex + ec, 0.0)
    vxc = np.where(pos, vx + vc, 0.0)
    return exc, vxc


def laplacian_apply(phi, cell):
    """The finite-difference Laplacian of the kinetic term (order cell.fd_order, periodic) applied to
    phi[n3, n2, n1] (x fastest), from shifted copies of the grid."""
    c = oracle.fd_coeffs(cell.fd_order)
    h = cell.h
    out = np.zeros_like(phi)
    for ax, npax in ((0, 2), (1, 1), (2, 0)):   # grid axis a is numpy axis 2 - a
        w = 1.0 / (h[ax] * h[ax])
        out += c[0] * w * phi
        for j in range(1, c.size):
            out += c[j] * w * (np.roll(phi, j, axis=npax) + np.roll(phi, -j, axis=npax))
    return out


def laplacian_symbol(cell):
    """Eigenvalues of the periodic FD Laplacian on the plane waves of the grid, shape [n3, n2, n1]."""
    c = oracle.fd_coeffs(cell.fd_order)
    n = [int(v) for v in cell.n]
    parts = []
    for ax in range(3):
        k = 2.0 * math.pi * np.arange(n[ax]) / n[ax]
        s = c[0] + 2.0 * sum(c[j] * np.cos(j * k) for j in range(1, c.size))
        parts.append(s / (cell.h[ax] * cell.h[ax]))
    return parts[2][:, None, None] + parts[1][None, :, None] + parts[0][None, None, :]


def poisson_periodic(f, cell):
    """phi with -(1/4 pi) L_h phi = f - mean(f) and mean(phi) = 0 (Eq. Poisson on the periodic grid),
    by the discrete Fourier transform of L_h's exact eigen-decomposition.  f: [N_d] or [n3, n2, n1]."""
    shape = (int(cell.n[2]), int(cell.n[1]), int(cell.n[0]))
    f3 = np.asarray(f, dtype=np.float64).reshape(shape)
    fh = np.fft.fftn(f3 - f3.mean())
    lam = laplacian_symbol(cell)
    lam[0, 0, 0] = 1.0
    ph = -4.0 * math.pi * fh / lam
    ph[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(ph)).reshape(np.shape(f))


def valence_charges(cell):
    """Z_J: 2 for the Mg-like sites, 3 for the Al-like ones (the cells' electron count N_e = sum Z_J)."""
    from paper_2011_13517_gb300 import cells as _cells
    return np.array([float(_cells.VALENCE[int(s)]) for s in np.asarray(cell.species)])


def pseudocharge(cell, sigma_b, Z=None):
    """Total pseudocharge b(x) = sum_J b_J(x) on the grid, [N_d] (reading above)."""
    Z = valence_charges(cell) if Z is None else np.asarray(Z, dtype=np.float64)
    n = [int(v) for v in cell.n]
    h = cell.h
    L = np.asarray(cell.box, dtype=np.float64)
    xs = [np.arange(n[a]) * h[a] for a in range(3)]
    b = np.zeros((n[2], n[1], n[0]))
    norm = (2.0 * math.pi * sigma_b * sigma_b) ** -1.5
    for J in range(cell.natom):
        d = []
        for a in range(3):
            t = xs[a] - cell.R[J, a]
            t = t - L[a] * np.round(t / L[a])
            d.append(t * t)
        r2 = d[2][:, None, None] + d[1][None, :, None] + d[0][None, None, :]
        b -= Z[J] * norm * np.exp(-r2 / (2.0 * sigma_b * sigma_b))
    return b.reshape(-1)


def self_energy_continuum(Z, sigma_b):
    """E_self = -(1/2) sum_J int b_J V_J for Gaussian pseudocharges in free space (Eq. Eself):
    -Z_J^2 / (2 sqrt(pi) sigma_b) per nucleus."""
    Z = np.asarray(Z, dtype=np.float64)
    return float(-np.sum(Z * Z) / (2.0 * math.sqrt(math.pi) * sigma_b))


def effective_potential(rho, cell, sigma_b):
    """V_eff = V_xc(rho) + phi(rho + b) on the grid (Sec. 3 'Electrostatic and effective potential')."""
    b = pseudocharge(cell, sigma_b)
    phi = poisson_periodic(np.asarray(rho) + b, cell)
    _, vxc = lda_pw92(rho)
    return vxc + phi, phi, vxc, b


def anderson_next(v_in, v_out, hist, beta, m):
    """One Anderson mixing step of the effective potential (Sec. 3, SCF mixing).  F = V_out - V_in; the
    history `hist` holds the previous (V_in, F) and the differences (dV_j, dF_j) of the last m steps;
    gamma minimises |F - sum_j gamma_j dF_j| and V_next = V_in + beta F - sum_j gamma_j (dV_j + beta dF_j).
    Returns (V_next, |F| / |V_out|)."""
    F = v_out - v_in
    if hist.get("prev") is not None:
        pv, pF = hist["prev"]
        hist.setdefault("d", []).append((v_in - pv, F - pF))
        hist["d"] = hist["d"][-m:] if m > 0 else []
    hist["prev"] = (v_in.copy(), F.copy())
    nxt = v_in + beta * F
    d = hist.get("d", [])
    if d:
        dF = np.array([x[1] for x in d])
        dV = np.array([x[0] for x in d])
        G = dF @ dF.T
        G = G + 1e-12 * np.trace(G) / len(d) * np.eye(len(d))
        gam = np.linalg.solve(G, dF @ F)
        nxt = nxt - gam @ (dV + beta * dF)
    return nxt, float(np.linalg.norm(F) / np.linalg.norm(v_out))


def scf(cell, sigma_b, beta=0.3, m=5, tol=1e-9, max_iter=100, K=None, v0=None, bounds=None):
    """Self-consistent field of the SQ density (Sec. 3 flow): V_in -> rho (Clenshaw-Curtis SQ with the
    library-independent oracle, spectral bounds of V_in unless given) -> V_out = V_xc(rho) + phi(rho + b) -> Anderson
    mixing, until |V_out - V_in| / |V_out| <= tol.  Returns the last V_in, rho, lambda_f, iterations and
    the error history."""
    import copy
    c = copy.deepcopy(cell)
    v = np.asarray(cell.veff if v0 is None else v0, dtype=np.float64).reshape(-1).copy()
    hist, errs = {}, []
    for it in range(1, max_iter + 1):
        c.veff = v.reshape(cell.veff.shape)
        r = oracle.sq_solve(c, force=False, K=K, bounds=bounds)
        vout, _, _, _ = effective_potential(r["rho"], c, sigma_b)
        v_next, err = anderson_next(v, vout, hist, beta, m)
        errs.append(err)
        if err <= tol:
            return dict(veff=v, rho=r["rho"], lam_f=r["lam_f"], iters=it, errors=errs)
        v = v_next
    return dict(veff=v, rho=r["rho"], lam_f=r["lam_f"], iters=max_iter, errors=errs)


# ------------------------------------------------------------------------------------------------
# Discrete free energy and local force (Sec. 3 "Free energy", "Atomic forces")

def grad_h(phi, cell):
    """The FD gradient nabla_h of the same order as the Laplacian, periodic: three arrays like phi."""
    a = oracle.fd1_coeffs(cell.fd_order)
    out = []
    for ax, npax in ((0, 2), (1, 1), (2, 0)):
        g = np.zeros_like(phi)
        for j in range(1, a.size):
            g += a[j] * (np.roll(phi, -j, axis=npax) - np.roll(phi, j, axis=npax))
        out.append(g / cell.h[ax])
    return out


def _min_image_r2(cell, J):
    n = [int(v) for v in cell.n]
    d2 = 0.0
    for a, npax in ((0, 2), (1, 1), (2, 0)):
        t = np.arange(n[a]) * cell.h[a] - cell.R[J, a]
        t = t - cell.box[a] * np.round(t / cell.box[a])
        shp = [1, 1, 1]
        shp[npax] = n[a]
        d2 = d2 + (t * t).reshape(shp)
    return d2


def pseudocharge_one(cell, sigma_b, J, Z):
    """b_J on the grid, [n3, n2, n1]."""
    norm = (2.0 * math.pi * sigma_b * sigma_b) ** -1.5
    return -Z * norm * np.exp(-_min_image_r2(cell, J) / (2.0 * sigma_b * sigma_b))


def self_energy_discrete(cell, sigma_b, Z=None):
    """E_self^h = -(1/2) h1 h2 h3 sum_q sum_I b_I^q V_I^q (Eq. DiscreteSelfEnergy), V_I the free-space
    potential of the Gaussian b_I: -Z_I erf(r / (sqrt 2 sigma_b)) / r (minimum image)."""
    from scipy.special import erf
    Z = valence_charges(cell) if Z is None else np.asarray(Z, dtype=np.float64)
    dV = float(np.prod(cell.h))
    e = 0.0
    for J in range(cell.natom):
        r = np.sqrt(_min_image_r2(cell, J))
        safe = np.where(r > 0, r, 1.0)
        V = -Z[J] * np.where(r > 0, erf(r / (math.sqrt(2.0) * sigma_b)) / safe, math.sqrt(2.0 / math.pi) / sigma_b)
        e += float(np.sum(pseudocharge_one(cell, sigma_b, J, Z[J]) * V))
    return -0.5 * dV * e


def free_energy(cell, sigma_b, rho, U, S, kT):
    """Discrete free energy (Eq. DiscreteEnergy) at the density rho whose band energy and entropy are
    U = sum_q u^q and S (k_B units, F_band = U - kT S):
    F^h = U - kT S + h1 h2 h3 sum_q [(eps_xc - V_xc) rho + (1/2)(b - rho) phi] + E_self^h,
    with phi of rho + b (zero mean) and eps_xc, V_xc of rho.  Returns (F, E_self)."""
    rho = np.asarray(rho, dtype=np.float64)
    b = pseudocharge(cell, sigma_b)
    phi = poisson_periodic(rho + b, cell)
    exc, vxc = lda_pw92(rho)
    dV = float(np.prod(cell.h))
    es_ = self_energy_discrete(cell, sigma_b)
    F = U - kT * S + dV * float(np.sum((exc - vxc) * rho + 0.5 * (b - rho) * phi)) + es_
    return F, es_


def local_force(cell, sigma_b, phi, Z=None):
    """f_J = h1 h2 h3 sum_q (nabla_h b_J)^q phi^q (Eq. DiscreteLocalForce), [natom, 3]: the gradient of
    each b_J on the grid, as printed."""
    Z = valence_charges(cell) if Z is None else np.asarray(Z, dtype=np.float64)
    shape = (int(cell.n[2]), int(cell.n[1]), int(cell.n[0]))
    ph = np.asarray(phi, dtype=np.float64).reshape(shape)
    dV = float(np.prod(cell.h))
    f = np.zeros((cell.natom, 3))
    for J in range(cell.natom):
        g = grad_h(pseudocharge_one(cell, sigma_b, J, Z[J]), cell)
        for d in range(3):
            f[J, d] = dV * float(np.sum(g[d] * ph))
    return f
