"""Dense-diagonalisation reference for tiny cells (TEST INFRASTRUCTURE ONLY).

Builds the full periodic discrete Hamiltonian as a dense matrix and evaluates the exact
finite-temperature quantities gamma = g(H) (Eq. FixedPoint), rho, U = 2 Tr(gamma H), the entropy
S = -2 Tr s(H) and the nonlocal force -dF/dR_J = 4 dV sum_lm c_l (d chi)^T gamma chi
(Eq. AtomicForce, Sec. 2.1).  The kinetic part is assembled as a Kronecker sum of 1D circulant
FD matrices, independently of the matrix-free stencil loops in sq_oracle.c.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import oracle


def circulant_second_derivative(n, h, c):
    """n x n periodic matrix of the central FD second derivative with weights c_0..c_p."""
    col = np.zeros(n)
    for j, cj in enumerate(c):
        if j == 0:
            col[0] += cj
        else:
            col[j % n] += cj
            col[(-j) % n] += cj
    return scipy.linalg.circulant(col) / (h * h)


def kinetic_matrix(cell):
    c = oracle.fd_coeffs(cell.fd_order)
    n1, n2, n3 = (int(x) for x in cell.n)
    h = cell.box / cell.n
    D = [circulant_second_derivative(int(cell.n[a]), h[a], c) for a in range(3)]
    I1, I2, I3 = np.eye(n1), np.eye(n2), np.eye(n3)
    # index q = i1 + n1 (i2 + n2 i3): kron(axis3, axis2, axis1)
    lap = (np.kron(I3, np.kron(I2, D[0])) + np.kron(I3, np.kron(D[1], I1)) +
           np.kron(D[2], np.kron(I2, I1)))
    return -0.5 * lap


def hamiltonian(cell, chi=None):
    """Full periodic H = -1/2 Lap_h + diag(V_eff) + sum_J sum_lm c_l dV chi chi^T."""
    H = kinetic_matrix(cell)
    H[np.diag_indices_from(H)] += cell.veff.reshape(-1)
    if cell.natom:
        chi = oracle.projectors(cell) if chi is None else chi
        dV = float(np.prod(cell.box / cell.n))
        for J in range(cell.natom):
            for lm in range(chi.shape[1]):
                cl = cell.proj_energy[0 if lm == 0 else 1]
                H += cl * dV * np.outer(chi[J, lm], chi[J, lm])
    return H


def fermi_level_exact(evals, kT, N_e):
    lo, hi = float(evals.min()) - 50 * kT, float(evals.max()) + 50 * kT
    for _ in range(300):
        mid = lo + 0.5 * (hi - lo)
        if mid <= lo or mid >= hi:
            break
        if 2.0 * oracle.fermi(evals, mid, kT).sum() < N_e:
            lo = mid
        else:
            hi = mid
    return lo + 0.5 * (hi - lo)


def solve(cell, force=True):
    """Exact (dense) finite-temperature solution for a tiny cell."""
    chi, dchi = oracle.projectors(cell, grad=True) if cell.natom else (None, None)
    H = hamiltonian(cell, chi)
    evals, U = np.linalg.eigh(H)
    lam_f = fermi_level_exact(evals, cell.kT, cell.N_e)
    g = oracle.fermi(evals, lam_f, cell.kT)
    dV = float(np.prod(cell.box / cell.n))
    rho_q = 2.0 * (U * U) @ g
    out = dict(evals=evals, lam_f=lam_f, rho=rho_q / dV, U=2.0 * float(np.dot(evals, g)),
               S=-2.0 * float(oracle.entropy_density(evals, lam_f, cell.kT).sum()), dV=dV)
    out["F"] = out["U"] - cell.kT * out["S"]
    if force and cell.natom:
        gamma = (U * g) @ U.T
        f = np.zeros((cell.natom, 3))
        for J in range(cell.natom):
            for lm in range(chi.shape[1]):
                cl = cell.proj_energy[0 if lm == 0 else 1]
                gchi = gamma @ chi[J, lm]
                for d in range(3):
                    f[J, d] += 4.0 * dV * cl * float(dchi[J, lm, d] @ gchi)
        out["force"] = f
    return out


def cube_moments(cell, q, omega, tau, K):
    """mu_k^q = sum_i U_ci^2 T_k(lambda_i) from the eigendecomposition of the dense cube operator
    Hhat_q = P_q Hhat P_q (principal submatrix of the full scaled H)."""
    H = hamiltonian(cell)
    gidx = oracle.cube_indices(cell, q)
    Hq = (H[np.ix_(gidx, gidx)] - omega * np.eye(gidx.size)) / tau
    lam, U = np.linalg.eigh(Hq)
    centre = int(np.flatnonzero(gidx == q)[0])
    w = U[centre] ** 2
    lam = np.clip(lam, -1.0, 1.0)
    return np.array([float(np.dot(w, np.cos(k * np.arccos(lam)))) for k in range(K + 1)]), lam
