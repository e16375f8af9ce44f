"""Seeded synthetic hcp Mg/Al-like cells: the inputs of the spectral-quadrature (SQ) path.

This module only *generates inputs* (atom positions, the local effective potential V_eff on the
finite-difference grid, projector parameters, and the run parameters R_cut, K, kT, N_e).  It holds
none of the SQ method's arithmetic, so both the FP64 CPU oracle and the CUDA path consume exactly
the same arrays.

The paper studies hcp Mg with Al solutes and vacancies (Sec. 4, Sec. 5) using Troullier-Martins
pseudopotentials and self-consistent potentials, neither of which is available here.  These cells
stand in for the shapes and sizes of those systems:

* hcp lattice a = 6.06 bohr, c = 1.624 a, orthohexagonal 4-site cell with fractional basis
  (0,0,0), (1/2,1/2,0), (0,1/3,1/2), (1/2,5/6,1/2) in the box (a, a*sqrt(3), c).  An "A x B x C"
  primitive replication is the orthohexagonal box (A a, (B/2) a sqrt(3), C c).
* regular periodic grid n_i = round(L_i / h), h_i = L_i / n_i (Sec. 3, "Discretization").
* V_eff = sum over atoms (and periodic images) of Gaussian wells depth * exp(-r^2 / (2 w^2)),
  plus a smooth seeded noise field made of the periodic Fourier modes with |k_i| <= 2, rescaled so
  that its maximum magnitude on the grid equals the stated amplitude.
* Kleinman-Bylander projectors (Sec. 2.1): Gaussian s (and p_x, p_y, p_z) of width sigma with
  energy c_l; their shape is fixed by the library and the oracle, only the parameters live here.
* seeds: numpy PCG64; stream 0 = atom displacements, 1 = noise, 2 = defect sites.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np

A_MG = 6.06
C_OVER_A = 1.624
HCP_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.0, 1.0 / 3.0, 0.5], [0.5, 5.0 / 6.0, 0.5]])

MG, AL = 0, 1
WELL_DEPTH = {MG: -1.2, AL: -1.5}
VALENCE = {MG: 2, AL: 3}


@dataclasses.dataclass
class Cell:
    """One SQ problem instance: grid, V_eff, atoms, projectors and run parameters."""

    name: str
    box: np.ndarray          # (3,) bohr, periodic
    n: np.ndarray            # (3,) int grid points per axis; h_i = box_i / n_i
    fd_order: int            # even finite-difference order n_o of the Laplacian
    R: np.ndarray            # (natom, 3) bohr
    species: np.ndarray      # (natom,) MG / AL
    veff: np.ndarray         # (n3, n2, n1) float64, x fastest
    lmax: int                # 0: s projector only, 1: s + p_x, p_y, p_z
    proj_sigma: float        # Gaussian width of the projectors (bohr)
    proj_rc: float           # support half-width of the projector window (bohr)
    proj_energy: np.ndarray  # (lmax+1,) KB energies c_l (Ha)
    R_cut: float             # half-width of the truncation cube (bohr)
    K: int                   # Chebyshev polynomial order
    kT: float                # electronic smearing k_B theta (Ha)
    N_e: float               # electron count

    @property
    def h(self) -> np.ndarray:
        return self.box / self.n

    @property
    def N_d(self) -> int:
        return int(np.prod(self.n))

    @property
    def natom(self) -> int:
        return int(self.R.shape[0])

    @property
    def m(self) -> np.ndarray:
        """Cube half-widths in grid points, m_i = round(R_cut / h_i)."""
        return np.array([int(round(self.R_cut / hi)) for hi in self.h])

    @property
    def n_c(self) -> np.ndarray:
        return 2 * self.m + 1

    def digest(self) -> str:
        """Short hash of the inputs, to detect generator drift between machines.  Floating-point
        arrays enter through sums, sums of squares and a few sampled values rounded to 10
        significant digits, so last-ulp differences of the platform's libm do not change it."""
        def sig(x):
            return float(f"{float(x):.10g}")
        v = self.veff.reshape(-1)
        picks = np.linspace(0, v.size - 1, 16).astype(np.int64)
        key = (tuple(int(x) for x in self.n), tuple(sig(x) for x in self.box), self.natom,
               tuple(int(x) for x in self.species), sig(self.R.sum()), sig((self.R ** 2).sum()),
               sig(v.sum()), sig((v * v).sum()), tuple(sig(v[i]) for i in picks),
               tuple(sig(x) for x in self.proj_energy), self.fd_order, self.lmax, self.proj_sigma,
               self.proj_rc, self.R_cut, self.K, self.kT, self.N_e)
        return hashlib.sha256(repr(key).encode()).hexdigest()[:16]


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, stream]))


def hcp_sites(reps, a=A_MG, c_over_a=C_OVER_A):
    """Ideal hcp sites of an orthohexagonal supercell with reps = (nx, ny, nz) 4-site cells."""
    a_vec = np.array([a, a * math.sqrt(3.0), a * c_over_a])
    sites = []
    for iz in range(reps[2]):
        for iy in range(reps[1]):
            for ix in range(reps[0]):
                for b in HCP_BASIS:
                    sites.append((np.array([ix, iy, iz]) + b) * a_vec)
    box = a_vec * np.asarray(reps)
    return np.array(sites), box


def _periodic_gauss_1d(x, centre, L, width):
    """sum_n exp(-(x - centre - n L)^2 / (2 width^2)) over enough images."""
    nimg = int(math.ceil(10.0 * width / L)) + 1
    out = np.zeros_like(x)
    for im in range(-nimg, nimg + 1):
        t = x - centre - im * L
        out += np.exp(-t * t / (2.0 * width * width))
    return out


def make_veff(box, n, R, depths, width, noise_amp, seed):
    """V_eff on the grid: periodic Gaussian wells + smooth seeded noise (Ha)."""
    h = box / n
    axes = [np.arange(n[i]) * h[i] for i in range(3)]
    v = np.zeros((n[2], n[1], n[0]))
    for J in range(R.shape[0]):
        gx = _periodic_gauss_1d(axes[0], R[J, 0], box[0], width)
        gy = _periodic_gauss_1d(axes[1], R[J, 1], box[1], width)
        gz = _periodic_gauss_1d(axes[2], R[J, 2], box[2], width)
        v += depths[J] * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    if noise_amp > 0.0:
        rng = _rng(seed, 1)
        noise = np.zeros_like(v)
        Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        for k1 in range(-2, 3):
            for k2 in range(-2, 3):
                for k3 in range(-2, 3):
                    if (k1, k2, k3) == (0, 0, 0):
                        continue
                    amp = rng.standard_normal()
                    phase = rng.uniform(0.0, 2.0 * math.pi)
                    arg = 2.0 * math.pi * (k1 * X / box[0] + k2 * Y / box[1] + k3 * Z / box[2])
                    noise += amp * np.cos(arg + phase)
        noise *= noise_amp / np.max(np.abs(noise))
        v += noise
    return v


def make_cell(name, reps, h, fd_order, lmax, R_cut, K, kT, *, seed=0, displace=0.05,
              n_vacancy=0, divacancy=False, n_al=0, noise_amp=0.02, well_width=1.1,
              proj_sigma=1.0, proj_rc=5.0, proj_energy=0.3, grid=None):
    """Build a seeded synthetic hcp cell.

    reps: orthohexagonal replication (4 sites per cell).  n_vacancy sites are removed (as an
    adjacent pair when divacancy), n_al further sites become Al-like solutes.  grid overrides the
    n_i = round(L_i/h) rule (used for lattice-commensurate symmetry tests).
    """
    sites, box = hcp_sites(reps)
    nsite = sites.shape[0]
    species = np.full(nsite, MG)
    keep = np.ones(nsite, dtype=bool)
    rng_def = _rng(seed, 2)
    if n_vacancy:
        first = int(rng_def.integers(nsite))
        removed = [first]
        if divacancy:
            d = sites - sites[first]
            d -= np.round(d / box) * box
            dist = np.linalg.norm(d, axis=1)
            dist[first] = np.inf
            nn = np.flatnonzero(dist < dist.min() + 1e-6)
            removed.append(int(rng_def.choice(nn)))
        else:
            while len(removed) < n_vacancy:
                s = int(rng_def.integers(nsite))
                if s not in removed:
                    removed.append(s)
        keep[removed] = False
    if n_al:
        candidates = np.flatnonzero(keep)
        al = rng_def.choice(candidates, size=n_al, replace=False)
        species[al] = AL
    sites = sites[keep]
    species = species[keep]
    if displace > 0.0:
        sites = sites + displace * _rng(seed, 0).standard_normal(sites.shape)
    sites = np.mod(sites, box)
    if grid is None:
        n = np.array([int(round(box[i] / h)) for i in range(3)])
    else:
        n = np.asarray(grid, dtype=int)
    depths = np.array([WELL_DEPTH[int(s)] for s in species])
    veff = make_veff(box, n, sites, depths, well_width, noise_amp, seed)
    N_e = float(sum(VALENCE[int(s)] for s in species))
    return Cell(name=name, box=box, n=n, fd_order=fd_order, R=sites, species=species, veff=veff,
                lmax=lmax, proj_sigma=proj_sigma, proj_rc=proj_rc,
                proj_energy=np.full(lmax + 1, proj_energy), R_cut=R_cut, K=K, kT=kT, N_e=N_e)


# --- the workloads -------------------------------------------------------------------------

def tiny_cell(seed=0):
    """2x2x1 hcp (8 atoms), h=0.7 (17x15x14 grid), 6th-order FD, s projector, R_cut=3.5 (11^3
    cube), K=20, kT=0.01 Ha."""
    return make_cell("tiny_8atom", (2, 1, 1), 0.7, 6, 0, 3.5, 20, 0.01, seed=seed)


def vacancy_cell(seed=0):
    """4x4x3 hcp, 96 sites minus one seeded vacancy (95 atoms), h=0.5 (48x42x59 grid), 12th-order
    FD, s+p projectors, R_cut=6 (25^3 cube), K=60, kT=0.005 Ha."""
    return make_cell("vacancy_95atom", (4, 2, 3), 0.5, 12, 1, 6.0, 60, 0.005, seed=seed,
                     n_vacancy=1)


def precision_cell(seed=0):
    """6x6x4 hcp, 288 sites, seeded divacancy and 2 Al-like solutes (286 atoms), h=0.5 (73x63x79
    grid), 12th-order FD, s+p projectors, R_cut=7 (29^3 cube), K=80, kT=0.005 Ha."""
    return make_cell("precision_286atom", (6, 3, 4), 0.5, 12, 1, 7.0, 80, 0.005, seed=seed,
                     n_vacancy=2, divacancy=True, n_al=2)


def batch_cells(count=32, seed=0):
    """Independent defect cells of uneven size: orthohexagonal reps from 3x2x2 (48 sites) to
    6x3x4 (288 sites), 0-2 vacancies, 0-2 Al, R_cut in {5,6,7}, K in {40,60,80}; other parameters
    as the vacancy cell."""
    rng = _rng(seed, 7)
    cells = []
    for b in range(count):
        reps = (int(rng.integers(3, 7)), int(rng.integers(2, 4)), int(rng.integers(2, 5)))
        nvac = int(rng.integers(0, 3))
        nal = int(rng.integers(0, 3))
        rcut = float(rng.choice([5.0, 6.0, 7.0]))
        K = int(rng.choice([40, 60, 80]))
        cells.append(make_cell(f"batch_{b}", reps, 0.5, 12, 1, rcut, K, 0.005, seed=seed * 1000 + b,
                               n_vacancy=nvac, n_al=nal))
    return cells


def sample_columns(cell: Cell, count: int, seed: int = 11) -> np.ndarray:
    """Seeded sample of grid-point (column) indices, always including the first and last."""
    rng = _rng(seed, 3)
    cols = rng.choice(cell.N_d, size=min(count, cell.N_d), replace=False)
    cols = np.unique(np.concatenate([cols, [0, cell.N_d - 1]]))
    return cols.astype(np.int64)
