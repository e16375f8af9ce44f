"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded
inputs.  Tolerances: FP64 recursion -- rho, U, S within 1e-10 relative, lambda_f within 1e-12
absolute, forces within 1e-9 of the largest force component, moments within 1e-12 absolute
(|mu_k| <= 1).  FP32 recursion -- the errors the arithmetic allows (see the FP32 tests)."""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle  # noqa: E402
from paper_2011_13517_gb300 import cells, sq  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def check_fp64(gpu, ref, cell, mu_cols=None):
    assert abs(gpu["lam_f"] - ref["lam_f"]) < 1e-12
    rho_scale = np.max(np.abs(ref["rho"]))
    np.testing.assert_allclose(gpu["rho"], ref["rho"], rtol=1e-10, atol=1e-10 * rho_scale)
    assert rel(gpu["U"], ref["U"]) < 1e-10
    assert rel(gpu["S"], ref["S"]) < 1e-10
    np.testing.assert_allclose(gpu["Msum"], ref["Msum"], rtol=1e-11, atol=1e-11 * cell.N_d)
    if mu_cols is None:
        np.testing.assert_allclose(gpu["mu"].T, ref["mu"], rtol=0, atol=1e-12)
    if "force" in ref:
        fs = np.max(np.abs(ref["force"]))
        np.testing.assert_allclose(gpu["force"], ref["force"], rtol=0, atol=1e-9 * fs)


# ---------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny():
    c = cells.tiny_cell()
    return c, oracle.sq_solve(c, force=True)


def test_library_bounds_match_oracle(tiny):
    c, ref = tiny
    h = sq.build_for_cell(c)
    lo, hi = sq.sq_get_spectral_bounds(h)
    h.close()
    assert rel(lo, ref["lmin"]) < 1e-12 and rel(hi, ref["lmax"]) < 1e-12
    assert sq.sq_get_cube(sq.build_for_cell(c)) == tuple(int(x) for x in c.m)


def test_tiny_cell_fp64_matches_oracle(tiny):
    """8-atom cell, 17x15x14 grid, 11^3 cubes (ragged against the 8-point x segments), K = 20, s
    projectors: every moment of every column, rho, lambda_f, U, S and forces."""
    c, ref = tiny
    gpu = sq.solve_cell(c, sq.SQ_FP64, force=True, bounds=(ref["lmin"], ref["lmax"]))
    check_fp64(gpu, ref, c)
    assert abs(gpu["rho"].sum() * ref["dV"] - c.N_e) < 1e-10 * c.N_e


def test_tiny_cell_fp64_is_deterministic(tiny):
    c, ref = tiny
    a = sq.solve_cell(c, sq.SQ_FP64, force=False, bounds=(ref["lmin"], ref["lmax"]))
    b = sq.solve_cell(c, sq.SQ_FP64, force=False, bounds=(ref["lmin"], ref["lmax"]))
    assert np.array_equal(a["rho"], b["rho"]) and a["lam_f"] == b["lam_f"] and a["U"] == b["U"]


@pytest.mark.parametrize("lmax,fd,reps,h,rcut", [(1, 6, (2, 1, 1), 0.7, 3.5), (1, 12, (2, 1, 1), 0.6, 2.4),
                                                (0, 2, (1, 1, 1), 0.8, 2.0), (1, 8, (2, 1, 2), 0.9, 3.0)])
def test_small_cells_fp64_match_oracle(lmax, fd, reps, h, rcut):
    """Several shapes: s and s+p projectors, FD orders 2-12, cubes from 5^3 to 11^3, boxes where the
    projector support wraps around the periodic cell."""
    c = cells.make_cell("var", reps, h, fd, lmax, rcut, 17, 0.02, seed=5)
    ref = oracle.sq_solve(c, force=True)
    gpu = sq.solve_cell(c, sq.SQ_FP64, force=True, bounds=(ref["lmin"], ref["lmax"]))
    check_fp64(gpu, ref, c)


def test_no_atoms_free_electron_fp64():
    """V = 0, no projectors: every cube is the same operator, so rho = N_e / (N_d dV) everywhere."""
    c = cells.make_cell("free", (2, 1, 1), 0.7, 6, 0, 3.5, 20, 0.01, noise_amp=0.0)
    c.veff = np.zeros_like(c.veff)
    c.R = np.zeros((0, 3))
    c.species = np.zeros(0, dtype=int)
    ref = oracle.sq_solve(c, force=False)
    gpu = sq.solve_cell(c, sq.SQ_FP64, force=False, bounds=(ref["lmin"], ref["lmax"]))
    check_fp64(gpu, ref, c)
    np.testing.assert_allclose(gpu["rho"], c.N_e / (c.N_d * ref["dV"]), rtol=1e-10)


# ---------------------------------------------------------------------------------------------
# full-size vacancy cell (118,944 columns, 25^3 cubes, K = 60, s+p projectors)

@pytest.fixture(scope="module")
def vacancy():
    c = cells.vacancy_cell()
    lo, hi = oracle.spectral_bounds(c)
    gpu = sq.solve_cell(c, sq.SQ_FP64, force=True, bounds=(lo, hi))
    return c, (lo, hi), gpu


def test_vacancy_fp64_sampled_columns_match_oracle(vacancy):
    """Moments of 34 sampled columns (first and last included) against the oracle, element by
    element, at the full size and in the same launch configuration as the benchmark."""
    c, (lo, hi), gpu = vacancy
    omega, tau = oracle.scale_shift(lo, hi)
    cols = cells.sample_columns(c, 32)
    mu = oracle.moments(c, omega, tau, cols=cols)
    np.testing.assert_allclose(gpu["mu"][:, cols].T, mu, rtol=0, atol=1e-12)


def test_vacancy_fp64_properties(vacancy):
    c, (lo, hi), gpu = vacancy
    dV = float(np.prod(c.h))
    assert abs(gpu["rho"].sum() * dV - c.N_e) < 1e-10 * c.N_e
    assert gpu["S"] >= 0.0
    assert np.all(np.abs(gpu["mu"]) <= 1.0 + 1e-12)
    assert np.all(gpu["mu"][0] == 1.0)


def test_vacancy_fp64_matches_golden(vacancy):
    """lambda_f, U, S, F, forces and sampled rho against the oracle's full-size run
    (tests/golden/vacancy_95atom.json, written by tests/golden/make_golden.py)."""
    path = os.path.join(GOLDEN, "vacancy_95atom.json")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    c, (lo, hi), gpu = vacancy
    g = json.load(open(path))
    assert g["digest"] == c.digest(), "input generator drift"
    assert abs(gpu["lam_f"] - g["lam_f"]) < 1e-12
    assert rel(gpu["U"], g["U"]) < 1e-10 and rel(gpu["S"], g["S"]) < 1e-10
    np.testing.assert_allclose(gpu["Msum"], g["Msum"], rtol=1e-11, atol=1e-11 * c.N_d)
    idx = np.array(g["rho_idx"])
    rs = np.max(np.abs(g["rho"]))
    np.testing.assert_allclose(gpu["rho"][idx], g["rho"], rtol=1e-10, atol=1e-10 * rs)
    f = np.array(g["force"])
    np.testing.assert_allclose(gpu["force"], f, rtol=0, atol=1e-9 * np.max(np.abs(f)))


# ---------------------------------------------------------------------------------------------
# FP32 recursion: stated error bounds

def fp32_errors(gpu, ref, cell):
    dV = float(np.prod(cell.h))
    out = dict(
        rho_l1=float(np.sum(np.abs(gpu["rho"] - ref["rho"])) * dV / cell.N_e),
        rho_max_rel=float(np.max(np.abs(gpu["rho"] - ref["rho"])) / np.max(np.abs(ref["rho"]))),
        dU_per_atom=abs(gpu["U"] - ref["U"]) / max(cell.natom, 1),
        dlam=abs(gpu["lam_f"] - ref["lam_f"]),
        mu_max=float(np.max(np.abs(gpu["mu"].T - ref["mu"]))),
    )
    if "force" in ref:
        out["df_max"] = float(np.max(np.abs(gpu["force"] - ref["force"])))
    return out


def test_tiny_cell_fp32_within_stated_error(tiny):
    c, ref = tiny
    gpu = sq.solve_cell(c, sq.SQ_FP32, force=True, bounds=(ref["lmin"], ref["lmax"]))
    e = fp32_errors(gpu, ref, c)
    print("FP32 tiny errors", e)
    assert e["mu_max"] < 5e-7          # observed 1.1e-7
    assert e["rho_l1"] < 1e-5 and e["dU_per_atom"] < 1e-5 and e["dlam"] < 1e-5
    assert e["df_max"] < 1e-5
    assert abs(gpu["rho"].sum() * ref["dV"] - c.N_e) < 1e-9 * c.N_e


def test_vacancy_fp32_sampled_columns(vacancy):
    """FP32 recursion (the 25^3 slab kernel) at full size: sampled moments against the oracle
    (~1e-7 per moment: K = 60 steps of ~40-term FP32 sums), and lambda_f, U, forces and sampled rho
    against the oracle's full-size golden values.  The energy and force tolerances are the paper's
    accuracy targets (1e-4 Ha/atom, 1e-4 Ha/bohr; Sec. 4): the FP32 error must stay below them."""
    c, (lo, hi), _ = vacancy
    gpu = sq.solve_cell(c, sq.SQ_FP32, force=True, bounds=(lo, hi))
    omega, tau = oracle.scale_shift(lo, hi)
    cols = cells.sample_columns(c, 16)
    mu = oracle.moments(c, omega, tau, cols=cols)
    err = float(np.max(np.abs(gpu["mu"][:, cols].T - mu)))
    print("FP32 vacancy max moment error", err)
    assert err < 5e-7                  # observed 8.5e-8 (K = 60)
    dV = float(np.prod(c.h))
    assert abs(gpu["rho"].sum() * dV - c.N_e) < 1e-9 * c.N_e
    path = os.path.join(GOLDEN, "vacancy_95atom.json")
    if os.path.exists(path):
        g = json.load(open(path))
        idx = np.array(g["rho_idx"])
        e = dict(dlam=abs(gpu["lam_f"] - g["lam_f"]), dU_atom=abs(gpu["U"] - g["U"]) / c.natom,
                 rho_rel=float(np.max(np.abs(gpu["rho"][idx] - g["rho"])) / np.max(np.abs(g["rho"]))),
                 df=float(np.max(np.abs(gpu["force"] - np.array(g["force"])))))
        print("FP32 vacancy errors vs oracle", e)
        assert e["dlam"] < 1e-5 and e["dU_atom"] < 1e-4 and e["rho_rel"] < 1e-4 and e["df"] < 1e-4


def test_precision_cell_fp32_against_oracle_golden():
    """FP32 recursion on the 286-atom divacancy + Al cell (73x63x79 grid, 29^3 cubes, K = 80; the
    generic column kernel): lambda_f, U, forces and sampled rho against the FP64 oracle's full-size
    golden values, within the paper's accuracy targets (1e-4 Ha/atom, 1e-4 Ha/bohr; Sec. 4), and
    sampled moments against the oracle column by column."""
    path = os.path.join(GOLDEN, "precision_286atom.json")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    g = json.load(open(path))
    c = cells.precision_cell()
    assert c.digest() == g["digest"]
    gpu = sq.solve_cell(c, sq.SQ_FP32, force=True, bounds=(g["lmin"], g["lmax"]))
    omega, tau = oracle.scale_shift(g["lmin"], g["lmax"])
    cols = cells.sample_columns(c, 4)
    mu = oracle.moments(c, omega, tau, cols=cols)
    err = float(np.max(np.abs(gpu["mu"][:, cols].T - mu)))
    print("FP32 precision-cell max moment error", err)
    assert err < 1e-6                  # K = 80 steps of FP32 sums
    idx = np.array(g["rho_idx"])
    e = dict(dlam=abs(gpu["lam_f"] - g["lam_f"]), dU_atom=abs(gpu["U"] - g["U"]) / c.natom,
             rho_rel=float(np.max(np.abs(gpu["rho"][idx] - g["rho"])) / np.max(np.abs(g["rho"]))),
             df=float(np.max(np.abs(gpu["force"] - np.array(g["force"])))))
    print("FP32 precision-cell errors vs oracle", e)
    assert e["dlam"] < 1e-5 and e["dU_atom"] < 1e-4 and e["rho_rel"] < 1e-4 and e["df"] < 1e-4


def energy_tolerance(g, kT, which):
    """Agreement two FP64 evaluations of U = 2 sum_k d_k M_k (or S = -2 sum_k e_k M_k) can reach:
    1e-10 relative, or, where the sum cancels heavily (U ~ 1 Ha from terms summing to ~3e5 Ha on
    the 286-atom cell), 1e-13 of the sum of the magnitudes of its terms -- the pointwise u^q of
    Eq. uq summed over N_d ~ 4e5 points in different orders."""
    c, d, e = sq.sq_fermi_weights(g["lam_f"], g["K"], g["omega"], g["tau"], kT)
    w = d if which == "U" else e
    return max(1e-10 * abs(g[which]), 1e-13 * 2.0 * float(np.sum(np.abs(w * np.array(g["Msum"])))))


def test_precision_cell_fp64_against_oracle_golden():
    """FP64 recursion on the 286-atom divacancy + Al cell (73x63x79 grid, 29^3 cubes, K = 80) against
    the FP64 oracle's full-size golden values: lambda_f within 1e-12, U and S within 1e-10 relative
    (or the summation-order bound of energy_tolerance where the energy sum cancels), rho within 1e-10
    relative at the 2,050 golden points, forces within 1e-9 of the largest component, and all K+1
    moments of the 34 golden columns within 1e-12."""
    path = os.path.join(GOLDEN, "precision_286atom.json")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    g = json.load(open(path))
    c = cells.precision_cell()
    assert c.digest() == g["digest"]
    gpu = sq.solve_cell(c, sq.SQ_FP64, force=True, bounds=(g["lmin"], g["lmax"]))
    assert abs(gpu["lam_f"] - g["lam_f"]) < 1e-12
    print("FP64 precision cell: dU", gpu["U"] - g["U"], "tolerance", energy_tolerance(g, c.kT, "U"),
          "dS", gpu["S"] - g["S"])
    assert abs(gpu["U"] - g["U"]) < energy_tolerance(g, c.kT, "U")
    assert abs(gpu["S"] - g["S"]) < energy_tolerance(g, c.kT, "S")
    np.testing.assert_allclose(gpu["Msum"], g["Msum"], rtol=1e-11, atol=1e-11 * c.N_d)
    idx = np.array(g["rho_idx"])
    gr = np.array(g["rho"])
    np.testing.assert_allclose(gpu["rho"][idx], gr, rtol=1e-10, atol=1e-10 * np.abs(gr).max())
    gf = np.array(g["force"])
    np.testing.assert_allclose(gpu["force"], gf, rtol=0, atol=1e-9 * np.abs(gf).max())
    np.testing.assert_allclose(gpu["mu"][:, np.array(g["mu_idx"])].T, np.array(g["mu"]), rtol=0, atol=1e-12)


def test_fp32_21_cube_matches_oracle():
    """FP32 on a 21^3 cube (R_cut = 5 bohr, the batch workload's smallest truncation): sampled
    moments of a 48-site cell against the oracle."""
    c = cells.make_cell("rc5", (3, 2, 2), 0.5, 12, 1, 5.0, 24, 0.005, seed=9, n_vacancy=1)
    assert np.all(c.n_c == 21)
    lo, hi = oracle.spectral_bounds(c)
    gpu = sq.solve_cell(c, sq.SQ_FP32, force=True, bounds=(lo, hi))
    ref64 = sq.solve_cell(c, sq.SQ_FP64, force=True, bounds=(lo, hi))
    omega, tau = oracle.scale_shift(lo, hi)
    cols = cells.sample_columns(c, 24)
    mu = oracle.moments(c, omega, tau, cols=cols)
    assert float(np.max(np.abs(gpu["mu"][:, cols].T - mu))) < 5e-7
    np.testing.assert_allclose(ref64["mu"][:, cols].T, mu, rtol=0, atol=1e-12)
    assert abs(gpu["lam_f"] - ref64["lam_f"]) < 1e-5


@pytest.mark.parametrize("kb", ["mma", "fma"])
def test_fp32_29_cube_cluster_matches_oracle(kb):
    """FP32 on 29^3 cubes (R_cut = 7 bohr), which run on the two-CTA cluster kernel, with the projector
    term on the tensor cores (3xTF32, the default) or on the CUDA cores (SQ_KB_FMA): a 48-site cell
    (36x42x39 grid) with a vacancy and an Al-like solute, K = 24.  Sampled moments against the oracle;
    every moment, rho, lambda_f and forces against the FP64 GPU path, whose moments are checked against
    the same oracle columns at 1e-12."""
    c = cells.make_cell("rc7", (3, 2, 2), 0.5, 12, 1, 7.0, 24, 0.005, seed=5, n_vacancy=1, n_al=1)
    assert np.all(c.n_c == 29)
    extra = sq.SQ_KB_FMA if kb == "fma" else 0
    lo, hi = oracle.spectral_bounds(c)
    g32 = sq.solve_cell(c, sq.SQ_FP32, force=True, bounds=(lo, hi), extra_flags=extra)
    g64 = sq.solve_cell(c, sq.SQ_FP64, force=True, bounds=(lo, hi))
    h = sq.build_for_cell(c, bounds=(lo, hi))
    rho = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    sq.sq_density(h, 2, c.kT, c.N_e, sq.SQ_FP32, extra, rho)
    assert sq.sq_kernel_name(h) == f"cluster_kernel<29,6,{kb}>"
    h.close()
    omega, tau = oracle.scale_shift(lo, hi)
    cols = cells.sample_columns(c, 48)
    mu = oracle.moments(c, omega, tau, cols=cols)
    np.testing.assert_allclose(g64["mu"][:, cols].T, mu, rtol=0, atol=1e-12)
    err_o = float(np.max(np.abs(g32["mu"][:, cols].T - mu)))
    err_all = float(np.max(np.abs(g32["mu"] - g64["mu"])))
    e = fp32_errors(g32, dict(g64, mu=g64["mu"].T), c)
    print(f"FP32 29^3 cluster kernel ({kb}): max moment error vs oracle", err_o, "vs FP64 (all columns)", err_all, e)
    assert err_o < 1e-6 and err_all < 1e-6
    assert e["dlam"] < 1e-6 and e["rho_max_rel"] < 1e-5 and e["dU_per_atom"] < 1e-5 and e["df_max"] < 1e-6
    dV = float(np.prod(c.h))
    assert abs(g32["rho"].sum() * dV - c.N_e) < 1e-9 * c.N_e


@pytest.mark.parametrize("lmax,fd,reps,h,rcut", [(0, 6, (2, 1, 1), 0.7, 3.5), (1, 12, (2, 1, 1), 0.6, 2.4),
                                                (1, 8, (2, 1, 2), 0.9, 3.0)])
def test_fd_gradient_force_fp64_matches_oracle(lmax, fd, reps, h, rcut):
    """SQ_GRAD_FD (the paper's discrete gradient nabla_h in the nonlocal force): FP64 forces against
    the oracle's FD-gradient forces at 1e-9 of the largest component, on cells whose FD reach wraps
    the periodic box; the density and energy are those of the analytic build."""
    c = cells.make_cell("gfd", reps, h, fd, lmax, rcut, 16, 0.01, seed=7)
    ref = oracle.sq_solve(c, force=True, grad_fd=True)
    gpu = sq.solve_cell(c, sq.SQ_FP64, force=True, bounds=(ref["lmin"], ref["lmax"]), grad=sq.SQ_GRAD_FD)
    fs = np.max(np.abs(ref["force"]))
    np.testing.assert_allclose(gpu["force"], ref["force"], rtol=0, atol=1e-9 * fs)
    assert abs(gpu["lam_f"] - ref["lam_f"]) < 1e-12
    ana = oracle.sq_solve(c, force=True, bounds=(ref["lmin"], ref["lmax"]))
    assert np.max(np.abs(ana["force"] - ref["force"])) > 1e-6 * fs   # the two gradients differ


@pytest.mark.parametrize("rcut", [5.0, 6.0, 7.0])
def test_fd_gradient_force_fp32_kernels(rcut):
    """SQ_GRAD_FD on the FP32 slab (21^3, 25^3) and cluster (29^3) kernels: forces against the FP64
    path with the same gradient (48-site cell, K = 12)."""
    c = cells.make_cell("gfd32", (3, 2, 2), 0.5, 12, 1, rcut, 12, 0.005, seed=12, n_vacancy=1, n_al=1)
    lo, hi = oracle.spectral_bounds(c)
    g32 = sq.solve_cell(c, sq.SQ_FP32, force=True, bounds=(lo, hi), grad=sq.SQ_GRAD_FD)
    g64 = sq.solve_cell(c, sq.SQ_FP64, force=True, bounds=(lo, hi), grad=sq.SQ_GRAD_FD)
    assert np.max(np.abs(g32["force"] - g64["force"])) < 1e-6
    assert np.max(np.abs(g32["mu"] - g64["mu"])) < 1e-6


# ---------------------------------------------------------------------------------------------
# error paths through the ABI

def test_cube_exceeding_box_is_rejected():
    c = cells.tiny_cell()
    c.R_cut = 6.0
    with pytest.raises(sq.SQError) as ei:
        sq.build_for_cell(c)
    assert ei.value.status == 2


def test_bad_arguments_and_state():
    c = cells.tiny_cell()
    h = sq.build_for_cell(c)
    rho = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SQError) as ei:
        sq.sq_energy(h)
    assert ei.value.status == 8
    with pytest.raises(sq.SQError) as ei:
        sq.sq_density(h, 0, c.kT, c.N_e, sq.SQ_FP64, 0, rho)
    assert ei.value.status == 1
    with pytest.raises(sq.SQError) as ei:
        sq.sq_density(h, c.K, -1.0, c.N_e, sq.SQ_FP64, 0, rho)
    assert ei.value.status == 1
    sq.sq_density(h, c.K, c.kT, c.N_e, sq.SQ_FP64, 0, rho)
    f = torch.empty((c.natom, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SQError) as ei:
        sq.sq_nonlocal_force(h, f)
    assert ei.value.status == 8
    # with kT far above the band width g is ~1/2 on the whole spectrum, so N(lambda_max) ~ N_d and
    # an electron count of 1.5 N_d cannot be bracketed
    with pytest.raises(sq.SQError) as ei:
        sq.sq_fermi_resolve(h, 1e4, 1.5 * c.N_d)
    assert ei.value.status == 3
    h.close()


def test_non_finite_potential_is_rejected():
    c = cells.tiny_cell()
    v = torch.from_numpy(c.veff.reshape(-1).copy()).cuda()
    v[17] = math.nan
    with pytest.raises(sq.SQError) as ei:
        sq.build_for_cell(c, d_veff=v)
    assert ei.value.status == 4


def test_fermi_level_resolve_matches_oracle(tiny):
    """sq_fermi_resolve re-solves Eq. Ne for another electron count from the stored moment sums."""
    c, ref = tiny
    h = sq.build_for_cell(c, bounds=(ref["lmin"], ref["lmax"]))
    rho = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    sq.sq_density(h, c.K, c.kT, c.N_e, sq.SQ_FP64, 0, rho)
    lam2 = sq.sq_fermi_resolve(h, 0.02, 20.0, rho)
    exp = oracle.fermi_level(ref["Msum"], ref["omega"], ref["tau"], 0.02, 20.0, ref["lmin"], ref["lmax"],
                             oracle.n_nodes(c.K, 0.02, ref["tau"]))
    assert abs(lam2 - exp) < 1e-12
    assert abs(rho.sum().item() * ref["dV"] - 20.0) < 1e-9
    h.close()
