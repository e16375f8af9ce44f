"""The Gauss (Lanczos) quadrature path on the GPU (sq_density with SQ_GAUSS; Sec. 2.2 "Spectral Gauss
quadrature", Eq. Lanczos, Eq. Ne, Eqs. rhoq, uq, sq) against the oracle's Gauss path on the same
seeded inputs.  Tolerances: FP64 -- lambda_f 1e-12, rho and U, S 1e-10 relative (rho per point
relative to max rho); FP32 -- the errors FP32 Lanczos vectors allow, stated per test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle  # noqa: E402
from paper_2011_13517_gb300 import cells, sq  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def gauss_gpu(cell, precision, bounds, K=None):
    h = sq.build_for_cell(cell, bounds=bounds)
    rho = torch.empty(cell.N_d, dtype=torch.float64, device="cuda")
    lam = sq.sq_density(h, cell.K if K is None else K, cell.kT, cell.N_e, precision, sq.SQ_GAUSS, rho)
    U, S, F = sq.sq_energy(h)
    name = sq.sq_kernel_name(h)
    h.close()
    return dict(lam_f=lam, U=U, S=S, rho=rho.cpu().numpy(), kernel=name)


@pytest.mark.parametrize("maker", [
    lambda: cells.tiny_cell(),
    lambda: cells.make_cell("g1", (2, 1, 1), 0.6, 12, 1, 2.4, 16, 0.01, seed=4),
    lambda: cells.make_cell("g2", (2, 1, 2), 0.9, 8, 1, 3.0, 24, 0.01, seed=6),
])
def test_gauss_fp64_matches_oracle(maker):
    c = maker()
    ref = oracle.gauss_solve(c)
    got = gauss_gpu(c, sq.SQ_FP64, (ref["lmin"], ref["lmax"]))
    assert got["kernel"] == "lanczos_kernel<double>"
    assert abs(got["lam_f"] - ref["lam_f"]) < 1e-12
    np.testing.assert_allclose(got["rho"], ref["rho"], rtol=0, atol=1e-10 * np.abs(ref["rho"]).max())
    assert abs(got["U"] - ref["U"]) < 1e-10 * max(1.0, abs(ref["U"]))
    assert abs(got["S"] - ref["S"]) < 1e-10 * max(1.0, abs(ref["S"]))
    assert abs(got["rho"].sum() * ref["dV"] - c.N_e) < 1e-9 * c.N_e


def test_gauss_fp64_vacancy_sampled_columns_and_properties():
    """95-atom vacancy cell, 25^3 cubes, K = 60: the Lanczos coefficients' Gauss rules of sampled
    columns against the oracle (through the density those columns get at the GPU's Fermi level), and
    the sum rule."""
    c = cells.vacancy_cell()
    lo, hi = oracle.spectral_bounds(c)
    got = gauss_gpu(c, sq.SQ_FP64, (lo, hi))
    omega, tau = oracle.scale_shift(lo, hi)
    cols = cells.sample_columns(c, 24)
    a, b = oracle.lanczos(c, omega, tau, cols=cols)
    nodes, w = oracle.gauss_rule(a, b, omega, tau)
    dV = float(np.prod(c.h))
    rho_ref = 2.0 * np.sum(w * oracle.fermi(nodes, got["lam_f"], c.kT), axis=1) / dV
    np.testing.assert_allclose(got["rho"][cols], rho_ref, rtol=0, atol=1e-10 * np.abs(got["rho"]).max())
    assert abs(got["rho"].sum() * dV - c.N_e) < 1e-9 * c.N_e
    assert got["S"] > 0


def test_gauss_fp32_within_stated_error():
    """FP32 Lanczos vectors (FP64 dots and Jacobi eigensolve) on a 48-site cell with 21^3 cubes, K = 24,
    against the FP64 GPU Gauss path: lambda_f within 1e-6 Ha, rho within 1e-5 of max rho, U within 1e-5
    Ha per atom."""
    c = cells.make_cell("g32", (3, 2, 2), 0.5, 12, 1, 5.0, 24, 0.005, seed=9, n_vacancy=1)
    lo, hi = oracle.spectral_bounds(c)
    g64 = gauss_gpu(c, sq.SQ_FP64, (lo, hi))
    g32 = gauss_gpu(c, sq.SQ_FP32, (lo, hi))
    print("Gauss FP32 vs FP64:", abs(g32["lam_f"] - g64["lam_f"]), np.abs(g32["rho"] - g64["rho"]).max(),
          abs(g32["U"] - g64["U"]) / c.natom)
    assert abs(g32["lam_f"] - g64["lam_f"]) < 1e-6
    assert np.abs(g32["rho"] - g64["rho"]).max() < 1e-5 * np.abs(g64["rho"]).max()
    assert abs(g32["U"] - g64["U"]) / c.natom < 1e-5


def test_gauss_rejects_force_and_reports_state():
    c = cells.tiny_cell()
    h = sq.build_for_cell(c)
    rho = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SQError) as ei:
        sq.sq_density(h, c.K, c.kT, c.N_e, sq.SQ_FP64, sq.SQ_GAUSS | sq.SQ_WANT_FORCE, rho)
    assert ei.value.status == 1
    sq.sq_density(h, c.K, c.kT, c.N_e, sq.SQ_FP64, sq.SQ_GAUSS, rho)
    f = torch.empty((c.natom, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SQError) as ei:
        sq.sq_nonlocal_force(h, f)
    assert ei.value.status == 8
    ref = oracle.gauss_solve(c, bounds=sq.sq_get_spectral_bounds(h))
    lam2 = sq.sq_fermi_resolve(h, 0.02, 20.0, rho)    # re-solve over the stored nodes
    exp = oracle.gauss_fermi_level(ref["nodes"], ref["weights"], 0.02, 20.0, ref["lmin"], ref["lmax"])
    assert abs(lam2 - exp) < 1e-12
    h.close()
