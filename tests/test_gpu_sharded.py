"""The column-range (sharded) form of the path on the GPU: the grid split into ranges, each range's
recursion by sq_moments_range, the moment sums added on the host (the one global reduction of
Eq. Ne), the Fermi level from the pure host sq_fermi_level, and each range's density, energy and
forces from sq_observables -- against the oracle and against the whole-grid sq_density."""
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


def sharded_solve(cell, bounds, precision, nshards):
    """Emulates nshards ranks one after another in this process (one handle per rank)."""
    lo, hi = bounds
    omega, tau = 0.5 * (hi + lo), 0.5 * (hi - lo)
    edges = np.linspace(0, cell.N_d, nshards + 1).astype(np.int64)
    handles, msum, A = [], 0.0, 0.0
    for r in range(nshards):
        h = sq.build_for_cell(cell, bounds=bounds)
        m, a = sq.sq_moments_range(h, cell.K, precision, sq.SQ_WANT_FORCE, edges[r], edges[r + 1])
        handles.append(h)
        msum = msum + m
        A = A + a
    lam = sq.sq_fermi_level(msum, cell.K, omega, tau, lo, hi, cell.kT, cell.N_e)
    rho = torch.empty(cell.N_d, dtype=torch.float64, device="cuda")
    force = torch.empty((cell.natom, 3), dtype=torch.float64, device="cuda")
    out = {}
    for r, h in enumerate(handles):
        sq.sq_observables(h, lam, cell.kT, cell.N_e, msum, A, rho[edges[r]:edges[r + 1]])
        U, S, F = sq.sq_energy(h)
        sq.sq_nonlocal_force(h, force)
        out.setdefault("U", []).append(U)
        out.setdefault("S", []).append(S)
        out.setdefault("force", []).append(force.cpu().numpy().copy())
        h.close()
    torch.cuda.synchronize()
    return dict(lam_f=lam, Msum=msum, rho=rho.cpu().numpy(), U=out["U"], S=out["S"], force=out["force"])


def test_sharded_tiny_cell_fp64_matches_oracle():
    c = cells.tiny_cell()
    ref = oracle.sq_solve(c, force=True)
    got = sharded_solve(c, (ref["lmin"], ref["lmax"]), sq.SQ_FP64, 3)
    assert abs(got["lam_f"] - ref["lam_f"]) < 1e-12
    np.testing.assert_allclose(got["Msum"], ref["Msum"], rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(got["rho"], ref["rho"], rtol=1e-10, atol=1e-10 * np.abs(ref["rho"]).max())
    fs = np.abs(ref["force"]).max()
    for U, S, f in zip(got["U"], got["S"], got["force"]):   # every rank reports the global values
        assert abs(U - ref["U"]) < 1e-10 * abs(ref["U"]) and abs(S - ref["S"]) < 1e-10 * abs(ref["S"])
        np.testing.assert_allclose(f, ref["force"], rtol=0, atol=1e-9 * fs)


def test_sharded_vacancy_fp32_equals_whole_grid():
    """FP32 slab kernel on ranges of the 95-atom cell (K = 12): the same moments as the whole-grid
    call, so lambda_f, rho and forces agree to FP64 summation-order rounding."""
    c = cells.vacancy_cell()
    c.K = 12
    lo, hi = oracle.spectral_bounds(c)
    got = sharded_solve(c, (lo, hi), sq.SQ_FP32, 2)
    whole = sq.solve_cell(c, sq.SQ_FP32, force=True, bounds=(lo, hi))
    assert abs(got["lam_f"] - whole["lam_f"]) < 1e-11
    np.testing.assert_allclose(got["Msum"], whole["Msum"], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(got["rho"], whole["rho"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(got["force"][0], whole["force"], rtol=0, atol=1e-10)


def test_sharded_calls_reject_bad_ranges_and_order():
    c = cells.tiny_cell()
    h = sq.build_for_cell(c)
    with pytest.raises(sq.SQError) as ei:
        sq.sq_moments_range(h, c.K, sq.SQ_FP64, 0, 10, 5)
    assert ei.value.status == 1
    with pytest.raises(sq.SQError) as ei:
        sq.sq_moments_range(h, c.K, sq.SQ_FP64, 0, 0, c.N_d + 1)
    assert ei.value.status == 1
    h.K, h.range = c.K, (0, c.N_d)
    with pytest.raises(sq.SQError) as ei:   # observables before any moments
        sq.sq_observables(h, 0.1, c.kT, c.N_e, np.ones(c.K + 1))
    assert ei.value.status == 8
    sq.sq_moments_range(h, c.K, sq.SQ_FP64, 0, 0, 100)
    vbar = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SQError) as ei:   # the derivative needs the whole grid
        sq.sq_density_vjp(h, vbar, 0.0, 1, vbar)
    assert ei.value.status == 8
    h.close()


def test_fma_probe_reports_the_pipes():
    t32, ms32 = sq.sq_fma_throughput(sq.SQ_FP32)
    t64, ms64 = sq.sq_fma_throughput(sq.SQ_FP64)
    print(f"FMA ceilings: FP32 {t32:.1f} TFLOP/s ({ms32:.1f} ms), FP64 {t64:.2f} TFLOP/s ({ms64:.1f} ms)")
    assert 10.0 < t32 < 200.0 and 0.1 < t64 < t32 and ms32 > 10 and ms64 > 10
    tf, mtf = sq.sq_mma_throughput(0)
    bf, mbf = sq.sq_mma_throughput(1)
    print(f"warp-level MMA: TF32 m16n8k8 {tf:.1f} TFLOP/s ({mtf:.1f} ms), BF16 m16n8k16 {bf:.1f} TFLOP/s ({mbf:.1f} ms)")
    assert tf > 1.0 and bf > 1.0 and mtf > 10 and mbf > 10
