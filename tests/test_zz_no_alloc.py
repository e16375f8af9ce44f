"""The allocation-free moments entry point against the regular path.

sq_moments_noalloc is for callers that cannot let the library allocate device memory in their
steady state -- a fixed device-memory budget handed out up front, or latency-critical loops where
cudaMalloc/cudaFree would synchronise the device.  It keeps its working vectors in a fixed device
array shared by all calls, so it must give the moments sq_density gives, call after call.  This file
is collected last so that a failure here cannot stop the other tests from running first."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2011_13517_gb300 import cells, sq  # noqa: E402

# the moment tolerances of the parity tests (|mu_k| <= 1): FP64 1e-12; FP32 1e-6 (sq_density may run
# a different FP32 kernel, so the two FP32 results agree only to FP32 rounding, ~1e-7)
ATOL = {sq.SQ_FP64: 1e-12, sq.SQ_FP32: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("cell_fn,K", [(cells.tiny_cell, None), (cells.vacancy_cell, 8)])
@pytest.mark.parametrize("precision", [sq.SQ_FP64, sq.SQ_FP32])
def test_noalloc_moments_match_density_on_two_calls(cell_fn, K, precision):
    cell = cell_fn()
    K = cell.K if K is None else K
    h = sq.build_for_cell(cell)
    rho = torch.empty(cell.N_d, dtype=torch.float64, device="cuda")
    sq.sq_density(h, K, cell.kT, cell.N_e, precision, 0, rho)
    ref, _ = sq.sq_copy_moments(h, cell.N_d)
    out = torch.empty_like(ref)
    for _ in range(2):
        out.fill_(float("nan"))
        sq.sq_moments_noalloc(h, K, precision, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        np.testing.assert_allclose(out.double().cpu().numpy(), ref.double().cpu().numpy(), rtol=0,
                                   atol=ATOL[precision])
    h.close()


def test_noalloc_rejects_a_cube_beyond_the_fixed_scratch():
    """Two FP64 vectors of a 129^3 cube (34 MB) do not fit in the 32 MiB array."""
    n = (136, 136, 136)
    L = tuple(0.5 * x for x in n)
    v = torch.zeros(int(np.prod(n)), dtype=torch.float64, device="cuda")
    h = sq.sq_build_hamiltonian(n, L, 2, v, np.zeros((0, 3)), 0, 1.0, 5.0, [0.3], 32.0)
    assert sq.sq_get_cube(h) == (64, 64, 64)
    out = torch.empty((3, v.numel()), dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SQError) as ei:
        sq.sq_moments_noalloc(h, 2, sq.SQ_FP64, out)
    assert ei.value.status == 9 and "static scratch" in str(ei.value)
    h.close()
