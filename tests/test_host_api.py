"""CPU checks of the library's host-side logic (no GPU needed):

- the pure host Fermi level (sq_fermi_level, Eq. Ne) and Chebyshev weights (sq_fermi_weights,
  Eq. ChebyshevWeights) against the oracle on the same moment sums;
- their error paths (no bracket, bad arguments);
- the binding's buffer-size checks, which run before anything reaches the library."""
import math

import numpy as np
import pytest

from oracle import oracle
from paper_2011_13517_gb300 import cells, sq


@pytest.fixture(scope="module")
def tiny_ref():
    c = cells.tiny_cell()
    return c, oracle.sq_solve(c, force=False)


def test_host_fermi_level_matches_oracle(tiny_ref):
    c, ref = tiny_ref
    lam = sq.sq_fermi_level(ref["Msum"], c.K, ref["omega"], ref["tau"], ref["lmin"], ref["lmax"], c.kT, c.N_e)
    assert abs(lam - ref["lam_f"]) < 1e-12
    # another smearing and electron count on the same sums
    M = oracle.n_nodes(c.K, 0.02, ref["tau"])
    exp = oracle.fermi_level(ref["Msum"], ref["omega"], ref["tau"], 0.02, 20.0, ref["lmin"], ref["lmax"], M)
    lam2 = sq.sq_fermi_level(ref["Msum"], c.K, ref["omega"], ref["tau"], ref["lmin"], ref["lmax"], 0.02, 20.0)
    assert abs(lam2 - exp) < 1e-12


def test_host_weights_match_oracle_and_give_the_observables(tiny_ref):
    c, ref = tiny_ref
    M = oracle.n_nodes(c.K, c.kT, ref["tau"])
    cw, dw, ew = sq.sq_fermi_weights(ref["lam_f"], c.K, ref["omega"], ref["tau"], c.kT)
    oc, od, oe = oracle.fermi_coeffs(ref["lam_f"], ref["omega"], ref["tau"], c.kT, c.K, M)
    np.testing.assert_allclose(cw, oc, rtol=0, atol=1e-13)
    np.testing.assert_allclose(dw, od, rtol=0, atol=1e-13 * max(1.0, np.abs(od).max()))
    np.testing.assert_allclose(ew, oe, rtol=0, atol=1e-13)
    assert abs(2.0 * dw @ ref["Msum"] - ref["U"]) < 1e-10 * abs(ref["U"])
    assert abs(-2.0 * ew @ ref["Msum"] - ref["S"]) < 1e-10 * abs(ref["S"])
    rho = 2.0 * (ref["mu"] @ cw) / ref["dV"]
    np.testing.assert_allclose(rho, ref["rho"], rtol=1e-11, atol=1e-13)


def test_host_fermi_full_band_weights():
    """lambda_f far above the spectrum: g = 1 on [-1, 1], so c_0 = 1 and c_k = 0 for k > 0."""
    c, _, _ = sq.sq_fermi_weights(1e3, 12, 0.0, 1.0, 0.01)
    assert abs(c[0] - 1.0) < 1e-14 and np.max(np.abs(c[1:])) < 1e-14


def test_host_fermi_errors(tiny_ref):
    c, ref = tiny_ref
    with pytest.raises(sq.SQError) as ei:   # more electrons than the band holds
        sq.sq_fermi_level(ref["Msum"], c.K, ref["omega"], ref["tau"], ref["lmin"], ref["lmax"], c.kT, 2.5 * c.N_d)
    assert ei.value.status == 3
    with pytest.raises(sq.SQError) as ei:
        sq.sq_fermi_level(ref["Msum"], c.K, ref["omega"], ref["tau"], ref["lmax"], ref["lmin"], c.kT, c.N_e)
    assert ei.value.status == 1
    bad = ref["Msum"].copy()
    bad[3] = math.nan
    with pytest.raises(sq.SQError) as ei:
        sq.sq_fermi_level(bad, c.K, ref["omega"], ref["tau"], ref["lmin"], ref["lmax"], c.kT, c.N_e)
    assert ei.value.status == 4
    with pytest.raises(ValueError):
        sq.sq_fermi_level(ref["Msum"][:5], c.K, ref["omega"], ref["tau"], ref["lmin"], ref["lmax"], c.kT, c.N_e)


def test_binding_rejects_short_output_buffers():
    """The library writes (K+1) N_d moments, N_d densities or 3 natom forces through raw pointers; a
    shorter tensor must be refused before any launch."""
    torch = pytest.importorskip("torch")
    h = sq.Handle(None, N_d=100, natom=4, nproj=4)
    with pytest.raises(ValueError, match="elements"):
        sq.sq_moments_noalloc(h, 3, sq.SQ_FP64, torch.zeros(399, dtype=torch.float64))
    with pytest.raises(ValueError, match="elements"):
        sq.sq_density(h, 3, 0.01, 8.0, sq.SQ_FP64, 0, torch.zeros(99, dtype=torch.float64))
    with pytest.raises(ValueError, match="elements"):
        sq.sq_nonlocal_force(h, torch.zeros(11, dtype=torch.float64))
    with pytest.raises(ValueError, match="elements"):
        sq.sq_density_vjp(h, torch.zeros(50, dtype=torch.float64), 0.0, 1, torch.zeros(100, dtype=torch.float64))


def test_host_gauss_rule_matches_scipy_eigh_tridiagonal():
    """sq_gauss_rule (the routine the GPU runs per column) against scipy's tridiagonal eigensolver:
    nodes = eigenvalues of the Jacobi matrix, weights = squared first eigenvector components."""
    from scipy.linalg import eigh_tridiagonal
    rng = np.random.default_rng(3)
    for K in (1, 2, 5, 40, 80, 256):
        a = rng.uniform(-0.9, 0.9, K)
        b = rng.uniform(0.05, 0.5, K)
        nodes, w = sq.sq_gauss_rule(a, b, omega=0.5, tau=2.0)
        lam, vec = eigh_tridiagonal(a, b[:K - 1]) if K > 1 else (a.copy(), np.ones((1, 1)))
        order = np.argsort(nodes)
        np.testing.assert_allclose(nodes[order], 2.0 * lam + 0.5, rtol=0, atol=1e-13 * K)
        np.testing.assert_allclose(w[order], vec[0] ** 2, rtol=0, atol=1e-13 * K)
        assert abs(w.sum() - 1.0) < 1e-13


def test_host_gauss_rule_matches_oracle_lanczos_rule(tiny_ref):
    """The same rule on Lanczos coefficients of real columns (tiny cell): equal to the oracle's."""
    c, ref = tiny_ref
    cols = np.array([0, 100, 2000])
    a, b = oracle.lanczos(c, ref["omega"], ref["tau"], cols=cols)
    on, ow = oracle.gauss_rule(a, b, ref["omega"], ref["tau"])
    for i in range(cols.size):
        nodes, w = sq.sq_gauss_rule(a[i], b[i], ref["omega"], ref["tau"])
        o1, o2 = np.argsort(nodes), np.argsort(on[i])
        np.testing.assert_allclose(nodes[o1], on[i][o2], rtol=0, atol=1e-12)
        np.testing.assert_allclose(w[o1], ow[i][o2], rtol=0, atol=1e-12)


def test_host_gauss_rule_cuts_at_an_exhausted_krylov_space():
    a = np.array([0.1, -0.2, 0.3, 0.0])
    b = np.array([0.5, 0.0, 0.7, 0.0])
    nodes, w = sq.sq_gauss_rule(a, b)
    assert abs(w.sum() - 1.0) < 1e-14 and w[2] == 0.0 and w[3] == 0.0
    lam = np.linalg.eigvalsh(np.array([[0.1, 0.5], [0.5, -0.2]]))
    np.testing.assert_allclose(np.sort(nodes[:2]), lam, rtol=0, atol=1e-14)


def test_scf_entry_points_reject_bad_arguments_before_any_launch():
    """sq_lda_pw92, sq_pseudocharge, sq_poisson_periodic and sq_effective_potential check their
    arguments on the host (no device work, so this runs without a GPU)."""
    import ctypes
    L = sq.lib()
    n = (ctypes.c_int * 3)(8, 8, 8)
    box = (ctypes.c_double * 3)(4.0, 4.0, 4.0)
    null = ctypes.c_void_p(0)
    it, res = ctypes.c_int(), ctypes.c_double()
    assert L.sq_lda_pw92(ctypes.c_longlong(0), null, null, null, null) == 1
    bad_n = (ctypes.c_int * 3)(8, 0, 8)
    assert L.sq_pseudocharge(bad_n, box, 0, null, null, ctypes.c_double(1.0), null, null) == 1
    assert L.sq_pseudocharge(n, box, 0, null, null, ctypes.c_double(-1.0), ctypes.c_void_p(8), null) == 1
    for order, tol, iters in ((3, 1e-10, 10), (18, 1e-10, 10), (12, 0.0, 10), (12, 1e-10, 0)):
        assert L.sq_poisson_periodic(n, box, order, ctypes.c_void_p(8), ctypes.c_double(tol), iters,
                                     ctypes.c_void_p(8), ctypes.byref(it), ctypes.byref(res), null) == 1
    assert L.sq_effective_potential(n, box, 12, null, null, ctypes.c_double(1e-10), 10, null, null, null, null,
                                    ctypes.byref(it), ctypes.byref(res), null) == 1


def test_mixer_and_energy_entry_points_reject_bad_arguments_on_the_host():
    """sq_mixer_create, sq_self_energy, sq_free_energy and sq_local_force validate their arguments
    before any device work (this runs without a GPU)."""
    import ctypes
    L = sq.lib()
    out = ctypes.c_void_p()
    for n, hist, beta in ((0, 5, 0.3), (10, -1, 0.3), (10, 33, 0.3), (10, 5, 0.0), (10, 5, 1.5)):
        assert L.sq_mixer_create(ctypes.c_longlong(n), hist, ctypes.c_double(beta), ctypes.byref(out)) == 1
    n3 = (ctypes.c_int * 3)(8, 8, 8)
    box = (ctypes.c_double * 3)(4.0, 4.0, 4.0)
    null = ctypes.c_void_p(0)
    e = ctypes.c_double()
    assert L.sq_self_energy(n3, box, 2, null, null, ctypes.c_double(1.0), ctypes.byref(e), null) == 1
    assert L.sq_self_energy(n3, box, 0, null, null, ctypes.c_double(0.0), ctypes.byref(e), null) == 1
    # no atoms: zero self energy without device work
    assert L.sq_self_energy(n3, box, 0, null, null, ctypes.c_double(1.0), ctypes.byref(e), null) == 0 and e.value == 0.0
    assert L.sq_free_energy(n3, box, null, null, null, null, null, ctypes.c_double(0.0), ctypes.c_double(0.0),
                            ctypes.byref(e), null) == 1
    f = (ctypes.c_double * 3)()
    assert L.sq_local_force(n3, box, 5, 1, null, null, ctypes.c_double(1.0), ctypes.c_void_p(8), f, null) == 1
