"""The self-consistency pieces on the GPU (sq_lda_pw92, sq_pseudocharge, sq_poisson_periodic,
sq_effective_potential; Sec. 2.1 LDA and Eq. Poisson, Sec. 3 "Electrostatic and effective potential")
against the oracle (oracle/electrostatics.py) on the same seeded inputs.  Tolerances: eps_xc, V_xc and
the pseudocharge to FP64 rounding (1e-12 relative); phi and V_eff to 10 cond(-L_h) times the conjugate-
gradient residual (1e-12) of their largest magnitude, against the oracle's exact Fourier solve."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import electrostatics as es  # noqa: E402
from oracle import oracle  # noqa: E402
from paper_2011_13517_gb300 import cells, sq  # noqa: E402

SIGMA_B = 1.0


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_lda_kernel_matches_oracle():
    rng = np.random.default_rng(21)
    rho = np.exp(rng.uniform(math.log(1e-7), math.log(5.0), 100_000))
    rho[:50] = 0.0
    rho[50:60] = -1e-9
    exc = torch.empty(rho.size, dtype=torch.float64, device="cuda")
    vxc = torch.empty_like(exc)
    sq.sq_lda_pw92(dev(rho), exc, vxc)
    e_ref, v_ref = es.lda_pw92(rho)
    np.testing.assert_allclose(exc.cpu().numpy(), e_ref, rtol=1e-12, atol=0)
    np.testing.assert_allclose(vxc.cpu().numpy(), v_ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("make", [cells.tiny_cell, cells.vacancy_cell])
def test_pseudocharge_kernel_matches_oracle(make):
    c = make()
    Z = es.valence_charges(c)
    b = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    sq.sq_pseudocharge(c.n, c.box, c.R, Z, SIGMA_B, b)
    ref = es.pseudocharge(c, SIGMA_B)
    np.testing.assert_allclose(b.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("make", [cells.tiny_cell, cells.vacancy_cell])
def test_poisson_matches_oracle(make):
    c = make()
    rng = np.random.default_rng(5)
    if c.natom > 20:   # a smooth density-like field plus the pseudocharges
        f = np.exp(-c.veff.reshape(-1)) + es.pseudocharge(c, SIGMA_B)
    else:
        f = rng.standard_normal(c.N_d)
    phi = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    it, res = sq.sq_poisson_periodic(c.n, c.box, c.fd_order, dev(f), phi, tol=1e-12, max_iter=20000)
    ref = es.poisson_periodic(f, c)
    err = float(np.max(np.abs(phi.cpu().numpy() - ref)))
    print(f"{c.name}: Poisson CG {it} iterations, residual {res:.2e}, max |phi - phi_oracle| / max |phi| "
          f"{err / np.abs(ref).max():.2e}")
    assert res <= 1e-12 and it < 20000
    # a residual r bounds the error by |r| / lambda_min, i.e. by cond(-L_h) times the relative residual
    lam = np.abs(es.laplacian_symbol(c)).reshape(-1)
    cond = lam.max() / lam[lam > 0].min()
    assert err < 10.0 * cond * 1e-12 * np.abs(ref).max(), (err, cond)


def test_effective_potential_matches_oracle():
    c = cells.tiny_cell()
    lo, hi = oracle.spectral_bounds(c)
    gpu = sq.solve_cell(c, sq.SQ_FP64, force=False, bounds=(lo, hi))
    rho = gpu["rho"]
    Z = es.valence_charges(c)
    b = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    sq.sq_pseudocharge(c.n, c.box, c.R, Z, SIGMA_B, b)
    out = [torch.empty(c.N_d, dtype=torch.float64, device="cuda") for _ in range(4)]
    it, res = sq.sq_effective_potential(c.n, c.box, c.fd_order, dev(rho), b, *out, tol=1e-12, max_iter=20000)
    phi, exc, vxc, veff = [t.cpu().numpy() for t in out]
    v_ref, phi_ref, vxc_ref, _ = es.effective_potential(rho, c, SIGMA_B)
    lam = np.abs(es.laplacian_symbol(c)).reshape(-1)
    tol = 10.0 * lam.max() / lam[lam > 0].min() * 1e-12
    np.testing.assert_allclose(phi, phi_ref, rtol=0, atol=tol * np.abs(phi_ref).max())
    np.testing.assert_allclose(vxc, vxc_ref, rtol=1e-12, atol=0)
    np.testing.assert_allclose(veff, v_ref, rtol=0, atol=tol * np.abs(phi_ref).max() + 1e-12 * np.abs(vxc_ref).max())
    # the electron density and the pseudocharges nearly cancel: the removed mean is the grid's
    # normalisation error of the Gaussians, tiny against the electron count
    dV = float(np.prod(c.h))
    assert abs((rho.sum() + b.cpu().numpy().sum()) * dV) < 1e-3 * c.N_e


def test_poisson_reports_non_convergence():
    c = cells.tiny_cell()
    f = np.random.default_rng(1).standard_normal(c.N_d)
    phi = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SQError) as ei:
        sq.sq_poisson_periodic(c.n, c.box, c.fd_order, dev(f), phi, tol=1e-14, max_iter=2)
    assert ei.value.status == 6


def test_scf_tiny_cell_matches_oracle():
    """The SCF loop on the GPU (sq_build_hamiltonian of V_in with the library's spectral bounds,
    sq_density FP64, sq_effective_potential, sq_mixer_step) against the oracle's SCF with the same
    Anderson mixing (beta 0.3, history 5) to |V_out - V_in| / |V_out| <= 1e-10: the same number of
    iterations, and V_eff, rho and lambda_f at the fixed point within 1e-8 (relative to their largest
    values; both iterate the same map, so they differ by rounding amplified over the iterations)."""
    c = cells.tiny_cell()
    ref = es.scf(c, SIGMA_B, beta=0.3, m=5, tol=1e-10, max_iter=80)
    Z = es.valence_charges(c)
    N = c.N_d
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    sq.sq_pseudocharge(c.n, c.box, c.R, Z, SIGMA_B, b)
    v_in = dev(c.veff.reshape(-1))
    rho = torch.empty(N, dtype=torch.float64, device="cuda")
    phi, exc, vxc, v_out = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4)]
    mixer = sq.sq_mixer_create(N, history=5, beta=0.3)
    errs, lam = [], None
    try:
        for it in range(1, 81):
            h = sq.build_for_cell(c, d_veff=v_in)
            lam = sq.sq_density(h, c.K, c.kT, c.N_e, sq.SQ_FP64, 0, rho)
            h.close()
            sq.sq_effective_potential(c.n, c.box, c.fd_order, rho, b, phi, exc, vxc, v_out, tol=1e-13)
            rho_it = rho.cpu().numpy()
            v_it = v_in.cpu().numpy()
            err = sq.sq_mixer_step(mixer, v_in, v_out, v_in)
            errs.append(err)
            if err <= 1e-10:
                break
    finally:
        mixer.close()
    print("GPU SCF errors", ["%.1e" % e for e in errs])
    print("oracle SCF errors", ["%.1e" % e for e in ref["errors"]])
    assert errs[-1] <= 1e-10 and abs(len(errs) - ref["iters"]) <= 1
    np.testing.assert_allclose(v_it, ref["veff"], rtol=0, atol=1e-8 * np.abs(ref["veff"]).max())
    np.testing.assert_allclose(rho_it, ref["rho"], rtol=0, atol=1e-8 * np.abs(ref["rho"]).max())
    assert abs(lam - ref["lam_f"]) < 1e-8


@pytest.mark.parametrize("make", [cells.tiny_cell, cells.vacancy_cell])
def test_free_energy_and_local_force_match_oracle(make):
    """E_self^h, the density terms of F^h (Eq. DiscreteEnergy) and the local force (Eq.
    DiscreteLocalForce; the GPU sums b_J against nabla_h phi, the oracle nabla_h b_J against phi) on a
    fixed smooth density of the cell's electron count: E_self to 1e-12 relative, F^h to the Poisson
    tolerance, forces to the same bound relative to the largest component."""
    c = make()
    rho = np.exp(-c.veff.reshape(-1))
    rho *= c.N_e / (rho.sum() * float(np.prod(c.h)))
    Z = es.valence_charges(c)
    b = torch.empty(c.N_d, dtype=torch.float64, device="cuda")
    sq.sq_pseudocharge(c.n, c.box, c.R, Z, SIGMA_B, b)
    phi, exc, vxc, veff = [torch.empty(c.N_d, dtype=torch.float64, device="cuda") for _ in range(4)]
    d_rho = dev(rho)
    sq.sq_effective_potential(c.n, c.box, c.fd_order, d_rho, b, phi, exc, vxc, veff, tol=1e-13)
    e_self = sq.sq_self_energy(c.n, c.box, c.R, Z, SIGMA_B)
    e_ref = es.self_energy_discrete(c, SIGMA_B)
    assert abs(e_self - e_ref) < 1e-12 * abs(e_ref)
    F = sq.sq_free_energy(c.n, c.box, d_rho, b, phi, exc, vxc, 0.0, e_self)
    F_ref, _ = es.free_energy(c, SIGMA_B, rho, 0.0, 0.0, c.kT)
    lam = np.abs(es.laplacian_symbol(c)).reshape(-1)
    tol = 10.0 * lam.max() / lam[lam > 0].min() * 1e-13
    assert abs(F - F_ref) < 1e-9 * abs(F_ref) + tol * abs(F_ref), (F, F_ref)
    f = sq.sq_local_force(c.n, c.box, c.fd_order, c.R, Z, SIGMA_B, phi)
    f_ref = es.local_force(c, SIGMA_B, es.poisson_periodic(rho + es.pseudocharge(c, SIGMA_B), c))
    np.testing.assert_allclose(f, f_ref, rtol=0, atol=1e-9 * np.abs(f_ref).max() + tol * np.abs(f_ref).max())
