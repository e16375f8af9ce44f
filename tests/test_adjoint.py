"""Derivatives of the SQ path with respect to V_eff.

CPU: the oracle's forward-mode tangent (differentiated Chebyshev recursion plus the implicit Fermi
level term) against central finite differences of the oracle itself.
GPU: the reverse-mode product (sq_density_vjp, reverse Clenshaw with checkpoints) against that
tangent through the dot-product identity <rho_bar, d rho> + U_bar dU = <V_bar, dV>, against
pointwise tangents, across checkpoint intervals, through the torch.autograd.Function, at the full
size of the 95-atom vacancy cell (K = 60), and in FP32 on a 21^3-cube cell (the slab mapping)
against the FP64 reverse mode."""
import json
import os

import numpy as np
import pytest

from oracle import oracle
from paper_2011_13517_gb300 import cells

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def smooth_field(cell, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.arange(cell.n[a]) / cell.n[a] for a in (2, 1, 0)], indexing="ij")
    f = np.zeros(cell.n[::-1])
    for _ in range(6):
        k = rng.integers(-2, 3, size=3)
        f += rng.standard_normal() * np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + rng.uniform(0, 6.28))
    return f.reshape(-1)


def test_oracle_tangent_matches_finite_differences():
    """d rho, dU, d lambda_f of the oracle's tangent = central differences of the oracle's solve
    (same fixed spectral bounds), step 1e-4 Ha along a smooth field."""
    c = cells.tiny_cell()
    bounds = oracle.spectral_bounds(c)
    dV = smooth_field(c, 1)
    drho, dU, dlam, _ = oracle.sq_tangent(c, dV, bounds=bounds)
    eps = 1e-4
    cp, cm = cells.tiny_cell(), cells.tiny_cell()
    cp.veff = c.veff + eps * dV.reshape(c.veff.shape)
    cm.veff = c.veff - eps * dV.reshape(c.veff.shape)
    rp = oracle.sq_solve(cp, force=False, bounds=bounds)
    rm = oracle.sq_solve(cm, force=False, bounds=bounds)
    fd_rho = (rp["rho"] - rm["rho"]) / (2 * eps)
    np.testing.assert_allclose(drho, fd_rho, rtol=0, atol=1e-6 * np.max(np.abs(fd_rho)))
    assert abs(dU - (rp["U"] - rm["U"]) / (2 * eps)) < 1e-6 * max(1.0, abs(dU))
    assert abs(dlam - (rp["lam_f"] - rm["lam_f"]) / (2 * eps)) < 1e-6 * max(1.0, abs(dlam))


# ---------------------------------------------------------------------------------------------
gpu = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_vjp(cell, bounds, rho_bar, U_bar, kc, precision=None):
    torch = _torch()
    from paper_2011_13517_gb300 import sq
    precision = sq.SQ_FP64 if precision is None else precision
    h = sq.build_for_cell(cell, bounds=bounds)
    rho = torch.empty(cell.N_d, dtype=torch.float64, device="cuda")
    sq.sq_density(h, cell.K, cell.kT, cell.N_e, precision, 0, rho)
    rb = torch.from_numpy(np.ascontiguousarray(rho_bar, dtype=np.float64)).cuda()
    vbar = torch.empty(cell.N_d, dtype=torch.float64, device="cuda")
    sq.sq_density_vjp(h, rb, U_bar, kc, vbar)
    out = vbar.cpu().numpy()
    h.close()
    return out


@gpu
def test_vjp_dot_product_against_oracle_tangent():
    c = cells.tiny_cell()
    bounds = oracle.spectral_bounds(c)
    rng = np.random.default_rng(2)
    rho_bar = rng.standard_normal(c.N_d)
    U_bar = 0.7
    vbar = gpu_vjp(c, bounds, rho_bar, U_bar, 8)
    for seed in (3, 4):
        dV = smooth_field(c, seed)
        drho, dU, _, _ = oracle.sq_tangent(c, dV, bounds=bounds)
        lhs = float(np.dot(rho_bar, drho) + U_bar * dU)
        rhs = float(np.dot(vbar, dV))
        assert abs(lhs - rhs) < 1e-9 * max(abs(lhs), 1e-12), (lhs, rhs)


@gpu
def test_vjp_pointwise_and_checkpoint_independence():
    """V_bar at seeded points against the oracle tangent along e_p; the same V_bar for checkpoint
    intervals 1, 8 and 16 (K = 20: 20, 3 and 2 segments)."""
    c = cells.tiny_cell()
    bounds = oracle.spectral_bounds(c)
    rng = np.random.default_rng(5)
    rho_bar = rng.standard_normal(c.N_d)
    U_bar = -0.3
    v = {kc: gpu_vjp(c, bounds, rho_bar, U_bar, kc) for kc in (1, 8, 16)}
    scale = np.max(np.abs(v[1]))
    for kc in (8, 16):
        np.testing.assert_allclose(v[kc], v[1], rtol=0, atol=1e-12 * scale)
    for p in rng.choice(c.N_d, 4, replace=False):
        e = np.zeros(c.N_d)
        e[p] = 1.0
        drho, dU, _, _ = oracle.sq_tangent(c, e, bounds=bounds)
        ref = float(np.dot(rho_bar, drho) + U_bar * dU)
        assert abs(v[8][p] - ref) < 1e-9 * scale, (p, v[8][p], ref)


@gpu
def test_autograd_function_matches_vjp():
    torch = _torch()
    from paper_2011_13517_gb300.autograd import sq_density_autograd
    c = cells.tiny_cell()
    bounds = oracle.spectral_bounds(c)
    veff = torch.from_numpy(c.veff.reshape(-1).copy()).cuda().requires_grad_(True)
    rho, U = sq_density_autograd(veff, c, bounds, checkpoint_k=4)
    rng = np.random.default_rng(7)
    w = torch.from_numpy(rng.standard_normal(c.N_d)).cuda()
    loss = (w * rho).sum() + 0.5 * U
    (g,) = torch.autograd.grad(loss, veff)
    ref = gpu_vjp(c, bounds, w.cpu().numpy(), 0.5, 4)
    np.testing.assert_allclose(g.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    # directional check against the oracle tangent
    dV = smooth_field(c, 8)
    drho, dU, _, _ = oracle.sq_tangent(c, dV, bounds=bounds)
    lhs = float(np.dot(w.cpu().numpy(), drho) + 0.5 * dU)
    assert abs(lhs - float(np.dot(g.cpu().numpy(), dV))) < 1e-9 * abs(lhs)


@pytest.fixture(scope="module")
def vacancy_vjp():
    """Reverse-mode products of the 95-atom vacancy cell (K = 60, the differentiation workload) for the
    seeded cotangent rho_bar ~ N(0, 1), U_bar = 0.25: FP32 with checkpoint intervals 1, 8, 16 and FP64
    with interval 8, all with the oracle's spectral bounds held fixed."""
    from paper_2011_13517_gb300 import sq
    _torch()
    c = cells.vacancy_cell()
    bounds = oracle.spectral_bounds(c)
    rho_bar = np.random.default_rng(9).standard_normal(c.N_d)
    U_bar = 0.25
    v32 = {kc: gpu_vjp(c, bounds, rho_bar, U_bar, kc, precision=sq.SQ_FP32) for kc in (1, 8, 16)}
    v64 = gpu_vjp(c, bounds, rho_bar, U_bar, 8, precision=sq.SQ_FP64)
    return dict(cell=c, bounds=bounds, rho_bar=rho_bar, U_bar=U_bar, v32=v32, v64=v64)


@gpu
def test_vjp_vacancy_checkpoint_intervals_agree(vacancy_vjp):
    v32 = vacancy_vjp["v32"]
    scale = np.max(np.abs(v32[8]))
    for kc in (1, 16):
        np.testing.assert_allclose(v32[kc], v32[8], rtol=0, atol=1e-6 * scale)


@gpu
def test_vjp_vacancy_directional_finite_difference(vacancy_vjp):
    """The FP64 reverse-mode directional derivative along a smooth field against central differences
    of the FP64 forward path (step 1e-4 Ha); FP32 within 1e-3."""
    from paper_2011_13517_gb300 import sq
    c, bounds = vacancy_vjp["cell"], vacancy_vjp["bounds"]
    rho_bar, U_bar = vacancy_vjp["rho_bar"], vacancy_vjp["U_bar"]
    dV = smooth_field(c, 10)
    eps = 1e-4
    vals = []
    for sgn in (1, -1):
        cc = cells.vacancy_cell()
        cc.veff = c.veff + sgn * eps * dV.reshape(c.veff.shape)
        r = sq.solve_cell(cc, sq.SQ_FP64, force=False, bounds=bounds)
        vals.append(float(np.dot(rho_bar, r["rho"]) + U_bar * r["U"]))
    fd = (vals[0] - vals[1]) / (2 * eps)
    ad64 = float(np.dot(vacancy_vjp["v64"], dV))
    ad32 = float(np.dot(vacancy_vjp["v32"][8], dV))
    print("vacancy VJP directional derivative: FD", fd, "FP64", ad64, "FP32", ad32)
    assert abs(ad64 - fd) < 1e-6 * abs(fd)
    assert abs(ad32 - fd) < 1e-3 * abs(fd)


@gpu
def test_vjp_vacancy_matches_oracle_tangent(vacancy_vjp):
    """Dot-product identity at full size against the oracle's forward-mode tangent (golden value from
    tests/golden/make_golden.py vacancy_tangent): <V_bar, dV> = <rho_bar, d rho> + U_bar dU, FP64 with
    checkpoint interval 8 within 1e-9, FP32 with intervals 1, 8 and 16 within 1e-4 (relative)."""
    path = os.path.join(GOLDEN, "vacancy_95atom_tangent.json")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    g = json.load(open(path))
    c = vacancy_vjp["cell"]
    assert g["digest"] == c.digest() and abs(g["U_bar"] - vacancy_vjp["U_bar"]) == 0.0
    assert abs(g["lmin"] - vacancy_vjp["bounds"][0]) < 1e-12 and abs(g["lmax"] - vacancy_vjp["bounds"][1]) < 1e-12
    dV = smooth_field(c, 10)
    d64 = float(np.dot(vacancy_vjp["v64"], dV))
    print("tangent golden", g["dot"], "FP64 reverse", d64, {kc: float(np.dot(v, dV)) for kc, v in vacancy_vjp["v32"].items()})
    assert abs(d64 - g["dot"]) < 1e-9 * abs(g["dot"])
    for kc in (1, 8, 16):
        assert abs(float(np.dot(vacancy_vjp["v32"][kc], dV)) - g["dot"]) < 1e-4 * abs(g["dot"])


@gpu
def test_vjp_vacancy_pointwise_finite_differences(vacancy_vjp):
    """Central differences (step 1e-4 Ha) at 64 seeded grid points of the vacancy cell against the FP64
    reverse-mode product there.  A change of V_eff at point p moves only the columns whose cube holds
    p (the cube of columns around p), so each difference recomputes those 15,625 columns in FP64
    (sq_moments_cols) and redoes the Fermi solve (Eq. Ne) and weights on the host (sq_fermi_level,
    sq_fermi_weights) with the other columns' moments unchanged -- exact, not an approximation."""
    torch = _torch()
    from paper_2011_13517_gb300 import sq
    c, bounds = vacancy_vjp["cell"], vacancy_vjp["bounds"]
    rho_bar, U_bar, v64 = vacancy_vjp["rho_bar"], vacancy_vjp["U_bar"], vacancy_vjp["v64"]
    lo, hi = bounds
    omega, tau = 0.5 * (hi + lo), 0.5 * (hi - lo)
    K, dV = c.K, float(np.prod(c.h))
    base = sq.solve_cell(c, sq.SQ_FP64, force=False, bounds=bounds)
    mu0 = base["mu"]                              # [K+1, N_d]
    M0 = mu0.sum(axis=1)
    R0 = mu0 @ rho_bar
    n = [int(x) for x in c.n]
    m = [int(x) for x in c.m]
    pts = np.random.default_rng(64).choice(c.N_d, size=64, replace=False)
    eps = 1e-4
    veff = torch.from_numpy(np.ascontiguousarray(c.veff.reshape(-1))).cuda()
    out = torch.empty((K + 1) * int(np.prod(c.n_c)), dtype=torch.float64, device="cuda")
    worst = 0.0
    scale = float(np.max(np.abs(v64)))
    for p in pts:
        px, py, pz = p % n[0], (p // n[0]) % n[1], p // (n[0] * n[1])
        gx = (px + np.arange(-m[0], m[0] + 1)) % n[0]
        gy = (py + np.arange(-m[1], m[1] + 1)) % n[1]
        gz = (pz + np.arange(-m[2], m[2] + 1)) % n[2]
        cols = (gx[None, None, :] + n[0] * (gy[None, :, None] + n[1] * gz[:, None, None])).reshape(-1)
        dcols = torch.from_numpy(cols.astype(np.int64)).cuda()
        parts = []
        for sgn in (1.0, -1.0):
            v = veff.clone()
            v[int(p)] += sgn * eps
            h = sq.build_for_cell(c, bounds=bounds, d_veff=v)
            sq.sq_moments_cols(h, K, sq.SQ_FP64, dcols, out)
            h.close()
            mu = out.view(K + 1, cols.size).cpu().numpy()
            dmu = mu - mu0[:, cols]
            dM = dmu.sum(axis=1)
            dR = dmu @ rho_bar[cols]
            lam = sq.sq_fermi_level(M0 + dM, K, omega, tau, lo, hi, c.kT, c.N_e)
            cw, dw, _ = sq.sq_fermi_weights(lam, K, omega, tau, c.kT)
            parts.append((cw, dw, dM, dR))
        # L = 2/dV c.(R0 + dR) + 2 U_bar d.(M0 + dM); the difference of the two sides is formed term by
        # term, so the large common parts c.R0 and d.M0 (about 1e3) do not cancel in FP64 rounding
        (cp, dp, dMp, dRp), (cm, dm, dMm, dRm) = parts
        dL = (2.0 / dV * (float((cp - cm) @ R0) + float(cp @ dRp) - float(cm @ dRm))
              + U_bar * 2.0 * (float((dp - dm) @ M0) + float(dp @ dMp) - float(dm @ dMm)))
        fd = dL / (2 * eps)
        err = abs(fd - v64[p])
        worst = max(worst, err / scale)
        assert err < 1e-7 * scale + 1e-6 * abs(v64[p]), (int(p), fd, v64[p])
    print("pointwise FD vs FP64 reverse mode at 64 points: max error / max |V_bar| =", worst)


@gpu
def test_fp32_slab_vjp_matches_fp64_on_21_cube():
    """FP32 reverse mode on a 47-atom cell with 21^3 cubes (the slab mapping of the recursion) against
    the FP64 reverse mode, which the dot-product tests hold to the oracle tangent: pointwise within
    2e-4 of the largest component, for checkpoint intervals 1, 5 and 12 (single-step segments,
    segments with recomputation, one segment), which agree with each other to 1e-6."""
    _torch()
    from paper_2011_13517_gb300 import sq
    c = cells.make_cell("rc5", (3, 2, 2), 0.5, 12, 1, 5.0, 12, 0.005, seed=9, n_vacancy=1)
    assert np.all(c.n_c == 21)
    bounds = oracle.spectral_bounds(c)
    rng = np.random.default_rng(21)
    rho_bar = rng.standard_normal(c.N_d)
    U_bar = 0.3
    v64 = gpu_vjp(c, bounds, rho_bar, U_bar, 4, precision=sq.SQ_FP64)
    scale = np.max(np.abs(v64))
    v32 = {kc: gpu_vjp(c, bounds, rho_bar, U_bar, kc, precision=sq.SQ_FP32) for kc in (1, 5, 12)}
    err = {kc: float(np.max(np.abs(v - v64)) / scale) for kc, v in v32.items()}
    print("FP32 slab VJP max error / max |Vbar|:", err)
    for kc in (1, 5, 12):
        assert err[kc] < 2e-4
    for kc in (1, 12):
        np.testing.assert_allclose(v32[kc], v32[5], rtol=0, atol=1e-6 * scale)
