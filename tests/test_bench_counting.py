"""Host-side pieces of bench.py that feed the reported roofline: the projector support geometry
behind the algorithmic FLOP count must be exactly the set where the oracle's periodised projector
factors are nonzero (the window (1 - t^2/r_c^2)^3 of Sec. 3's projectors vanishes from |t| = r_c on),
and the count must reduce to the plain stencil count when there are no atoms."""
import numpy as np

import bench
from oracle import oracle
from paper_2011_13517_gb300 import cells


def test_support_mask_matches_oracle_factors():
    for c in (cells.tiny_cell(), cells.vacancy_cell()):
        for J in range(c.natom):
            for a in range(3):
                g = oracle.axis_factors(c.R[J, a], c.box[a], int(c.n[a]), c.proj_sigma, c.proj_rc)[0]
                assert np.array_equal(g != 0, bench.support_mask(c.R[J, a], c.box[a], int(c.n[a]), c.proj_rc))


def test_flop_count_without_atoms_is_the_stencil_count():
    c = cells.tiny_cell()
    c.R = c.R[:0]
    nc3 = int(np.prod(c.n_c))
    assert bench.algorithmic_flops(c) == 2.0 * c.N_d * c.K * nc3 * (3 * c.fd_order + 2)


def test_vacancy_flop_count():
    """24.968 TFLOP per launch on the vacancy cell (the figure the bench's roofline divides)."""
    assert abs(bench.algorithmic_flops(cells.vacancy_cell()) / 1e12 - 24.96816041472) < 1e-9


def test_ball_count_matches_periodic_convolution():
    """The ball-support FLOP count (sum_q |B ^ C_q| = |B| n_c^3, and the force term as the ball's
    autocorrelation over the cube offsets) against a direct periodic convolution on the full grid:
    for every column q, |B ^ C_q| = (1_B * 1_C)(q), summed over all q, and over q inside B."""
    c = cells.vacancy_cell()
    nz, ny, nx = int(c.n[2]), int(c.n[1]), int(c.n[0])
    m = c.m
    cube = np.zeros((nz, ny, nx))
    for dz in range(-m[2], m[2] + 1):
        for dy in range(-m[1], m[1] + 1):
            cube[dz % nz, dy % ny, (np.arange(-m[0], m[0] + 1)) % nx] = 1.0
    Fc = np.fft.fftn(cube)
    for J in (0, 17, 94):
        x = [np.arange(int(c.n[a])) * c.h[a] - c.R[J, a] for a in range(3)]
        d = [xa - c.box[a] * np.round(xa / c.box[a]) for a, xa in enumerate(x)]
        ball = (d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2) < c.proj_rc ** 2
        per_q = np.rint(np.real(np.fft.ifftn(np.fft.fftn(ball.astype(float)) * Fc)))
        b = bench.ball_support(c, J)
        assert int(ball.sum()) == int(b.sum())
        from scipy.signal import fftconvolve
        ac = fftconvolve(b.astype(float), b[::-1, ::-1, ::-1].astype(float))
        cz, cy, cx = np.array(b.shape) - 1
        force = np.rint(ac[cz - m[2]:cz + m[2] + 1, cy - m[1]:cy + m[1] + 1, cx - m[0]:cx + m[0] + 1].sum())
        assert int(per_q.sum()) == int(ball.sum()) * int(np.prod(c.n_c))
        assert int(per_q[ball].sum()) == int(force)


def test_ball_count_without_atoms_is_the_stencil_count():
    c = cells.tiny_cell()
    c.R = c.R[:0]
    nc3 = int(np.prod(c.n_c))
    assert bench.algorithmic_flops_ball(c) == 2.0 * c.N_d * c.K * nc3 * (3 * c.fd_order + 2)
