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
