"""The cell grid the library picks (host C++, no GPU), pinned to the geometry
that follows from the paper's model and density (Sec. II.A: rho = 1.2,
sigma = 0.9, 1, 1.1, FENE range 1.5 sigma_ab).  In an {A, B, C} molecule the
widest bonded pair is B-C, sigma_BC = (1 + 1.1) / 2 = 1.05, so the longest
interaction is its FENE range 1.5 x 1.05 = 1.575 (above every WCA cutoff,
2^(1/6) x 1.1 = 1.235), and n_c is the largest even count of cells at least
that wide."""
import numpy as np
import pytest

from paper_2506_21290_gb300 import build as B
from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    F.load()


@pytest.mark.parametrize("M,nc", [(64, 2), (256, 4), (1000, 8), (2000, 10), (8000, 16), (64000, 34)])
def test_cells_per_axis_at_the_papers_density(M, nc):
    L = W.box_length(M)
    types = np.tile(np.array([0, 1, 2], dtype=np.int32), M)
    got, rng = F.mc_cell_grid(L, types, W.PAPER_POT)
    assert rng == pytest.approx(1.575, rel=1e-12)
    assert got == nc
    # the largest even n_c: cells of n_c + 2 per axis would be narrower than the range
    assert np.floor(2 ** 32 / got) * L / 2 ** 32 >= rng
    assert np.floor(2 ** 32 / (got + 2)) * L / 2 ** 32 < rng


def test_range_without_a_bond_of_the_widest_pair():
    # molecules of types A, A, B only: bonded pairs A-A and A-B, so the FENE range is 1.5 x 0.95
    types = np.tile(np.array([0, 0, 1], dtype=np.int32), 10)
    nc, rng = F.mc_cell_grid(10.0, types, W.PAPER_POT)
    assert rng == pytest.approx(max(1.5 * 0.95, 2 ** (1 / 6) * 1.1), rel=1e-12)


def test_requests_and_errors():
    L = W.box_length(1000)
    types = np.tile(np.array([0, 1, 2], dtype=np.int32), 1000)
    assert F.mc_cell_grid(L, types, W.PAPER_POT, request=6)[0] == 6
    for bad in (7, 10, 1):            # odd, cells too narrow, fewer than 2
        with pytest.raises(F.McError):
            F.mc_cell_grid(L, types, W.PAPER_POT, request=bad)
    with pytest.raises(F.McError):
        F.mc_cell_grid(2.5, np.tile(np.array([0, 1, 2], dtype=np.int32), 2), W.PAPER_POT)   # L < 2 x range
    with pytest.raises(F.McError):
        F.mc_cell_grid(L, np.array([0, 1, 3], dtype=np.int32), W.PAPER_POT)
