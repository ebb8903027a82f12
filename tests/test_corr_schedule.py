"""The library's correlation-origin schedule (host C++, no GPU) against closed
forms and against the oracle's correlator, which implements the same schedule
separately."""
import numpy as np
import pytest

from oracle import correlation as OC
from paper_2506_21290_gb300 import build as B
from paper_2506_21290_gb300 import flipmc as F


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    F.load()


class _Still:
    """A chain that never moves (the schedule does not look at the state)."""

    def __init__(self, n_mol=2):
        self.L = 5.0
        tri = np.array([[0, 0, 0], [10_000_000, 0, 0], [0, 10_000_000, 0]], dtype=np.int64)
        self.X = (tri[None, :, :] + 50_000_000 * np.arange(n_mol)[:, None, None]).reshape(-1, 3)
        self.q = (self.X & 0xFFFFFFFF).astype(np.uint32)
        self.t = np.tile(np.array([0, 1, 2], dtype=np.int32), n_mol)

    def run(self, n, T, mix, seed):
        pass


@pytest.mark.parametrize("lags,every,n", [([0, 1, 4, 10], 3, 40), ([2, 5], 1, 17), ([0, 6], 4, 50)])
def test_without_slot_limit(lags, every, n):
    assert F.mc_corr_schedule(lags, every, 100, n).tolist() == [len(range(0, n - lag + 1, every)) for lag in lags]


@pytest.mark.parametrize("lags,every,n", [([0, 3, 8], 2, 30), ([1, 7], 3, 40), ([0, 5], 5, 26)])
def test_one_slot(lags, every, n):
    P = -(-lags[-1] // every) * every
    want = [sum(1 for t0 in range(0, n + 1, P) if t0 + lag <= n) for lag in lags]
    assert F.mc_corr_schedule(lags, every, 1, n).tolist() == want


@pytest.mark.parametrize("lags,every,max_o,n", [([1, 4, 9], 2, 2, 50), ([0, 2, 3, 11], 3, 3, 77), ([5], 2, 1, 33),
                                                 ([0], 1, 1, 9), ([0, 1, 2, 3, 5, 8, 13], 2, 5, 40)])
def test_matches_the_oracle_schedule(lags, every, max_o, n):
    qa = np.array([[7.4, 0.0, 0.0]])
    c = OC.Correlator(_Still(), lags, every, max_o, qa, qa)
    c.run(n, 1.0, None, 0)
    assert F.mc_corr_schedule(lags, every, max_o, n).tolist() == c.counts().tolist()


def test_bad_arguments():
    for lags, every, max_o in (([3, 3], 1, 4), ([-1, 2], 1, 4), ([0, 2], 0, 4), ([0, 2], 1, 0), ([0, 2], 1, 2000)):
        with pytest.raises(F.McError) as e:
            F.mc_corr_schedule(lags, every, max_o, 10)
        assert e.value.code == F.MC_ERR_INVALID_ARG
