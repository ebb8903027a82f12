"""The library's host arithmetic of the correlator (no GPU): the statistics
derived from the sums, and the relaxation-time interpolation, against the
oracle's separately written forms (numpy var and corrcoef on the stored
samples; its own interpolation)."""
import numpy as np
import pytest

from oracle import correlation as OC
from paper_2506_21290_gb300 import build as B
from paper_2506_21290_gb300 import flipmc as F


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    F.load()


def _samples(rng, n_samples, M, corr=0.0):
    out = []
    for _ in range(n_samples):
        fcm = rng.uniform(-0.2, 1.0, M)
        c2 = corr * fcm + (1 - abs(corr)) * rng.uniform(-0.5, 1.0, M)
        out.append((rng.uniform(-0.3, 1.0, 3 * M), fcm, c2))
    return out


@pytest.mark.parametrize("n_samples,M,corr", [(1, 10, 0.0), (5, 40, 0.7), (12, 125, -0.4), (3, 1000, 1.0)])
def test_derived_statistics_match_the_oracle(n_samples, M, corr):
    ss = _samples(np.random.default_rng(n_samples * 7 + M), n_samples, M, corr)
    got = F.mc_corr_derive(OC.sums_of_samples(ss), 3 * M)
    want = OC.stats_of_samples(ss)
    assert got[0] == want[0]
    assert np.allclose(got[1:4], want[1:4], rtol=0, atol=1e-13)
    assert np.allclose(got[4:7], want[4:7], rtol=0, atol=1e-10 * 3 * M)
    assert np.allclose(got[7:10], want[7:10], rtol=0, atol=1e-12)
    assert got[10] == pytest.approx(want[10], abs=1e-9)


def test_derived_statistics_edge_cases():
    nan_row = F.mc_corr_derive(np.zeros(16), 3)
    assert nan_row[0] == 0 and np.all(np.isnan(nan_row[1:]))
    # every particle the same in every sample: no fluctuation, and rho undefined
    ss = [(np.full(6, 0.5), np.full(2, 0.25), np.full(2, 0.1)) for _ in range(3)]
    r = F.mc_corr_derive(OC.sums_of_samples(ss), 6)
    assert np.allclose(r[1:4], [0.5, 0.25, 0.1], atol=1e-15)
    assert np.allclose(r[4:10], 0.0, atol=1e-14)
    assert np.isnan(r[10])
    # rows of several replicas at once, each with its own size
    rows = np.stack([OC.sums_of_samples(_samples(np.random.default_rng(k), 2, m)) for k, m in enumerate((5, 9))])
    r2 = F.mc_corr_derive(rows, np.array([15, 27]))
    assert r2.shape == (2, 11)
    with pytest.raises(F.McError):
        F.mc_corr_derive(rows, np.array([15, 26]))


def test_relaxation_time_matches_the_oracle():
    rng = np.random.default_rng(3)
    lags = np.array([0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144])
    for trial in range(200):
        f = np.sort(rng.uniform(-0.1, 1.0, lags.size))[::-1].copy()
        n = (rng.uniform(size=lags.size) > 0.2).astype(np.float64)
        level = rng.uniform(0.0, 1.0)
        want = OC.relaxation_time(lags, f, n, level)
        got = F.mc_relaxation_time(lags, f, n, level)
        assert (np.isnan(want) and np.isnan(got)) or got == pytest.approx(want, rel=1e-12), trial
    # a series linear in ln t is crossed exactly where the line crosses
    t = np.array([1, 10, 100, 1000])
    assert F.mc_relaxation_time(t, 0.9 - 0.3 * np.log(t), np.ones(4), 0.5) == pytest.approx(np.exp(0.4 / 0.3), rel=1e-12)
