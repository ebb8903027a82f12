"""Pins of the oracle's multiple-origin correlator (no GPU).

The statistics are checked against values that follow from their definitions
by hand (Sec. III.E-F), and the whole correlator against closed forms on
stand-in chains whose motion is known exactly: a rigid translation of every
atom (F_s and F_s^cm are then cosines of the known displacement, C_2 = 1) and
a rotation of every molecule in its plane (C_2 = P_2(cos of the angle)).  The
origin schedule is checked against closed-form sample counts.
"""
import numpy as np
import pytest

from oracle import correlation as OC

TWO32 = 4294967296.0


class TranslatingChain:
    """Every atom moves by the fixed-point vector D each sweep."""

    def __init__(self, M, L, D, seed=0):
        rng = np.random.default_rng(seed)
        self.L = L
        self.X = rng.integers(0, 2**32, size=(3 * M, 3), dtype=np.int64)
        self.q = (self.X & 0xFFFFFFFF).astype(np.uint32)
        self.t = np.tile(np.array([0, 1, 2], dtype=np.int32), M)
        self.D = np.asarray(D, dtype=np.int64)

    def run(self, n, T, mix, seed):
        self.X = self.X + n * self.D[None, :]
        self.q = (self.X & 0xFFFFFFFF).astype(np.uint32)


class RotatingChain:
    """Planar triangles (xy-plane) that each turn by theta per sweep about
    their centroid; the atom of slot 1 has type B."""

    def __init__(self, M, L, theta, seed=0):
        rng = np.random.default_rng(seed)
        self.L, self.theta, self.k = L, theta, 0
        self.c = rng.uniform(1.0, L - 1.0, size=(M, 3))
        self.phi = rng.uniform(0.0, 2 * np.pi, size=M)
        self.t = np.tile(np.array([0, 1, 2], dtype=np.int32), M)
        self._place()

    def _place(self):
        ang = self.phi[:, None] + self.k * self.theta + 2 * np.pi * np.arange(3)[None, :] / 3
        pos = np.stack([self.c[:, None, 0] + 0.5 * np.cos(ang), self.c[:, None, 1] + 0.5 * np.sin(ang),
                        np.broadcast_to(self.c[:, None, 2], ang.shape)], axis=-1).reshape(-1, 3)
        self.X = np.round(pos / self.L * TWO32).astype(np.int64)
        self.q = (self.X & 0xFFFFFFFF).astype(np.uint32)

    def run(self, n, T, mix, seed):
        self.k += n
        self._place()


def _qvecs(qmag, n=6, seed=3):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return qmag * v / np.linalg.norm(v, axis=1, keepdims=True)


def test_statistics_by_hand():
    # F_s constant within each sample: 0.2, 0.4, 0.9 -> mean 0.5, variance 0.26/3
    N, M = 6, 2
    ss = []
    for a in (0.2, 0.4, 0.9):
        fcm = np.array([a, -a])
        ss.append((np.full(N, a), fcm, 3.0 * fcm - 1.0))
    r = OC.stats_of_samples(ss)
    assert r[0] == 3
    assert r[1] == pytest.approx(0.5, abs=1e-15)
    assert r[4] == pytest.approx(N * 0.26 / 3, rel=1e-13)      # chi_4 of F_s
    assert r[7] == pytest.approx(0.26 / 3, rel=1e-13)          # chi_4^self of F_s
    # F_s^cm: means 0 in every sample -> chi_4 0; pooled values +-a -> <x^2> = (0.04+0.16+0.81)/3
    assert r[2] == pytest.approx(0.0, abs=1e-15)
    assert r[5] == pytest.approx(0.0, abs=1e-15)
    assert r[8] == pytest.approx(1.01 / 3, rel=1e-13)
    # c2 = 3 fcm - 1 exactly linear: rho = 1
    assert r[10] == pytest.approx(1.0, abs=1e-12)


def test_pearson_signs_and_independence():
    rng = np.random.default_rng(5)
    fcm = [rng.normal(size=400) for _ in range(5)]
    neg = [(np.zeros(3 * 400), f, -0.5 * f + 2.0) for f in fcm]
    assert OC.stats_of_samples(neg)[10] == pytest.approx(-1.0, abs=1e-12)
    ind = [(np.zeros(3 * 400), f, rng.normal(size=400)) for f in fcm]
    assert abs(OC.stats_of_samples(ind)[10]) < 4.0 / np.sqrt(2000)


def test_sums_layout_reproduces_the_statistics():
    rng = np.random.default_rng(7)
    ss = [(rng.uniform(-1, 1, 30), rng.uniform(-1, 1, 10), rng.uniform(-0.5, 1, 10)) for _ in range(4)]
    S = OC.sums_of_samples(ss)
    r = OC.stats_of_samples(ss)
    n, N, M = S[0], 30, 10
    assert n == 4
    assert S[1] / n == pytest.approx(r[1], rel=1e-13)
    assert N * (S[2] / n - (S[1] / n) ** 2) == pytest.approx(r[4], rel=1e-10)
    assert S[8] / (n * M) - (S[7] / (n * M)) ** 2 == pytest.approx(r[8], rel=1e-10)
    cov = S[13] / (n * M) - (S[11] / (n * M)) * (S[7] / (n * M))
    var_c = S[12] / (n * M) - (S[11] / (n * M)) ** 2
    var_f = S[8] / (n * M) - (S[7] / (n * M)) ** 2
    assert cov / np.sqrt(var_c * var_f) == pytest.approx(r[10], rel=1e-10)


def test_translation_closed_form():
    L, M = 9.0, 20
    D = np.array([3_000_000, -1_000_000, 7_000_000], dtype=np.int64)
    qa, qc = _qvecs(7.4), _qvecs(5.1, seed=4)
    lags = [0, 1, 3, 7]
    c = OC.Correlator(TranslatingChain(M, L, D), lags, 2, 10, qa, qc)
    c.run(20, 1.0, None, 0)
    r = c.results()
    h = L / TWO32
    for li, lag in enumerate(lags):
        d = D * lag * h
        assert r[li, 1] == pytest.approx(np.cos(qa @ d).mean(), abs=1e-13)
        assert r[li, 2] == pytest.approx(np.cos(qc @ d).mean(), abs=1e-13)
        assert r[li, 3] == pytest.approx(1.0, abs=1e-13)
        # every particle and every sample the same: no fluctuation
        assert abs(r[li, 4]) < 1e-10 and abs(r[li, 7]) < 1e-12


def test_rotation_closed_form():
    L, M, theta = 8.0, 30, 0.3
    lags = [0, 1, 2, 5]
    c = OC.Correlator(RotatingChain(M, L, theta), lags, 1, 8, _qvecs(7.4), _qvecs(5.1, seed=4))
    c.run(12, 1.0, None, 0)
    r = c.results()
    for li, lag in enumerate(lags):
        x = np.cos(lag * theta)
        assert r[li, 3] == pytest.approx(1.5 * x * x - 0.5, abs=1e-7)    # C_2 = P_2(cos(lag theta))
        assert r[li, 2] == pytest.approx(1.0, abs=1e-7)                  # centroids do not move
        assert abs(r[li, 9]) < 1e-12                                     # same C_2 for every molecule


def _counts(lags, every, max_o, n):
    c = OC.Correlator(TranslatingChain(4, 7.0, [1, 2, 3]), lags, every, max_o, _qvecs(7.4, 2), _qvecs(5.1, 2))
    c.run(n, 1.0, None, 0)
    return c.counts().tolist()


def _want(starts, lags, n):
    return [sum(1 for t0 in starts if t0 + lag <= n) for lag in lags]


@pytest.mark.parametrize("lags,every,n", [([0, 1, 4, 10], 3, 40), ([2, 5], 1, 17), ([0, 6], 4, 50)])
def test_sample_counts_without_slot_limit(lags, every, n):
    # every multiple of `every` becomes an origin
    assert _counts(lags, every, 100, n) == [len(range(0, n - lag + 1, every)) for lag in lags]


@pytest.mark.parametrize("lags,every,n", [([0, 3, 8], 2, 30), ([1, 7], 3, 40), ([0, 5], 5, 26)])
def test_sample_counts_one_slot(lags, every, n):
    # one live origin: the next one starts at the first multiple of `every` at
    # or after the previous one's last lag
    P = -(-lags[-1] // every) * every
    assert _counts(lags, every, 1, n) == _want(range(0, n + 1, P), lags, n)


def test_sample_counts_two_slots():
    # lags up to 9, origins every 2, two slots: origins at 0 and 2, the slot of
    # 0 frees at 9 and the next origin starts at 10, then 12, ... (period 10)
    starts = [t for k in range(6) for t in (10 * k, 10 * k + 2)]
    assert _counts([1, 4, 9], 2, 2, 50) == _want([t for t in starts if t <= 50], [1, 4, 9], 50)


def test_relaxation_time_interpolation():
    lags = [0, 1, 10, 100, 1000]
    # a series linear in ln t crosses exactly where the line does
    f = [1.0, 0.9, 0.9 - 0.3 * np.log(10), 0.9 - 0.3 * np.log(100), 0.9 - 0.3 * np.log(1000)]
    level = 0.5
    want = np.exp((0.9 - level) / 0.3)
    assert OC.relaxation_time(lags, f, [1] * 5, level) == pytest.approx(want, rel=1e-12)
    # crossing between lag 0 and lag 1: linear in t
    assert OC.relaxation_time([0, 1], [1.0, 0.0], [1, 1], 0.25) == pytest.approx(0.75, rel=1e-12)
    # a crossing exactly at a lag point, lags without samples skipped, never crossing
    assert OC.relaxation_time(lags, [1, 0.8, np.exp(-1), 0.1, 0.0], [1] * 5, np.exp(-1)) == pytest.approx(10.0, rel=1e-12)
    # lag 1 has no sample: the crossing lies between lag 0 and lag 10, linear in t
    assert OC.relaxation_time(lags, [1, 0.2, 0.1, 0.05, 0.0], [1, 0, 1, 1, 1], 0.3) == pytest.approx(
        10 * 0.7 / 0.9, rel=1e-12)
    assert np.isnan(OC.relaxation_time(lags, [1, 0.9, 0.8, 0.7, 0.6], [1] * 5, 0.5))
