"""Pins of the oracle's static observables (no GPU).

The pair virial W = sum -r dphi/dr is pinned to the energy, which the oracle
computes by separate code (the C chain): scaling the box by lambda at fixed
fractional coordinates scales every pair distance by lambda, so
W = -dU/dlambda at lambda = 1, taken here by a central difference.
"""
import numpy as np
import pytest

import oracle
from oracle import structure as S
from paper_2506_21290_gb300 import workloads as W

POT = W.PAPER_POT


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _state(M, T, sweeps, seed):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    ch = oracle.Chain(L, xyz, t, POT)
    n = 2
    while np.floor(2 ** 32 / (n + 2)) * L / 2 ** 32 >= 1.575:
        n += 2
    ch.run(sweeps, T, W.PAPER_MIX, seed=seed, nc=n)
    return L, ch


@pytest.mark.parametrize("M,T,sweeps,seed", [(64, 2.0, 20, 1), (125, 1.0, 10, 2)])
def test_virial_is_minus_the_volume_derivative_of_the_energy(M, T, sweeps, seed):
    L, ch = _state(M, T, sweeps, seed)
    d = 1e-6
    up = oracle.energy(L * (1 + d), ch.q, ch.t, POT)
    dn = oracle.energy(L * (1 - d), ch.q, ch.t, POT)
    dU = (up - dn) / (2 * d)
    Wv = S.virial(L, ch.q, ch.t, POT)
    assert Wv == pytest.approx(-dU, rel=2e-6, abs=1e-6 * abs(oracle.energy(L, ch.q, ch.t, POT)))


def test_pressure_ideal_part_and_units():
    # P - N T / V is T-independent (the virial part), and N T / V = rho T
    L, ch = _state(64, 3.0, 5, 3)
    p1 = S.pressure(L, ch.q, ch.t, POT, 1.0)
    p2 = S.pressure(L, ch.q, ch.t, POT, 2.0)
    assert p2 - p1 == pytest.approx(ch.t.size / L ** 3, rel=1e-12)
    assert ch.t.size / L ** 3 == pytest.approx(1.2, rel=1e-4)    # the paper's density


def _cubic_lattice(n, a, L):
    """n^3 atoms on a simple cubic lattice of spacing a in a box of side L = n a."""
    g = np.arange(n) * a
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return oracle.quantize(x, L)


def test_structure_factor_of_a_lattice_is_a_bragg_comb():
    n, a = 6, 1.0
    L = n * a
    q = _cubic_lattice(n, a, L)
    N = n ** 3
    two_pi_L = 2 * np.pi / L
    qv = np.array([[n, 0, 0], [0, n, 0], [n, n, 0], [1, 0, 0], [2, 3, 0], [1, 1, 1], [0, 0, 2 * n]]) * two_pi_L
    Sq = S.structure_factor(L, q, qv)
    # reciprocal-lattice vectors of the lattice (multiples of 2 pi / a): S = N; other box vectors: S = 0
    assert np.allclose(Sq[[0, 1, 2, 6]], N, rtol=1e-9)
    assert np.all(np.abs(Sq[[3, 4, 5]]) < 1e-9)


def test_pair_histogram_of_a_lattice():
    n, a = 8, 1.0
    L = n * a
    q = _cubic_lattice(n, a, L)
    N = n ** 3
    dr = 0.05
    c = S.pair_histogram(L, q, dr, 50)          # up to r = 2.5 < L / 2
    # shells of the simple cubic lattice: a (6 neighbours), a sqrt 2 (12), a sqrt 3 (8), 2a (6), a sqrt 5 (24)
    want = {1.0: 6, np.sqrt(2): 12, np.sqrt(3): 8, 2.0: 6, np.sqrt(5): 24, np.sqrt(6): 24}
    total = 0
    for r, z in want.items():
        b = int(np.floor(r / dr + 1e-6))
        # the lattice points are quantised to 2^-32 L: a shell lands in its bin or a neighbour
        got = c[max(b - 1, 0):b + 2].sum()
        assert got == N * z // 2, (r, got)
        total += N * z // 2
    assert c.sum() == total
    g = S.pair_correlation(L, c, N, dr)
    assert np.all(g >= 0)


def test_ideal_gas_g_and_S_are_one():
    """Uniform random points: g(r) = 1 at every r (the normalisation 2 counts /
    (N rho V_shell)), and S(q) averages to 1 over box wavevectors."""
    rng = np.random.default_rng(11)
    L, N = 12.0, 3000
    q = oracle.quantize(rng.uniform(0, L, size=(N, 3)), L)
    dr, nb = 0.25, 20
    c = S.pair_histogram(L, q, dr, nb)
    g = S.pair_correlation(L, c, N, dr)
    shells = slice(4, nb)                          # r in [1, 5): enough pairs per bin for a 5% check
    assert np.all(np.abs(g[shells] - 1.0) < 0.05)
    assert abs(g[shells].mean() - 1.0) < 0.01
    n = np.array([[1, 0, 0], [0, 2, 1], [3, 1, 1], [2, 2, 2], [5, 0, 1], [4, 3, 0], [1, 6, 2], [7, 1, 3]])
    vecs = np.concatenate([n, n[:, [1, 2, 0]], n[:, [2, 0, 1]]]) * (2 * np.pi / L)
    Sq = S.structure_factor(L, q, vecs)
    assert abs(Sq.mean() - 1.0) < 0.35              # exponential spread, 24 vectors
