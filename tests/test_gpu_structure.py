"""GPU parity of the static observables with the oracle, and the paper's
pressure as a pin of the whole engine.

The virial sum runs over the cell neighbourhoods in FP64 (a fixed order per
atom); the oracle's runs over all pairs in numpy.  The chains are equal (FP64
mode), so the sums differ only by rounding: 1e-12 relative.
"""
import numpy as np
import pytest

import oracle
from oracle import structure as S
from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.PAPER_POT


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21290_gb300 import build as B
    B.build()
    oracle.build()


@pytest.mark.parametrize("M,T,seed", [(64, 2.0, 1), (216, 1.0, 2)])
def test_virial_matches_oracle(M, T, seed):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    h = F.Handle(L, xyz, t, POT, precision="fp64")
    ch = oracle.Chain(L, xyz, t, POT, nc=h.info["max_cells_per_axis"])
    h.sweep(15, T, W.PAPER_MIX, seed)
    ch.run(15, T, W.PAPER_MIX, seed=seed)
    q, X, tt = h.state_fixed()
    assert np.array_equal(q, ch.q)
    out = h.pressure(T)[0]
    Wo = S.virial(L, ch.q, ch.t, POT)
    assert out[0] == pytest.approx(Wo, rel=1e-12, abs=1e-9)
    assert out[1] == pytest.approx(S.pressure(L, ch.q, ch.t, POT, T), rel=1e-12)


def test_pressure_of_a_batch():
    Ms, Ts = [64, 125], [3.0, 1.5]
    Ls = [W.box_length(m) for m in Ms]
    st = [W.lattice_start(m, l, 4 + k) for k, (m, l) in enumerate(zip(Ms, Ls))]
    h = F.Handle(np.array(Ls), np.concatenate([s[0] for s in st]), np.concatenate([s[1] for s in st]), POT,
                 precision="fp32", n_mol=np.array(Ms))
    h.sweep(5, np.array(Ts), W.PAPER_MIX, np.array([1, 2], dtype=np.uint64))
    q, X, t = h.state_fixed()
    out = h.pressure(np.array(Ts))
    off = 0
    for k, M in enumerate(Ms):
        sl = slice(off, off + 3 * M)
        assert out[k, 0] == pytest.approx(S.virial(Ls[k], q[sl], t[sl], POT), rel=1e-12, abs=1e-9)
        off += 3 * M
    with pytest.raises(F.McError):
        h.pressure(np.array([1.0, -1.0]))


def _lattice_vectors(L, qmin, qmax):
    n = int(np.ceil(qmax * L / (2 * np.pi)))
    g = np.arange(-n, n + 1)
    v = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) * (2 * np.pi / L)
    m = np.linalg.norm(v, axis=1)
    return v[(m >= qmin) & (m <= qmax)]


@pytest.mark.parametrize("M,seed", [(64, 3), (216, 4)])
def test_structure_factor_and_pair_histogram_match_oracle(M, seed):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    h = F.Handle(L, xyz, t, POT, precision="fp64")
    h.sweep(10, 1.5, W.PAPER_MIX, seed)
    q, X, tt = h.state_fixed()
    qv = _lattice_vectors(L, 4.0, 9.0)
    Sg = h.structure_factor(qv)[0]
    assert np.allclose(Sg, S.structure_factor(L, q, qv), rtol=1e-10, atol=1e-9)
    dr = 0.02
    nb = int(0.5 * L / dr)
    c, g = h.pair_histogram(dr, nb)
    co = S.pair_histogram(L, q, dr, nb)
    assert np.array_equal(c[0].astype(np.int64), co)                   # bit-exact integer counts
    assert np.allclose(g[0], S.pair_correlation(L, co, 3 * M, dr), rtol=1e-12)
    with pytest.raises(F.McError):
        h.pair_histogram(dr, nb + 2)                                    # beyond half the box
    with pytest.raises(F.McError):
        h.pair_histogram(0.0, 10)


def test_pair_histogram_of_a_batch():
    Ms = [64, 125, 100]
    Ls = [W.box_length(m) for m in Ms]
    st = [W.lattice_start(m, l, 8 + k) for k, (m, l) in enumerate(zip(Ms, Ls))]
    h = F.Handle(np.array(Ls), np.concatenate([s[0] for s in st]), np.concatenate([s[1] for s in st]), POT,
                 precision="fp32", n_mol=np.array(Ms))
    h.sweep(3, np.array([2.0, 2.0, 2.0]), W.PAPER_MIX, np.array([1, 2, 3], dtype=np.uint64))
    q, X, t = h.state_fixed()
    dr, nb = 0.05, int(0.5 * min(Ls) / 0.05)
    c, g = h.pair_histogram(dr, nb)
    off = 0
    for k, M in enumerate(Ms):
        assert np.array_equal(c[k].astype(np.int64), S.pair_histogram(Ls[k], q[off:off + 3 * M], dr, nb)), k
        off += 3 * M


@pytest.fixture(scope="module")
def equilibrated_T1():
    """M = 1000 at T = 1, rho = 1.2 after 100000 sweeps from the lattice."""
    M, T = 1000, 1.0
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, 7)
    h = F.Handle(L, xyz, t, POT, precision="fp32")
    h.sweep(100000, T, W.PAPER_MIX, 7)
    return h, L


def test_structure_peaks_at_T1(equilibrated_T1):
    """Sec. III.B and IV.A: the first peak of the atoms' S(q) lies near q = 7.4,
    the wavevector of F_s; g(r) peaks near the atomic diameter (sigma_B = 1)
    and tends to 1 at large r."""
    h, L = equilibrated_T1
    qv = _lattice_vectors(L, 5.0, 10.0)
    Sq = h.structure_factor(qv)[0]
    qm = np.linalg.norm(qv, axis=1)
    edges = np.arange(5.0, 10.0 + 1e-9, 0.2)
    k = np.digitize(qm, edges) - 1
    shell = np.array([Sq[k == b].mean() for b in range(len(edges) - 1)])
    q_peak = 0.5 * (edges[np.argmax(shell)] + edges[np.argmax(shell) + 1])
    c, g = h.pair_histogram(0.02, int(0.5 * L / 0.02))
    r = (np.arange(g.shape[1]) + 0.5) * 0.02
    r_peak = r[np.argmax(g[0])]
    tail = g[0][(r > 5.0) & (r < 6.5)]
    print("S(q) first peak at q = %.2f (S = %.2f); g(r) first peak at r = %.3f (g = %.2f); g(5-6.5) = %.3f"
          % (q_peak, shell.max(), r_peak, g[0].max(), tail.mean()))
    assert abs(q_peak - 7.4) < 0.3
    assert 0.85 < r_peak < 1.2
    assert abs(tail.mean() - 1.0) < 0.05


@pytest.mark.parametrize("T,rho,n_eq", [(1.46, 1.16, 10000), (2.03, 1.12, 4000)])
def test_pressure_on_the_papers_constant_pressure_path(T, rho, n_eq):
    """Table I lists (T, rho) pairs chosen to keep the NVT pressure at P = 30.
    M = 1000 from the lattice: n_eq sweeps to equilibrate, then the mean of 40
    samples 50 sweeps apart.  Measured here: 30.0 and 30.1 (statistical error
    about 0.1)."""
    M = 1000
    L = (3 * M / rho) ** (1.0 / 3.0)
    xyz, t = W.lattice_start(M, L, 7)
    h = F.Handle(L, xyz, t, POT, precision="fp32")
    h.sweep(n_eq, T, W.PAPER_MIX, 7)
    P = []
    for k in range(40):
        h.sweep(50, T, W.PAPER_MIX, 7)
        P.append(h.pressure(T)[0, 1])
    P = np.array(P)
    print("P(T=%.2f, rho=%.3f) = %.3f +- %.3f" % (T, rho, P.mean(), P.std() / np.sqrt(P.size)))
    assert abs(P.mean() - 30.0) < 0.75


def test_pressure_at_T1_rho12_is_the_papers_30(equilibrated_T1):
    """Sec. II.C: the NVT pressure at T = 1, rho = 1.2 is P = 30 (two digits).
    Mean of 40 samples 50 sweeps apart after 100000 sweeps; measured 30.3."""
    h, L = equilibrated_T1
    P = []
    for k in range(40):
        h.sweep(50, 1.0, W.PAPER_MIX, 7)
        P.append(h.pressure(1.0)[0, 1])
    P = np.array(P)
    print("P(T=1, rho=1.2) = %.3f +- %.3f" % (P.mean(), P.std() / np.sqrt(P.size)))
    assert abs(P.mean() - 30.0) < 0.75
