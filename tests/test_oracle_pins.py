"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms of Eq. 1-2, invariances of the energy, the
exact running-energy bookkeeping, and the Boltzmann stationarity of the chain.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2506_21290_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
POT = W.PAPER_POT


def _golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


def test_paper_constants_match_workloads():
    c = _golden_constants()
    assert W.SIGMA == (c["sigma_A"], c["sigma_B"], c["sigma_C"])
    assert (W.EPS, W.FENE_K, W.FENE_R0, W.RHO, W.P_FLIP) == (c["eps"], c["fene_K"], c["fene_R0"], c["rho"],
                                                            c["p_flip"])
    assert W.PAPER_MIX[1] == c["p_flip"] and W.PAPER_MIX[0] == 1.0 - c["p_flip"]
    assert (W.T_HIGH, W.T_LOW) == (c["T_highest"], c["T_lowest"])


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def _ulp(x):
    return math.ulp(x)


def test_own_log_against_libm():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.random(20000), 1.0 - rng.random(2000) * 1e-12, rng.random(2000) * 1e-300,
                         np.exp(rng.uniform(-700, 700, 4000)), [0.5, 2.0, 4.0, 1.0 - 2 ** -53, 2 ** -53, 1e-310]])
    worst = 0.0
    for x in xs:
        if x <= 0:
            continue
        ref = math.log(x)
        got = oracle.ln(x)
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, abs(got - ref) / _ulp(ref))
    assert worst <= 2.0, worst
    assert oracle.ln(1.0) == 0.0
    assert oracle.ln(0.0) == -math.inf
    assert math.isnan(oracle.ln(-1.0))


def test_wca_closed_forms():
    sig = W.SIGMA
    for a in range(3):
        for b in range(3):
            s = 0.5 * (sig[a] + sig[b])
            # U(sigma_ab) = 4(1 - 1) + 1 = eps exactly (Eq. 1, additive diameters)
            assert oracle.phi(s * s, a, b, False, POT) == 1.0
            rc = 2.0 ** (1.0 / 6.0) * s
            # vanishes beyond the cutoff
            assert oracle.phi((rc * 1.0001) ** 2, a, b, False, POT) == 0.0
            assert oracle.phi(4.0, a, b, False, POT) == 0.0
            # with r = 2^(1/6) s y: (s/r)^6 = y^-6 / 2, so U = (y^-6 - 1)^2 exactly,
            # a double zero at the cutoff (U ~ 36 (1-y)^2)
            for y in (0.9, 0.99, 0.999, 0.9999):
                u = oracle.phi((rc * y) ** 2, a, b, False, POT)
                assert u == pytest.approx((y ** -6 - 1.0) ** 2, rel=1e-7)
            # steep wall: U(0.8 sigma) = 4(0.8^-12 - 0.8^-6) + 1
            x = 0.8 ** -6
            assert oracle.phi((0.8 * s) ** 2, a, b, False, POT) == pytest.approx(4 * (x * x - x) + 1, rel=1e-14)


def test_fene_closed_forms():
    sig = W.SIGMA
    for a in range(3):
        for b in range(3):
            s = 0.5 * (sig[a] + sig[b])
            R = 1.5 * s
            wca_part = lambda r2: oracle.phi(r2, a, b, False, POT)
            fene = lambda r2: oracle.phi(r2, a, b, True, POT) - wca_part(r2)
            # -33.75 ln(1 - x) = 33.75 when 1 - x = 1/e
            r2 = R * R * (1.0 - math.exp(-1.0))
            assert fene(r2) == pytest.approx(33.75, rel=1e-13)
            # beyond the WCA cutoff a bond carries FENE alone; check against the
            # library logarithm at a few lengths in (2^(1/6) s, 1.5 s)
            for frac in (0.76, 0.85, 0.95, 0.999):
                r = frac * R
                assert oracle.phi(r * r, a, b, False, POT) == 0.0
                assert oracle.phi(r * r, a, b, True, POT) == pytest.approx(-33.75 * math.log1p(-frac * frac),
                                                                         rel=1e-12)
            # diverges at 1.5 sigma_ab
            assert fene(R * R * (1 - 1e-12)) > 900
            assert math.isinf(oracle.phi(R * R, a, b, True, POT))


def test_mag_closed_forms():
    """The conditioning scale mag(r2) that every FP32 tolerance is measured
    against: the summed magnitudes of the pieces of Eq. 1 (4 eps s^12,
    4 eps s^6, eps) inside the cutoff and, for a bond, of Eq. 2
    (K eps (|ln(1-x)| + x/(1-x))).  Closed forms at points where they are
    simple; a dropped term, a doubled 4 eps, a missing eps factor or x in
    place of x/(1-x) each fails one of them."""
    sig = W.SIGMA
    K = 33.75
    for a in range(3):
        for b in range(3):
            s = 0.5 * (sig[a] + sig[b])
            R = 1.5 * s
            rc2 = 2.0 ** (1.0 / 3.0) * s * s
            # r = sigma_ab: s^6 = s^12 = 1, so 4 + 4 + 1
            assert oracle.mag(s * s, a, b, False, POT) == 9.0
            # r^2 = y sigma_ab^2 inside the cutoff: 4 y^-6 + 4 y^-3 + 1
            for y in (0.85, 1.1, 1.25):
                assert oracle.mag(y * s * s, a, b, False, POT) == pytest.approx(4 * y ** -6 + 4 * y ** -3 + 1,
                                                                               rel=1e-14)
            # just inside the cutoff s^6 -> 1/2: 1 + 2 + 1; at and beyond it nothing
            assert oracle.mag(rc2 * (1 - 1e-12), a, b, False, POT) == pytest.approx(4.0, rel=1e-11)
            assert oracle.mag(rc2, a, b, False, POT) == 0.0
            assert oracle.mag(1.3 * rc2, a, b, False, POT) == 0.0
            # a bond beyond the WCA cutoff at 1 - x = 1/e: K (1 + (1 - 1/e) e) = K e
            r2 = R * R * (1.0 - math.exp(-1.0))
            assert r2 > rc2
            assert oracle.mag(r2, a, b, True, POT) == pytest.approx(K * math.e, rel=1e-13)
            # a bond at r = sigma_ab: both pieces, x = 1/2.25
            x = 1.0 / 2.25
            want = 9.0 + K * (abs(math.log(1.0 - x)) + x / (1.0 - x))
            assert oracle.mag(s * s, a, b, True, POT) == pytest.approx(want, rel=1e-13)
    # every piece scales with eps
    pot2 = list(POT)
    pot2[3] = 2.5
    assert oracle.mag(1.0, 1, 1, False, pot2) == 9.0 * 2.5
    r2 = 2.25 * (1.0 - math.exp(-1.0))
    assert oracle.mag(r2, 1, 1, True, pot2) == pytest.approx(2.5 * K * math.e, rel=1e-13)


def _random_start(M, seed=3):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    return L, xyz, t


def test_energy_invariances():
    M = 27
    L, xyz, t = _random_start(M)
    q = oracle.quantize(xyz, L)
    E = oracle.energy(L, q, t, POT)
    assert np.isfinite(E) and E > 0
    # global translation by any fixed-point vector: identical bits
    for shift in ([12345, 999999999, 3], [2 ** 31, 2 ** 31, 2 ** 31], [4294967295, 7, 0]):
        q2 = (q.astype(np.uint64) + np.array(shift, dtype=np.uint64)).astype(np.uint32)
        assert oracle.energy(L, q2, t, POT) == E
    rng = np.random.default_rng(1)
    # relabel molecules
    perm = rng.permutation(M)
    idx = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
    assert oracle.energy(L, q[idx], t[idx], POT) == pytest.approx(E, rel=1e-13)
    # permute the three sites inside every molecule, carrying their types
    inner = np.stack([rng.permutation(3) for _ in range(M)])
    idx = (3 * np.arange(M)[:, None] + inner).reshape(-1)
    assert oracle.energy(L, q[idx], t[idx], POT) == pytest.approx(E, rel=1e-13)
    # a periodic image of a whole molecule is the same configuration
    xyz2 = xyz.copy()
    xyz2[0:3] += np.array([L, -2 * L, 5 * L])
    assert oracle.energy(L, oracle.quantize(xyz2, L), t, POT) == E


def test_energy_pair_decomposition():
    """Two molecules far apart: E = E(mol 0) + E(mol 1), each a sum of 3 bonded
    pair energies (WCA + FENE), computed here from the pair routine."""
    L = 20.0
    tpl = W._template()
    xyz = np.concatenate([tpl + 3.0, tpl + 13.0])
    t = np.array([0, 1, 2, 2, 0, 1], dtype=np.int32)
    q = oracle.quantize(xyz, L)
    h = L / 2 ** 32
    E_parts = 0.0
    for m in range(2):
        for i, j in ((0, 1), (0, 2), (1, 2)):
            a, b = 3 * m + i, 3 * m + j
            d = (q[b] - q[a]).view(np.int32).astype(np.float64) * h
            E_parts += oracle.phi(float((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]), t[a], t[b], True, POT)
    assert oracle.energy(L, q, t, POT) == pytest.approx(E_parts, rel=1e-14)


@pytest.mark.parametrize("mix", [W.PAPER_MIX, W.RIGID_MIX, (0.0, 0.0, 0.5, 0.5, 0.1, 0.05, 0.1)])
def test_running_energy_matches_brute_force(mix):
    """Sum of accepted Delta E (single-site O(N) loops) = change of the O(N^2)
    total energy: catches a dropped term, a wrong sign or a wrong index."""
    M = 64
    L, xyz, t = _random_start(M, seed=5)
    ch = oracle.Chain(L, xyz, t, POT, nc=2)
    lg = ch.run(30, 2.0, mix, seed=11, log=True)
    assert ch.counters[4:].sum() > 100
    Eb = ch.energy()
    assert ch.e_run == pytest.approx(Eb, rel=1e-12)
    acc = lg["accepted"] == 1
    assert np.all(lg["status"][acc] == oracle.ST_EVAL)


def test_sweep_structure():
    M = 125
    L, xyz, t = _random_start(M, seed=2)
    ch = oracle.Chain(L, xyz, t, POT, nc=4)
    t_before = ch.t.copy()
    lg = ch.run(3, 3.0, W.PAPER_MIX, seed=4, log=True)
    assert lg.size == 3 * 3 * M                    # one MC step = N attempted moves
    assert ch.counters[:4].sum() == 3 * 3 * M
    # flips change types, never indices: each molecule still holds one A, B, C
    assert np.all(np.sort(ch.t.reshape(-1, 3), axis=1) == np.array([0, 1, 2]))
    assert np.any(ch.t != t_before)
    # unwrapped and wrapped positions agree modulo 2^32
    assert np.all((ch.X & 0xFFFFFFFF).astype(np.uint32) == ch.q)
    # log status codes are the documented ones; moves left unevaluated carry NaN
    assert set(np.unique(lg["status"])) <= {0, 1, 2, 3}
    assert np.all(np.isnan(lg["dE"][lg["status"] != 0]))


def test_cells_keep_their_sites_within_a_sweep():
    """No accepted move takes an atom out of its cell: with the sweep's shift,
    the cell of every atom is the same before and after the sweep."""
    M = 125
    L, xyz, t = _random_start(M, seed=8)
    ch = oracle.Chain(L, xyz, t, POT, nc=4)
    nc = 4
    for s in range(3):
        shift = oracle.sweep_shift(ch.sweep, 9)

        def cells(q):
            c = ((q.astype(np.uint64) + shift.astype(np.uint64)) & 0xFFFFFFFF) * nc >> 32
            return (c[:, 2] * nc + c[:, 1]) * nc + c[:, 0]

        before = cells(ch.q)
        ch.run(1, 3.0, W.PAPER_MIX, seed=9)
        assert np.array_equal(before, cells(ch.q))


def _two_molecules():
    """Two equilateral molecules (side 0.97) with a few intermolecular contacts.
    Type permutations leave each molecule's own energy unchanged, so the 36
    type states differ only through the contacts (a spread of about 4 eps)."""
    L = 3.3
    side = 0.97
    tri = np.array([[0, 0, 0], [side, 0, 0], [side / 2, side * math.sqrt(3) / 2, 0]])
    tri -= tri.mean(axis=0)
    R = W._random_rotations(np.random.default_rng(0), 2)
    xyz = np.concatenate([tri @ R[0].T + 0.8, tri @ R[1].T + np.array([0.8, 0.8, 0.8 + 1.35])])
    return L, xyz


def test_flip_chain_is_boltzmann_stationary():
    """Flip-only chain on two molecules with frozen positions: the 36 type
    states are visited with probability exp(-E/T)/Z (Sec. II.B: Metropolis
    with a symmetric flip proposal)."""
    L, xyz = _two_molecules()
    q = oracle.quantize(xyz, L)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    T = 2.0
    states = {}
    E = []
    for i, p0 in enumerate(perms):
        for j, p1 in enumerate(perms):
            t = np.array(p0 + p1, dtype=np.int32)
            states[tuple(t)] = len(E)
            E.append(oracle.energy(L, q, t, POT))
    E = np.array(E)
    w = np.exp(-(E - E.min()) / T)
    p_exact = w / w.sum()
    assert p_exact.min() > 2e-3      # every state is reachable in a reasonable run
    ch = oracle.Chain(L, q=q, types=np.array([0, 1, 2, 0, 1, 2], dtype=np.int32), pot=POT, nc=2)
    mix = (0.0, 1.0, 0.0, 0.0, 0.1, 0.05, 0.05)
    counts = np.zeros(36)
    n_samples = 60000
    for _ in range(n_samples):
        ch.run(4, T, mix, seed=21)
        counts[states[tuple(ch.t)]] += 1
    assert np.all(ch.q == q)            # flips never move atoms
    expected = p_exact * n_samples
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 90.0, (chi2, counts, expected)   # 35 dof; allows for residual correlation


def test_rotation_chain_samples_uniform_orientations():
    """A single molecule with only rigid rotations feels no torque: its
    orientation must become uniform on the sphere (<u_z^2> = 1/3, flat cos)."""
    L = 4.0
    tpl = W._template()
    xyz = tpl + 2.0
    t = np.array([0, 1, 2], dtype=np.int32)
    ch = oracle.Chain(L, xyz, t, POT, nc=2)
    mix = (0.0, 0.0, 0.0, 1.0, 0.1, 0.05, 0.4)
    cz = []
    for _ in range(6000):
        ch.run(3, 1.0, mix, seed=5)
        d = (ch.q[1] - ch.q[0]).view(np.int32).astype(np.float64)
        cz.append(d[2] / np.linalg.norm(d))
    cz = np.array(cz[500:])
    assert np.mean(cz * cz) == pytest.approx(1.0 / 3.0, abs=0.03)
    hist, _ = np.histogram(cz, bins=5, range=(-1, 1))
    assert hist.min() > 0.75 * hist.mean()


def _bond_density(T, r_grid, pot):
    """Marginal density of |r_1 - r_0| for one free molecule, by quadrature:
    p(r) ~ r^2 exp(-phi01(r)/T) Int d^3 r2 exp(-(phi02 + phi12)/T)."""
    t = (0, 1, 2)
    z = np.linspace(-2.0, 3.0, 501)
    rho = np.linspace(1e-4, 2.5, 500)
    Z, P = np.meshgrid(z, rho, indexing="ij")
    dz, drho = z[1] - z[0], rho[1] - rho[0]
    def vphi(r2, a, b):
        v = oracle.phi_many(r2, a, b, True, pot)
        return np.where(np.isnan(v) | (r2 >= (1.5 * 0.5 * (W.SIGMA[a] + W.SIGMA[b])) ** 2), np.inf, v)
    r02 = Z * Z + P * P
    e02 = np.exp(-vphi(r02, t[0], t[2]) / T)
    out = []
    for r in r_grid:
        r12 = (Z - r) ** 2 + P * P
        inner = (e02 * np.exp(-vphi(r12, t[1], t[2]) / T) * 2 * np.pi * P).sum() * dz * drho
        out.append(r * r * math.exp(-oracle.phi(r * r, t[0], t[1], True, pot) / T) * inner)
    out = np.array(out)
    return out / (out.sum() * (r_grid[1] - r_grid[0]))


@pytest.mark.slow
def test_translation_chain_bond_length_distribution():
    """One molecule, atom translations only: the A-B bond length histogram
    follows the Boltzmann marginal computed by quadrature."""
    L = 4.0
    tpl = W._template()
    ch = oracle.Chain(L, tpl + 2.0, np.array([0, 1, 2], dtype=np.int32), POT, nc=2)
    mix = (1.0, 0.0, 0.0, 0.0, 0.15, 0.05, 0.05)
    T = 2.0
    rs = []
    for _ in range(40000):
        ch.run(2, T, mix, seed=13)
        d = (ch.q[1] - ch.q[0]).view(np.int32).astype(np.float64) * (L / 2 ** 32)
        rs.append(np.linalg.norm(d))
    rs = np.array(rs[1000:])
    edges = np.linspace(0.7, 1.25, 23)
    hist, _ = np.histogram(rs, bins=edges, density=True)
    centres = 0.5 * (edges[1:] + edges[:-1])
    fine = np.linspace(0.7, 1.25, 221)
    dens = _bond_density(T, fine, POT)
    ref = np.array([dens[(fine >= lo) & (fine <= hi)].mean() for lo, hi in zip(edges[:-1], edges[1:])])
    ref /= (ref * np.diff(edges)).sum()
    mask = ref > 0.2
    assert np.max(np.abs(hist[mask] - ref[mask]) / ref[mask]) < 0.15, (centres[mask], hist[mask], ref[mask])
    assert abs(rs.mean() - (centres * ref * np.diff(edges)).sum()) < 0.01


def _energy_series(mix, n_sweeps, seed, M=32, T=3.0, burn=1500):
    L, xyz, t = _random_start(M, seed=4)
    ch = oracle.Chain(L, xyz, t, POT, nc=2)
    ch.run(burn, T, mix, seed=seed)
    E = np.empty(n_sweeps)
    for k in range(n_sweeps):
        ch.run(1, T, mix, seed=seed)
        E[k] = ch.e_run
    assert ch.e_run == pytest.approx(ch.energy(), rel=1e-10)
    return E


def _block_mean_se(x, nblocks=40):
    b = x[: len(x) // nblocks * nblocks].reshape(nblocks, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nblocks)


@pytest.mark.slow
def test_flip_and_local_mc_sample_the_same_energies():
    """Sec. II.C: energy distributions of flip MC (p_flip = 0.2) and of local
    MC (translations only) coincide; here at T = 3 on 32 molecules."""
    Ef = _energy_series(W.PAPER_MIX, 16000, seed=1)
    El = _energy_series(W.LOCAL_MIX, 16000, seed=2)
    mf, sf = _block_mean_se(Ef)
    ml, sl = _block_mean_se(El)
    assert abs(mf - ml) < 4.0 * math.hypot(sf, sl), (mf, sf, ml, sl)
    assert Ef.std() == pytest.approx(El.std(), rel=0.12)
