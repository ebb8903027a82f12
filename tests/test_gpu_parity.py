"""GPU parity: the CUDA library against the FP64 oracle, element by element.

FP64 mode must reproduce the oracle's chain bit for bit: positions (fixed
point), unwrapped positions, types, and every attempt's site, move, status,
decision and Delta E.  FP32 mode must take the same decisions (the FP64
recheck near the threshold makes them identical) and agree on every
evaluated Delta E within 1e-5 of the move's conditioning scale.
"""
import numpy as np
import pytest

import oracle
from oracle import observables as O
from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.PAPER_POT
TOL_FP32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21290_gb300 import build as B
    B.build()
    oracle.build()


def _start(M, seed, L=None):
    L = W.box_length(M) if L is None else L
    xyz, t = W.lattice_start(M, L, seed)
    return L, xyz, t


def _pair(M, seed, precision, nc=0, L=None):
    L, xyz, t = _start(M, seed, L)
    h = F.Handle(L, xyz, t, POT, precision=precision, n_cells=nc)
    nc_used = h.info["max_cells_per_axis"]
    ch = oracle.Chain(L, xyz, t, POT, nc=nc_used)
    return h, ch


def _compare_state(h, ch):
    q, X, t = h.state_fixed()
    assert np.array_equal(q, ch.q), "positions differ"
    assert np.array_equal(X, ch.X), "unwrapped positions differ"
    assert np.array_equal(t, ch.t), "types differ"


def _compare_logs_exact(lg, lo):
    assert lg.size == lo.size
    for f in ("site", "move", "status", "accepted"):
        bad = np.nonzero(lg[f] != lo[f])[0]
        assert bad.size == 0, (f, bad[:5], lg[bad[:5]], lo[bad[:5]])
    ev = lo["status"] == 0
    assert np.array_equal(lg["dE"][ev], lo["dE"][ev])          # bit-exact FP64
    assert np.all(np.isnan(lg["dE"][~ev]))


@pytest.mark.parametrize("M,nc,seed,T,mix", [
    (64, 2, 0, 3.0, W.PAPER_MIX),          # tiny box, 8 distinct neighbour cells
    (125, 4, 1, 2.0, W.PAPER_MIX),         # 27-cell neighbourhoods, ragged cells
    (64, 2, 2, 2.0, W.RIGID_MIX),          # all four move types
    (216, 4, 3, 1.0, W.RIGID_MIX),
])
def test_fp64_trajectory_and_log_bit_exact(M, nc, seed, T, mix):
    h, ch = _pair(M, seed, "fp64", nc)
    assert h.info["max_cells_per_axis"] == nc
    lg = h.sweep_logged(20, T, mix, 100 + seed)
    lo = ch.run(20, T, mix, seed=100 + seed, log=True)
    _compare_logs_exact(lg, lo)
    _compare_state(h, ch)
    st = h.stats()[0]
    assert st["attempts"] == list(ch.counters[:4])
    assert st["accepts"] == list(ch.counters[4:])
    assert st["e_run"] == pytest.approx(ch.e_run, rel=1e-12, abs=1e-9)


def test_fp64_100_sweeps_bit_exact_small_config():
    """Tiny box of the paper's density at T = 3, seed 0, paper mix: 100 sweeps."""
    h, ch = _pair(64, 0, "fp64")
    h.sweep(100, 3.0, W.PAPER_MIX, 0)
    ch.run(100, 3.0, W.PAPER_MIX, seed=0)
    _compare_state(h, ch)
    E = h.energy()[0]
    assert E == pytest.approx(ch.energy(), rel=1e-12)
    assert h.stats()[0]["e_run"] == pytest.approx(E, rel=1e-10)


def test_fp64_1000_molecules_bit_exact():
    """1000 molecules (n_c = 8, 512 cells): several tiles and ragged cells."""
    h, ch = _pair(1000, 1, "fp64")
    h.sweep(3, 1.1, W.PAPER_MIX, 1)
    ch.run(3, 1.1, W.PAPER_MIX, seed=1)
    _compare_state(h, ch)


@pytest.mark.parametrize("M,seed,T,mix,wpc", [(125, 4, 2.0, W.PAPER_MIX, 1), (125, 4, 2.0, W.PAPER_MIX, 2),
                                               (125, 4, 2.0, W.PAPER_MIX, 4), (216, 5, 0.75, W.RIGID_MIX, 1),
                                               (216, 5, 0.75, W.RIGID_MIX, 4), (64, 6, 3.0, W.PAPER_MIX, 2),
                                               (343, 7, 1.1, W.PAPER_MIX, 0), (343, 8, 1.1, W.PAPER_MIX, 8),
                                               (216, 9, 0.75, W.RIGID_MIX, 8)])
def test_fp32_same_decisions_and_dE_within_tolerance(M, seed, T, mix, wpc):
    L, xyz, t = _start(M, seed)
    h = F.Handle(L, xyz, t, POT, precision="fp32", warps_per_cell=wpc)
    assert wpc == 0 or h.info["warps_per_cell"] == wpc
    ch = oracle.Chain(L, xyz, t, POT, nc=h.info["max_cells_per_axis"])
    lg = h.sweep_logged(15, T, mix, 7 + seed)
    lo = ch.run(15, T, mix, seed=7 + seed, log=True)
    for f in ("site", "move", "status", "accepted"):
        assert np.array_equal(lg[f], lo[f]), f
    _compare_state(h, ch)
    ev = lo["status"] == 0
    err = np.abs(lg["dE"][ev] - lo["dE"][ev])
    scale = np.maximum(np.abs(lo["dE"][ev]), lo["scale"][ev])
    assert np.all(err <= TOL_FP32 * scale), (err / scale).max()
    re = (lg["flags"] & 1) == 1
    assert np.array_equal(lg["dE64"][re & ev], lo["dE"][re & ev])     # rechecks are the exact FP64 value


# FP32 Delta E error bound that the default recheck margin (1e-5 of the summed
# magnitudes) relies on: distances to 7-9 units of FP32 rounding, each term's
# sensitivity to them (at most 6x its magnitude for WCA), its own evaluation
# (about 31 units) and the sums (at most 21 units) give <= 106 u = 6.3e-6.
FP32_DE_BOUND = 6.3e-6


@pytest.mark.parametrize("M,seed,T,mix", [(343, 51, 1.1, W.PAPER_MIX), (216, 52, 0.75, W.RIGID_MIX),
                                          (64, 53, 2.0, W.RIGID_MIX)])
def test_fp32_error_within_derived_bound(M, seed, T, mix):
    """Every FP32 Delta E is within FP32_DE_BOUND x (the oracle's summed term
    magnitudes) of the oracle's FP64 value, on the split-coordinate path and
    on the n_c = 2 raw-record path; so with the default margin no decision
    taken in FP32 can differ from the FP64 one."""
    L, xyz, t = _start(M, seed)
    h = F.Handle(L, xyz, t, POT, precision="fp32")
    ch = oracle.Chain(L, xyz, t, POT, nc=h.info["max_cells_per_axis"])
    assert h.info["recheck_gap"] == pytest.approx(1e-5)
    lg = h.sweep_logged(20, T, mix, seed)
    lo = ch.run(20, T, mix, seed=seed, log=True)
    assert np.array_equal(lg["accepted"], lo["accepted"])
    ev = (lo["status"] == 0) & ((lg["flags"] & 1) == 0)
    assert ev.sum() > 1000
    err = np.abs(lg["dE"][ev] - lo["dE"][ev])
    # measured against the oracle's own scale (pinned to its closed forms on
    # the CPU), not the library's
    assert np.all(err <= FP32_DE_BOUND * lo["scale"][ev]), (err / lo["scale"][ev]).max()


def test_energy_matches_brute_force():
    for M in (64, 343, 1000):
        L, xyz, t = _start(M, 9)
        h = F.Handle(L, xyz, t, POT, precision="fp32")
        h.sweep(2, 1.5, W.PAPER_MIX, 3)
        q, X, tt = h.state_fixed()
        assert h.energy()[0] == pytest.approx(oracle.energy(L, q, tt, POT), rel=1e-12)


def test_observables_match_numpy_oracle():
    M = 343
    L, xyz, t = _start(M, 11)
    h = F.Handle(L, xyz, t, POT, precision="fp32")
    h.set_t0()
    q0, X0, t0 = h.state_fixed()
    h.sweep(40, 3.0, W.PAPER_MIX, 5)
    q, X, tt = h.state_fixed()
    qa, qc = W.qvectors(L, 7.4), W.qvectors(L, 5.1)
    out, fs, fscm, c2 = h.observables(qa, qc, per_particle=True)
    kref = O.reference_sites(t0)
    ref = O.observables(L, X, X0, q, O.orientation(q0, L, kref), kref, qa, qc)
    assert out[0, 0] == pytest.approx(ref["F_s"], abs=1e-12)
    assert out[0, 1] == pytest.approx(ref["F_s_cm"], abs=1e-12)
    assert out[0, 2] == pytest.approx(ref["C_2"], abs=1e-12)
    assert np.allclose(fs, ref["F_s_i"], atol=1e-12)
    assert np.allclose(fscm, ref["F_s_cm_i"], atol=1e-12)
    assert np.allclose(c2, ref["C_2_i"], atol=1e-12)
    assert 0.0 < out[0, 0] < 1.0 and out[0, 2] < 1.0


def test_batched_replicas_match_independent_oracle_runs():
    Ms = [64, 125, 100, 216]
    Ts = [3.0, 1.0, 2.0, 0.75]
    seeds = [0, 1, 2, 3]
    Ls, xyzs, ts = [], [], []
    for k, M in enumerate(Ms):
        L, xyz, t = _start(M, 20 + k)
        Ls.append(L); xyzs.append(xyz); ts.append(t)
    h = F.Handle(np.array(Ls), np.concatenate(xyzs), np.concatenate(ts), POT, precision="fp64",
                 n_mol=np.array(Ms))
    h.sweep(6, np.array(Ts), W.PAPER_MIX, np.array(seeds, dtype=np.uint64))
    q, X, t = h.state_fixed()
    off = 0
    for k, M in enumerate(Ms):
        nc = 2 if Ls[k] < 4 * 1.575 else None
        ch = oracle.Chain(Ls[k], xyzs[k], ts[k], POT)
        # the replica's cells per axis: largest even n_c with cells >= 1.575 wide
        n = 2
        while np.floor(2 ** 32 / (n + 2)) * Ls[k] / 2 ** 32 >= 1.575:
            n += 2
        ch.run(6, Ts[k], W.PAPER_MIX, seed=seeds[k], nc=n)
        sl = slice(off, off + 3 * M)
        assert np.array_equal(q[sl], ch.q), k
        assert np.array_equal(t[sl], ch.t), k
        off += 3 * M


def test_runs_are_reproducible_and_resumable():
    L, xyz, t = _start(343, 12)
    a = F.Handle(L, xyz, t, POT, precision="fp32")
    b = F.Handle(L, xyz, t, POT, precision="fp32")
    a.sweep(10, 1.2, W.PAPER_MIX, 99)
    b.sweep(4, 1.2, W.PAPER_MIX, 99)
    # checkpoint b after 4 sweeps, restore exactly into a fresh handle c, continue there
    q4, X4, t4 = b.state_fixed()
    c = F.Handle(L, xyz, t, POT, precision="fp32")
    c.set_state_fixed(q4, X4, t4)
    c.set_sweep(4)
    c.sweep(6, 1.2, W.PAPER_MIX, 99)
    b.sweep(6, 1.2, W.PAPER_MIX, 99)
    qa, Xa, ta = a.state_fixed()
    qb, Xb, tb = b.state_fixed()
    qc, Xc, tc = c.state_fixed()
    assert np.array_equal(qa, qb) and np.array_equal(ta, tb) and np.array_equal(Xa, Xb)
    assert np.array_equal(qa, qc) and np.array_equal(ta, tc) and np.array_equal(Xa, Xc)
    assert a.stats()[0]["e_run"] == b.stats()[0]["e_run"]
    # a restore through doubles lands on the same fixed-point grid when the
    # positions are cell centres of the grid (q + 1/2) h
    d = F.Handle(L, (q4.astype(np.float64) + 0.5) * (L / 2 ** 32), t4, POT, precision="fp32")
    assert np.array_equal(d.state_fixed()[0], q4)


@pytest.mark.parametrize("precision,M", [("fp32", 343), ("fp64", 125)])
def test_autotune_leaves_the_chain_unchanged(precision, M):
    """mc_autotune times every schedule from a snapshot and restores it: the
    chain after it is the chain without it, bit for bit (positions, types,
    decisions); only the cell schedule may differ."""
    L, xyz, t = _start(M, 41)
    a = F.Handle(L, xyz, t, POT, precision=precision)
    b = F.Handle(L, xyz, t, POT, precision=precision)
    for h in (a, b):
        h.sweep(3, 1.4, W.PAPER_MIX, 23)
    res = a.autotune(3, 1.4, W.PAPER_MIX, 23)
    assert res.shape == (8,) and (res > 0).any()
    assert a.info["warps_per_cell"] in (1, 2, 4, 8)
    ms = {(w, form == 0): res[4 * form + k] for form in (0, 1) for k, w in enumerate((1, 2, 4, 8))}
    chosen = ms[(a.info["warps_per_cell"], a.info["persistent_blocks"] > 0)]
    assert chosen == min(v for v in res if v > 0)
    for h in (a, b):
        h.sweep(5, 1.4, W.PAPER_MIX, 23)
        h.sweep(2, 2.2, W.RIGID_MIX, 24)
    qa, Xa, ta = a.state_fixed()
    qb, Xb, tb = b.state_fixed()
    assert np.array_equal(qa, qb) and np.array_equal(Xa, Xb) and np.array_equal(ta, tb)
    sa, sb = a.stats()[0], b.stats()[0]
    for k in ("attempts", "accepts", "rejected_geometry", "rejected_bond", "fp64_rechecks", "sweeps"):
        assert sa[k] == sb[k], k
    # the running energy sums the same accepted Delta E; in FP32 mode a cell's
    # FP32 partial sums depend on how its attempts were spread over warps
    assert sa["e_run"] == pytest.approx(sb["e_run"], rel=1e-9, abs=1e-6)


@pytest.mark.parametrize("precision,wpc,M", [("fp64", 1, 125), ("fp32", 1, 343), ("fp32", 2, 343), ("fp32", 4, 1000),
                                             ("fp64", 4, 216), ("fp32", 8, 1000), ("fp64", 8, 125)])
def test_persistent_launch_matches_graphs(precision, wpc, M):
    """One cooperative launch for all sweeps of a call gives the same chain,
    bit for bit, as one CUDA graph per sweep."""
    L, xyz, t = _start(M, 31)
    hg = F.Handle(L, xyz, t, POT, precision=precision, warps_per_cell=wpc, launch_mode=1)
    hp = F.Handle(L, xyz, t, POT, precision=precision, warps_per_cell=wpc, launch_mode=2)
    for h in (hg, hp):
        h.sweep(7, 1.3, W.PAPER_MIX, 17)
        h.sweep(4, 2.0, W.RIGID_MIX, 18)
    qg, Xg, tg = hg.state_fixed()
    qp, Xp, tp = hp.state_fixed()
    assert np.array_equal(qg, qp) and np.array_equal(Xg, Xp) and np.array_equal(tg, tp)
    sg, sp = hg.stats()[0], hp.stats()[0]
    assert sg == sp
    if precision == "fp64":
        ch = oracle.Chain(L, xyz, t, POT, nc=hp.info["max_cells_per_axis"])
        ch.run(7, 1.3, W.PAPER_MIX, seed=17)
        ch.run(4, 2.0, W.RIGID_MIX, seed=18)
        _compare_state(hp, ch)


def test_kernels_are_built_for_sm_103():
    L, xyz, t = _start(64, 0)
    h = F.Handle(L, xyz, t, POT)
    assert h.info["binary_version"] == 103


def test_invalid_inputs_are_rejected():
    L, xyz, t = _start(64, 0)
    bad_t = t.copy()
    bad_t[5] = 3
    with pytest.raises(F.McError) as e:
        F.Handle(L, xyz, bad_t, POT)
    assert e.value.code == F.MC_ERR_INVALID_ARG
    broken = xyz.copy()
    broken[1] += 1.4        # stretch a bond past 1.5 sigma_ab
    with pytest.raises(F.McError) as e:
        F.Handle(L, broken, t, POT)
    assert e.value.code == F.MC_ERR_BAD_STATE
    with pytest.raises(F.McError) as e:
        F.Handle(3.0, xyz[:3], t[:3], POT)          # box below two interaction ranges
    assert e.value.code == F.MC_ERR_INVALID_ARG
    h = F.Handle(L, xyz, t, POT)
    with pytest.raises(F.McError):
        h.sweep(1, -1.0, W.PAPER_MIX, 0)
    with pytest.raises(F.McError):
        h.sweep(1, 1.0, (0.5, 0.2, 0, 0, 0.1, 0.05, 0.05), 0)
    # a staging capacity below the neighbourhood size is reported, not ignored
    h2 = F.Handle(W.box_length(1000), *W.lattice_start(1000, W.box_length(1000), 0), POT, stencil_cap=32)
    h2.sweep(1, 1.0, W.PAPER_MIX, 0)
    with pytest.raises(F.McError) as e:
        h2.sync()
    assert e.value.code == F.MC_ERR_CELL_OVERFLOW


def test_sparse_box_with_empty_cells():
    """Two molecules in a large box: most cells are empty, the chain still
    matches the oracle exactly."""
    L = 8.0
    tpl = W._template()
    xyz = np.concatenate([tpl + 1.0, tpl + 5.0])
    t = np.array([0, 1, 2, 0, 1, 2], dtype=np.int32)
    h = F.Handle(L, xyz, t, POT, precision="fp64")
    nc = h.info["max_cells_per_axis"]
    ch = oracle.Chain(L, xyz, t, POT, nc=nc)
    h.sweep(50, 2.0, W.RIGID_MIX, 4)
    ch.run(50, 2.0, W.RIGID_MIX, seed=4)
    _compare_state(h, ch)
