"""Parity at the full sizes of the measured workloads.

M = 8000 (single-8000): the FP32 chain, in the launch form the bench times,
is compared with the FP64 oracle's chain over two sweeps, atom for atom.

M = 64000 (large-64000): the oracle's O(N) Delta E per move makes a sweep
take minutes, so the checks are properties that hold at any size:
  - the persistent launch, whose colour phases are ordered cell by cell, gives
    the chain of the graph path, which orders them by kernel boundaries;
  - FP32 and FP64 modes give the same chain (every FP32 decision is the FP64
    one);
  - the running FP64 total agrees with a full FP64 recompute;
  - the FP64 total energy is unchanged by a global translation of the
    fixed-point positions, which moves every atom relative to the cell grid.
"""
import numpy as np
import pytest

import oracle
from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.PAPER_POT


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21290_gb300 import build as B
    B.build()
    oracle.build()


def _workload(name):
    spec = W.WORKLOADS[name]
    M = spec["M"]
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, spec["seed"])
    return L, xyz, t, spec["T"], spec["seed"]


def test_single_8000_fp32_chain_equals_oracle():
    L, xyz, t, T, seed = _workload("single-8000")
    h = F.Handle(L, xyz, t, POT, precision="fp32")       # the schedule mc_create picks, persistent launch
    assert h.info["persistent_blocks"] > 0
    ch = oracle.Chain(L, xyz, t, POT, nc=h.info["max_cells_per_axis"])
    h.sweep(2, T, W.PAPER_MIX, seed)
    ch.run(2, T, W.PAPER_MIX, seed=seed)
    q, X, tt = h.state_fixed()
    assert np.array_equal(q, ch.q) and np.array_equal(X, ch.X) and np.array_equal(tt, ch.t)
    # FP32 mode's running total sums the FP32 Delta E of the accepted moves
    assert h.stats()[0]["e_run"] == pytest.approx(ch.e_run, rel=1e-6)


def test_large_64000_properties():
    L, xyz, t, T, seed = _workload("large-64000")
    hp = F.Handle(L, xyz, t, POT, precision="fp32", launch_mode=2)
    hg = F.Handle(L, xyz, t, POT, precision="fp32", launch_mode=1)
    h64 = F.Handle(L, xyz, t, POT, precision="fp64", launch_mode=2)
    for h in (hp, hg, h64):
        h.sweep(2, T, W.PAPER_MIX, seed)
    qp, Xp, tp = hp.state_fixed()
    for other in (hg, h64):
        q, X, tt = other.state_fixed()
        assert np.array_equal(qp, q) and np.array_equal(Xp, X) and np.array_equal(tp, tt)
    sp, sg, s64 = hp.stats()[0], hg.stats()[0], h64.stats()[0]
    assert sp["accepts"] == sg["accepts"] == s64["accepts"]
    assert sum(sp["attempts"]) == 2 * 3 * 64000
    E = hp.energy()[0]
    assert sp["e_run"] == pytest.approx(E, rel=1e-6)
    assert s64["e_run"] == pytest.approx(h64.energy()[0], rel=1e-10)
    # a global translation by a fixed-point vector: the same configuration, seen
    # from a shifted cell grid
    shift = np.array([0x12345678, 0x9ABCDEF0, 0x0F1E2D3C], dtype=np.uint64)
    q_shift = ((qp.astype(np.uint64) + shift[None, :]) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    hs = F.Handle(L, xyz, t, POT, precision="fp32")
    hs.set_state_fixed(q_shift, None, tp)
    assert hs.energy()[0] == pytest.approx(E, rel=1e-12)


def test_batched_256_energies_equal_the_oracles_brute_force():
    """The whole batched workload (256 replicas, 823k atoms), after three FP32
    sweeps in the launch form the bench times: the per-replica FP64 energies
    (warp per cell, neighbour cells) against the oracle's brute force over all
    pairs of the same fixed-point state, for the smallest, the largest and
    a spread of replicas."""
    Ms, Ts = W.replica_mix(W.WORKLOADS["batched-256"]["R"], seed=W.WORKLOADS["batched-256"]["seed"])
    Ls = np.array([W.box_length(int(M)) for M in Ms])
    starts = [W.lattice_start(int(M), Ls[k], k) for k, M in enumerate(Ms)]
    h = F.Handle(Ls, np.concatenate([s[0] for s in starts]), np.concatenate([s[1] for s in starts]), POT,
                 precision="fp32", n_mol=Ms.astype(np.int32), warps_per_cell=1, launch_mode=1)
    h.sweep(3, Ts, W.PAPER_MIX, np.arange(len(Ms), dtype=np.uint64))
    E = h.energy()
    q, X, t = h.state_fixed()
    offs = np.concatenate([[0], np.cumsum(3 * Ms)])
    pick = sorted(set([int(np.argmin(Ms)), int(np.argmax(Ms))] + list(range(0, len(Ms), 37))))
    for k in pick:
        sl = slice(offs[k], offs[k + 1])
        assert E[k] == pytest.approx(oracle.energy(float(Ls[k]), q[sl], t[sl], POT), rel=1e-12), k
