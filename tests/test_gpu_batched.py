"""Batched FP32 parity at the scale the batched bench runs: replicas of uneven
size (from the smallest boxes, n_c = 4 with the largest neighbourhoods, up to
2000 molecules) at mixed temperatures, one warp per cell, against independent
oracle chains.  The attempt-by-attempt log (separate kernels) takes the
oracle's decisions with Delta E within the FP32 bound; the graph-per-sweep and
the persistent launches end in the oracle's states bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.PAPER_POT
MS = [256, 337, 338, 700, 1100, 1500, 1800, 2000]
TS = [0.75, 3.0, 1.2, 2.2, 0.9, 1.6, 2.8, 0.75]
SWEEPS = 2


@pytest.fixture(scope="module")
def batch():
    from paper_2506_21290_gb300 import build as B
    B.build()
    oracle.build()
    Ls = np.array([W.box_length(M) for M in MS])
    starts = [W.lattice_start(M, Ls[k], 60 + k) for k, M in enumerate(MS)]
    xyz = np.concatenate([s[0] for s in starts])
    t = np.concatenate([s[1] for s in starts])
    seeds = np.arange(len(MS), dtype=np.uint64) + np.uint64(500)
    chains, logs = [], []
    for k, M in enumerate(MS):
        nc, _ = F.mc_cell_grid(Ls[k], starts[k][1], POT)
        ch = oracle.Chain(Ls[k], starts[k][0], starts[k][1], POT, nc=nc)
        logs.append(ch.run(SWEEPS, TS[k], W.PAPER_MIX, seed=int(seeds[k]), log=True))
        chains.append(ch)
    return dict(Ls=Ls, xyz=xyz, t=t, seeds=seeds, chains=chains, logs=logs)


def _handle(b, launch):
    return F.Handle(b["Ls"], b["xyz"], b["t"], POT, precision="fp32", n_mol=np.array(MS), warps_per_cell=1,
                    launch_mode=launch)


def _check_states(h, b):
    q, X, t = h.state_fixed()
    off = 0
    for k, M in enumerate(MS):
        sl = slice(off, off + 3 * M)
        ch = b["chains"][k]
        assert np.array_equal(q[sl], ch.q), k
        assert np.array_equal(X[sl], ch.X), k
        assert np.array_equal(t[sl], ch.t), k
        off += 3 * M


def test_batched_fp32_log_takes_the_oracles_decisions(batch):
    h = _handle(batch, 1)
    assert h.info["warps_per_cell"] == 1
    assert h.info["max_cells_per_axis"] == 10 and h.info["stencil_cap"] >= 480
    lg = h.sweep_logged(SWEEPS, np.array(TS), W.PAPER_MIX, batch["seeds"])
    off = 0
    for k, M in enumerate(MS):
        n = SWEEPS * 3 * M
        g, o = lg[off:off + n], batch["logs"][k]
        for f in ("site", "move", "status", "accepted"):
            assert np.array_equal(g[f], o[f]), (k, f)
        ev = o["status"] == 0
        err = np.abs(g["dE"][ev] - o["dE"][ev])
        assert np.all(err <= 6.3e-6 * o["scale"][ev]), (k, (err / o["scale"][ev]).max())
        off += n
    _check_states(h, batch)


@pytest.mark.parametrize("launch", [1, 2])
def test_batched_fp32_launches_end_in_the_oracles_states(batch, launch):
    h = _handle(batch, launch)
    h.sweep(SWEEPS, np.array(TS), W.PAPER_MIX, batch["seeds"])
    _check_states(h, batch)
    st = h.stats()
    for k in range(len(MS)):
        assert st[k]["attempts"] == list(batch["chains"][k].counters[:4])
        assert st[k]["accepts"] == list(batch["chains"][k].counters[4:])
