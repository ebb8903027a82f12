"""The periodic FP64 drift check (mc_options.recompute_every): every k-th
sweep ends with an FP64 recompute of the total energy, the relative drift of
the running total is recorded and the running total restarts from the
recompute.  The chain itself does not change."""
import numpy as np
import pytest

from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.PAPER_POT


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21290_gb300 import build as B
    B.build()


@pytest.mark.parametrize("launch", [1, 2])
def test_recompute_every_k_sweeps_leaves_the_chain_and_bounds_the_drift(launch):
    M, T, seed, k = 1000, 0.75, 3, 7
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    a = F.Handle(L, xyz, t, POT, precision="fp32", launch_mode=launch, recompute_every=k)
    b = F.Handle(L, xyz, t, POT, precision="fp32", launch_mode=launch)
    assert a.info["recompute_every"] == k and b.info["recompute_every"] == 0
    # 30 sweeps in uneven calls: recomputes after sweeps 7, 14, 21, 28
    for n in (5, 11, 3, 9, 2):
        a.sweep(n, T, W.PAPER_MIX, seed)
        b.sweep(n, T, W.PAPER_MIX, seed)
    qa, Xa, ta = a.state_fixed()
    qb, Xb, tb = b.state_fixed()
    assert np.array_equal(qa, qb) and np.array_equal(Xa, Xb) and np.array_equal(ta, tb)
    sa, sb = a.stats()[0], b.stats()[0]
    assert sa["recomputes"] == 4 and sb["recomputes"] == 0
    assert 0.0 < sa["drift_max"] < 1e-6 and sa["drift_last"] <= sa["drift_max"]
    assert sb["drift_max"] == 0.0
    # two sweeps past the last recompute: e_run = that recompute + two sweeps
    # of FP32 Delta E; a recompute now agrees to FP32 rounding
    E = a.energy()[0]
    assert abs(sa["e_run"] - E) <= 1e-7 * abs(E)
    # at a boundary the running total is the recompute itself
    a.sweep(5, T, W.PAPER_MIX, seed)      # sweeps 31..35: a recompute after 35
    assert a.stats()[0]["e_run"] == a.energy()[0]
    a.reset_stats()
    s = a.stats()[0]
    assert s["recomputes"] == 0 and s["drift_max"] == 0.0 and s["drift_last"] == 0.0


def test_recompute_every_rejects_negative():
    L = W.box_length(64)
    xyz, t = W.lattice_start(64, L, 0)
    with pytest.raises(F.McError) as e:
        F.Handle(L, xyz, t, POT, recompute_every=-1)
    assert e.value.code == F.MC_ERR_INVALID_ARG
