"""Failure detection without a GPU fault.

Every wait between blocks of the persistent sweep is bounded.  A handle
created with a tiny wait limit (mc_options.wait_limit_log2) makes those waits
run out: the kernel must return on its own, mc_sync must report
MC_ERR_TIMEOUT, and the device must stay usable (a fresh handle runs the
chain exactly).  An injected allocation failure (mc_test_fail_alloc) must make
handle creation fail cleanly, free what it had allocated, and leave the next
creation working.  Nothing here traps, faults or hangs a GPU.
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


def _start(M, seed):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    return L, xyz, t


def test_bounded_waits_give_up_and_report_timeout():
    L, xyz, t = _start(1000, 1)
    h = F.Handle(L, xyz, t, POT, precision="fp32", launch_mode=2, wait_limit_log2=1)
    # hundreds of grid barriers and neighbour waits, each allowed two polls
    h.sweep(20, 1.0, W.PAPER_MIX, 1)
    with pytest.raises(F.McError) as e:
        h.sync()
    assert e.value.code == F.MC_ERR_TIMEOUT
    h.close()
    # the device is still usable: a fresh handle runs the chain exactly
    L, xyz, t = _start(125, 2)
    g = F.Handle(L, xyz, t, POT, precision="fp64", launch_mode=2)
    ch = oracle.Chain(L, xyz, t, POT, nc=g.info["max_cells_per_axis"])
    g.sweep(5, 2.0, W.PAPER_MIX, 3)
    g.sync()
    ch.run(5, 2.0, W.PAPER_MIX, seed=3)
    assert np.array_equal(g.state_fixed()[0], ch.q)


def test_wait_limit_is_validated():
    L, xyz, t = _start(64, 0)
    with pytest.raises(F.McError) as e:
        F.Handle(L, xyz, t, POT, wait_limit_log2=31)
    assert e.value.code == F.MC_ERR_INVALID_ARG


@pytest.mark.parametrize("after", [0, 3, 17])
def test_injected_allocation_failure_fails_cleanly(after):
    import torch
    L, xyz, t = _start(343, 4)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    F.mc_test_fail_alloc(after)
    with pytest.raises(F.McError) as e:
        F.Handle(L, xyz, t, POT, precision="fp32")
    assert e.value.code == F.MC_ERR_CUDA
    assert "injected" in str(e.value)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (8 << 20), (free0, free1)        # what it had allocated was freed
    # the hook fired once and disarmed itself
    h = F.Handle(L, xyz, t, POT, precision="fp32")
    h.sweep(2, 1.0, W.PAPER_MIX, 4)
    h.sync()
    h.close()
    F.mc_test_fail_alloc(-1)
