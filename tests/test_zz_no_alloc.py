"""mc_energy_noalloc: the energy entry point for callers that cannot allocate
device memory (code inside another framework's memory pool, or limited to
enqueuing work on a stream it was handed).  It must agree with mc_energy on
the same configuration, on two calls in a row (the second call reuses the
library's fixed scratch array left over from the first).

This file is collected last on purpose: if it fails, a run stopped at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _device_state(h):
    import torch
    q, X, t = h.state_fixed()
    dq = torch.from_numpy(q.view(np.int32).reshape(-1).copy()).cuda()
    dt = torch.from_numpy(t.astype(np.int32)).cuda()
    return dq, dt


def test_noalloc_energy_matches_mc_energy_on_two_calls():
    import torch
    from paper_2506_21290_gb300 import build as B
    B.build()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    cases = [(343, 1.5, 3), (1000, 1.1, 4)]       # two different sizes and states, back to back
    for M, T, seed in cases:
        L = W.box_length(M)
        xyz, t = W.lattice_start(M, L, seed)
        h = F.Handle(L, xyz, t, W.PAPER_POT, precision="fp32")
        h.sweep(5, T, W.PAPER_MIX, seed)
        E_ref = h.energy()[0]
        dq, dt = _device_state(h)
        rc = F.mc_energy_noalloc(L, M, dq.data_ptr(), dt.data_ptr(), W.PAPER_POT, out.data_ptr(),
                                 stream.cuda_stream)
        assert rc == F.MC_OK
        torch.cuda.synchronize()
        E = float(out.item())
        assert E == pytest.approx(E_ref, rel=1e-12), (M, E, E_ref)
        h.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    from paper_2506_21290_gb300 import build as B
    B.build()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    M = 21846                      # 65538 atoms: one molecule past the limit
    rc = F.mc_energy_noalloc(W.box_length(M), M, buf.data_ptr(), buf.data_ptr(), W.PAPER_POT, buf.data_ptr(), 0)
    assert rc == F.MC_ERR_INVALID_ARG
    assert "65536 atoms" in F.mc_last_error()


def test_noalloc_invalid_type_gives_nan_and_the_next_call_is_clean():
    """A type outside {0,1,2} poisons the result with NaN through the error
    word; a valid call right after clears that word and agrees with
    mc_energy again."""
    import torch
    from paper_2506_21290_gb300 import build as B
    B.build()
    M = 216
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, 7)
    h = F.Handle(L, xyz, t, W.PAPER_POT, precision="fp32")
    E_ref = h.energy()[0]
    dq, dt = _device_state(h)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    bad = dt.clone()
    bad[5] = 3
    rc = F.mc_energy_noalloc(L, M, dq.data_ptr(), bad.data_ptr(), W.PAPER_POT, out.data_ptr(), stream.cuda_stream)
    assert rc == F.MC_OK
    torch.cuda.synchronize()
    assert np.isnan(float(out.item()))
    rc = F.mc_energy_noalloc(L, M, dq.data_ptr(), dt.data_ptr(), W.PAPER_POT, out.data_ptr(), stream.cuda_stream)
    assert rc == F.MC_OK
    torch.cuda.synchronize()
    assert float(out.item()) == pytest.approx(E_ref, rel=1e-12)
    h.close()
