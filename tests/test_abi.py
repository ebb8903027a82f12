"""The C ABI library builds for sm_103a, loads, and exports every function
include/flipmc.h declares.  No compute call runs here (no GPU on this host)."""
import ctypes
import subprocess

import pytest
import torch

from paper_2506_21290_gb300 import build as B
from paper_2506_21290_gb300 import flipmc as F


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.load()


def test_header_declares_the_boundary():
    names = F.header_symbols()
    for n in ("mc_create", "mc_create_batch", "mc_sweep", "mc_sweep_batch", "mc_sweep_logged", "mc_energy",
              "mc_state", "mc_state_fixed", "mc_set_state", "mc_set_t0", "mc_observables", "mc_destroy",
              "mc_last_error", "mc_sync", "mc_set_sweep"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in F.header_symbols():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", B.SO], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in F.header_symbols() if n not in exported]
    assert not missing, missing


def test_library_is_built_for_sm_103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", B.SO], capture_output=True, text=True).stdout
    assert "sm_103a" in out


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_create_fails_loudly_without_a_gpu(lib):
    from paper_2506_21290_gb300 import workloads as W
    xyz, t = W.lattice_start(8, 5.0, 0)
    with pytest.raises(F.McError) as e:
        F.Handle(5.0, xyz, t, W.PAPER_POT)
    assert e.value.code in (F.MC_ERR_NO_DEVICE, F.MC_ERR_CUDA)
    assert F.mc_last_error()
