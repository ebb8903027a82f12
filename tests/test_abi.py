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
    # the build compiles every source for sm_103a alone (no PTX, no other
    # architecture); on a GPU, mc_get_info reports the kernels' binary version
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-arch" not in B.NVCC_FLAGS and not any("gencode" in f for f in B.NVCC_FLAGS)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_create_fails_loudly_without_a_gpu(lib):
    from paper_2506_21290_gb300 import workloads as W
    xyz, t = W.lattice_start(8, 5.0, 0)
    with pytest.raises(F.McError) as e:
        F.Handle(5.0, xyz, t, W.PAPER_POT)
    assert e.value.code in (F.MC_ERR_NO_DEVICE, F.MC_ERR_CUDA)
    assert F.mc_last_error()


def test_header_is_plain_c_and_cpp(tmp_path):
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        r = subprocess.run([gcc, "-fsyntax-only", "-Wall", "-Werror", std, "-x", lang, F.HEADER],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_c_program_links_every_entry_point(lib, tmp_path):
    """A C program that takes the address of every declared function links
    against the library (no call runs: this host has no GPU)."""
    import os
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    names = F.header_symbols()
    src = tmp_path / "use.c"
    src.write_text('#include "%s"\n#include <stdio.h>\nint main(void) {\n    void *p[] = {%s};\n'
                   '    printf("%%d\\n", (int)(sizeof p / sizeof p[0]));\n    return p[0] == 0;\n}\n'
                   % (F.HEADER, ", ".join("(void *)%s" % n for n in names)))
    exe = tmp_path / "use"
    libdir = os.path.dirname(B.SO)
    r = subprocess.run([gcc, "-std=c99", str(src), "-o", str(exe), "-L" + libdir, "-lflipmc",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
