"""Build the CUDA library in-tree: nvcc for sm_103a, one object per .cu file
(compiled in parallel), linked into ``paper_2506_21290_gb300/_lib/libflipmc.so``."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
SO = os.path.join(OUT_DIR, "libflipmc.so")
SOURCES = ["cell_list.cu", "sweep.cu", "energy.cu", "engine.cu", "noalloc.cu", "md.cu"]
HEADERS = ["flipmc_device.cuh", "flipmc_types.h", "cell_list.h", "cell_list_dev.cuh", "energy.h", "md.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    inc = os.path.join(os.path.dirname(HERE), "include", "flipmc.h")
    return [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [inc, os.path.abspath(__file__)]


def stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    if not force and not stale():
        return SO
    os.makedirs(OUT_DIR, exist_ok=True)
    nv = nvcc()
    flags = ARCH + NVCC_FLAGS + (extra or [])

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nv, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err)
    tmp = SO + ".tmp%d" % os.getpid()
    cmd = [nv, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra=sys.argv[1:]))
