"""Flip Monte Carlo oracle (test infrastructure only).

A plain, slow FP64 CPU implementation of the chain of arXiv 2506.21290,
Sec. II (model: Eq. 1-2; moves and acceptance: Sec. II.B), used to check the
CUDA library.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the product library never does.

The chain itself lives in ``flipmc_oracle.c`` (built here with
``-ffp-contract=off`` so that each FP64 operation rounds once, as written).
The observables of Sec. III.B (Eq. 5-7) are plain numpy in ``observables.py``,
and their multiple-origin statistics (Sec. III.E-F) in ``correlation.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flipmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

LOG_DTYPE = np.dtype([("site", "<i4"), ("move", "<i4"), ("status", "<i4"), ("accepted", "<i4"),
                      ("dE", "<f8"), ("scale", "<f8")])

MV_ATOM, MV_FLIP, MV_MOLT, MV_MOLR = 0, 1, 2, 3
ST_EVAL, ST_LEFT_CELL, ST_BOND_BREAK, ST_NOT_IN_CELL = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle's C file into ``_build/liborc.so`` (if stale)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_ln.argtypes = [ctypes.c_double]
            L.orc_ln.restype = ctypes.c_double
            L.orc_quantize.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_quantize.restype = ctypes.c_uint32
            L.orc_quantize_all.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
            L.orc_energy.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
            L.orc_energy.restype = ctypes.c_double
            L.orc_site_energy.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int]
            L.orc_site_energy.restype = ctypes.c_double
            L.orc_phi.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            L.orc_phi.restype = ctypes.c_double
            L.orc_mag.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            L.orc_mag.restype = ctypes.c_double
            L.orc_phi_many.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p]
            L.orc_sweep_shift.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
            L.orc_run.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                  ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_run.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def philox4x32_10(ctr, key) -> tuple:
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(o)


def ln(x: float) -> float:
    """The oracle's own atanh-series logarithm (not libm's)."""
    return lib().orc_ln(float(x))


def quantize(xyz: np.ndarray, L: float) -> np.ndarray:
    """Positions (any real) -> 32-bit fixed point q = floor(frac(x/L) 2^32)."""
    x = np.ascontiguousarray(xyz, dtype=np.float64)
    q = np.empty(x.shape, dtype=np.uint32)
    lib().orc_quantize_all(int(x.size), _ptr(x), float(L), _ptr(q))
    return q


def pot_array(pot) -> np.ndarray:
    """{sigma_A, sigma_B, sigma_C, eps, fene_K, fene_R0} as float64[6]."""
    return np.ascontiguousarray(np.asarray(pot, dtype=np.float64).reshape(6))


def mix_array(mix) -> np.ndarray:
    """{p_atom, p_flip, p_mol_trans, p_mol_rot, d_atom, d_mol, rot_a} as float64[7]."""
    return np.ascontiguousarray(np.asarray(mix, dtype=np.float64).reshape(7))


def energy(L: float, q: np.ndarray, t: np.ndarray, pot) -> float:
    """Brute-force total energy, all pairs i<j in ascending order (Eq. 1 + Eq. 2)."""
    q = np.ascontiguousarray(q, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.int32)
    return lib().orc_energy(float(L), int(t.size // 3), _ptr(q), _ptr(t), _ptr(pot_array(pot)))


def site_energy(L: float, q: np.ndarray, t: np.ndarray, pot, i: int) -> float:
    q = np.ascontiguousarray(q, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.int32)
    return lib().orc_site_energy(float(L), int(t.size // 3), _ptr(q), _ptr(t), _ptr(pot_array(pot)), int(i))


def phi(r2: float, a: int, b: int, bonded: bool, pot) -> float:
    """Pair energy of types (a, b) at squared distance r2: WCA (Eq. 1) plus, for
    a bond, FENE (Eq. 2)."""
    return lib().orc_phi(float(r2), int(a), int(b), int(bool(bonded)), _ptr(pot_array(pot)))


def mag(r2: float, a: int, b: int, bonded: bool, pot) -> float:
    """Conditioning scale of one pair evaluation of types (a, b) at squared
    distance r2: the summed magnitudes 4eps s^12 + 4eps s^6 + eps of the WCA
    pieces inside the cutoff plus, for a bond, K eps (|ln(1-x)| + x/(1-x)),
    x = r2 / (R0 sigma_ab)^2.  The FP32 tolerances are measured against it."""
    return lib().orc_mag(float(r2), int(a), int(b), int(bool(bonded)), _ptr(pot_array(pot)))


def phi_many(r2: np.ndarray, a: int, b: int, bonded: bool, pot) -> np.ndarray:
    """Vectorised phi over an array of squared distances."""
    x = np.ascontiguousarray(r2, dtype=np.float64)
    out = np.empty_like(x)
    lib().orc_phi_many(int(x.size), _ptr(x), int(a), int(b), int(bool(bonded)), _ptr(pot_array(pot)), _ptr(out))
    return out


def sweep_shift(sweep: int, seed: int) -> np.ndarray:
    s = np.zeros(3, dtype=np.uint32)
    lib().orc_sweep_shift(int(sweep), int(seed), _ptr(s))
    return s


class Chain:
    """State of one replica as the oracle sees it.

    q: (N,3) uint32 fixed-point positions; X: (N,3) int64 unwrapped fixed point;
    t: (N,) int32 types; e_run: running FP64 energy; counters: attempts[4] +
    accepts[4]; sweep: next sweep number.
    """

    def __init__(self, L, xyz=None, types=None, pot=None, q=None, nc=None):
        self.L = float(L)
        if q is None:
            q = quantize(np.asarray(xyz, dtype=np.float64).reshape(-1, 3), self.L)
        self.q = np.ascontiguousarray(np.asarray(q, dtype=np.uint32).reshape(-1, 3))
        self.X = self.q.astype(np.int64)
        self.t = np.ascontiguousarray(np.asarray(types, dtype=np.int32).reshape(-1))
        self.pot = pot_array(pot)
        self.M = self.t.size // 3
        self.nc = nc
        self.e_run = energy(self.L, self.q, self.t, self.pot)
        self.counters = np.zeros(8, dtype=np.uint64)
        self.sweep = 0

    def run(self, n_sweeps, T, mix, seed, nc=None, log=False):
        nc = self.nc if nc is None else nc
        e = ctypes.c_double(self.e_run)
        lg = np.zeros(n_sweeps * 3 * self.M, dtype=LOG_DTYPE) if log else None
        rc = lib().orc_run(self.L, self.M, _ptr(self.q), _ptr(self.X), _ptr(self.t), _ptr(self.pot),
                           int(nc), int(seed), int(self.sweep), int(n_sweeps), float(T),
                           _ptr(mix_array(mix)), ctypes.addressof(e), _ptr(self.counters),
                           _ptr(lg) if log else None)
        if rc != 0:
            raise RuntimeError("orc_run failed: %d" % rc)
        self.e_run = e.value
        self.sweep += n_sweeps
        return lg

    def energy(self) -> float:
        return energy(self.L, self.q, self.t, self.pot)

    def positions(self) -> np.ndarray:
        return self.q.astype(np.float64) * (self.L / 4294967296.0)
