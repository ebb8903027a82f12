"""ctypes binding of the flip Monte Carlo C ABI (include/flipmc.h).

Argument marshalling only: every step of the method runs in the CUDA library
``_lib/libflipmc.so``.  Importing works without the library; the first call
that needs it raises if it has not been built (``python -m
paper_2506_21290_gb300.build`` or ``__graft_entry__.build()``), and creating a
handle raises when no CUDA device is present: there is no CPU fallback.

The module-level functions carry the C names (mc_create, mc_sweep, ...);
``Handle`` wraps them for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_lib", "libflipmc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "flipmc.h")

MC_OK = 0
MC_ERR_INVALID_ARG = -1
MC_ERR_BAD_STATE = -2
MC_ERR_CUDA = -3
MC_ERR_TIMEOUT = -4
MC_ERR_CELL_OVERFLOW = -5
MC_ERR_NO_DEVICE = -6
MC_PREC_FP64 = 0
MC_PREC_FP32 = 1
PREC = {"fp64": MC_PREC_FP64, "fp32": MC_PREC_FP32}


class McError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__("%s failed (%d): %s" % (fn, code, msg))
        self.code = code


class mc_params(C.Structure):
    _fields_ = [("sigma", C.c_double * 3), ("eps", C.c_double), ("fene_k", C.c_double), ("fene_r0", C.c_double)]


class mc_move_mix(C.Structure):
    _fields_ = [("p", C.c_double * 4), ("d_atom", C.c_double), ("d_mol", C.c_double), ("rot_a", C.c_double)]


class mc_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("n_cells", C.c_int), ("device", C.c_int), ("stencil_cap", C.c_int),
                ("recheck_gap", C.c_double), ("warps_per_cell", C.c_int), ("launch_mode", C.c_int),
                ("recompute_every", C.c_int), ("wait_limit_log2", C.c_int)]


class mc_stats(C.Structure):
    _fields_ = [("attempts", C.c_uint64 * 4), ("accepts", C.c_uint64 * 4), ("rejected_geometry", C.c_uint64),
                ("rejected_bond", C.c_uint64), ("pair_evals", C.c_uint64), ("fp64_rechecks", C.c_uint64),
                ("pair_interactions", C.c_uint64), ("sweeps", C.c_uint64), ("e_run", C.c_double),
                ("recomputes", C.c_uint64), ("drift_last", C.c_double), ("drift_max", C.c_double)]


class mc_info(C.Structure):
    _fields_ = [("n_rep", C.c_int), ("precision", C.c_int), ("stencil_cap", C.c_int), ("total_sites", C.c_int),
                ("total_cells", C.c_int), ("max_cells_per_axis", C.c_int), ("recheck_gap", C.c_double),
                ("warps_per_cell", C.c_int), ("active_cells_per_colour", C.c_int), ("launch_mode", C.c_int),
                ("persistent_blocks", C.c_int), ("recompute_every", C.c_int), ("binary_version", C.c_int)]


LOG_DTYPE = np.dtype([("site", "<i4"), ("move", "<i2"), ("flags", "<i2"), ("status", "<i4"), ("accepted", "<i4"),
                      ("dE", "<f8"), ("dE64", "<f8"), ("scale", "<f8")])

_lib = None


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def load():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO):
        raise RuntimeError("flipmc CUDA library not built (%s missing); run __graft_entry__.build()" % SO)
    L = C.CDLL(SO)
    vp, i32, u64, dbl = C.c_void_p, C.c_int, C.c_uint64, C.c_double
    sig = {
        "mc_create": ([vp, dbl, i32, vp, vp, vp, vp], i32),
        "mc_create_batch": ([vp, i32, vp, vp, vp, vp, vp, vp], i32),
        "mc_destroy": ([vp], None),
        "mc_set_stream": ([vp, vp], i32),
        "mc_sweep": ([vp, i32, dbl, vp, u64], i32),
        "mc_sweep_batch": ([vp, i32, vp, vp, vp], i32),
        "mc_sweep_logged": ([vp, i32, vp, vp, vp, vp], i32),
        "mc_sync": ([vp], i32),
        "mc_energy_device": ([vp, vp], i32),
        "mc_sweep_timed": ([vp, i32, vp, vp, vp, vp], i32),
        "mc_autotune": ([vp, i32, vp, vp, vp, vp], i32),
        "mc_energy": ([vp, vp], i32),
        "mc_state": ([vp, vp, vp, vp], i32),
        "mc_state_fixed": ([vp, vp, vp, vp], i32),
        "mc_set_state": ([vp, vp, vp], i32),
        "mc_set_state_fixed": ([vp, vp, vp, vp], i32),
        "mc_set_sweep": ([vp, u64], i32),
        "mc_reset_stats": ([vp], i32),
        "mc_set_t0": ([vp], i32),
        "mc_observables": ([vp, vp, i32, vp, i32, vp, vp, vp, vp], i32),
        "mc_get_info": ([vp, vp], i32),
        "mc_pressure": ([vp, vp, vp], i32),
        "mc_cell_grid": ([dbl, i32, vp, vp, i32, vp, vp], i32),
        "mc_structure_factor": ([vp, vp, i32, vp], i32),
        "mc_pair_histogram": ([vp, dbl, i32, vp, vp], i32),
        "mc_corr_setup": ([vp, i32, vp, i32, i32, vp, i32, vp, i32], i32),
        "mc_corr_schedule": ([i32, vp, i32, i32, C.c_int64, vp], i32),
        "mc_corr_run": ([vp, i32, vp, vp, vp], i32),
        "mc_corr_sums": ([vp, vp], i32),
        "mc_corr_results": ([vp, vp], i32),
        "mc_corr_relaxation_time": ([vp, i32, dbl, vp], i32),
        "mc_corr_derive": ([i32, vp, vp, vp], i32),
        "mc_relaxation_time": ([i32, vp, vp, vp, dbl, vp], i32),
        "mc_md_setup": ([vp, dbl, dbl, vp, vp, i32], i32),
        "mc_md_run": ([vp, i32], i32),
        "mc_md_state": ([vp, vp, vp], i32),
        "mc_last_error": ([], C.c_char_p),
        "mc_energy_noalloc": ([dbl, i32, vp, vp, vp, vp, vp], i32),
        "mc_test_fail_alloc": ([i32], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def header_symbols():
    """Function names declared in include/flipmc.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(mc_\w+)\s*\(", txt, flags=re.M)))


def _check(rc, fn):
    if rc != MC_OK:
        raise McError(rc, fn, load().mc_last_error().decode())


def make_params(pot):
    p = mc_params()
    p.sigma[:] = [float(x) for x in pot[:3]]
    p.eps, p.fene_k, p.fene_r0 = float(pot[3]), float(pot[4]), float(pot[5])
    return p


def make_mix(mix):
    m = mc_move_mix()
    m.p[:] = [float(x) for x in mix[:4]]
    m.d_atom, m.d_mol, m.rot_a = float(mix[4]), float(mix[5]), float(mix[6])
    return m


def make_options(precision="fp32", n_cells=0, device=0, stencil_cap=0, recheck_gap=0.0, warps_per_cell=0,
                 launch_mode=0, recompute_every=0, wait_limit_log2=0):
    o = mc_options()
    o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    o.n_cells, o.device, o.stencil_cap, o.recheck_gap = int(n_cells), int(device), int(stencil_cap), float(recheck_gap)
    o.warps_per_cell = int(warps_per_cell)
    o.launch_mode = int(launch_mode)
    o.recompute_every = int(recompute_every)
    o.wait_limit_log2 = int(wait_limit_log2)
    return o


# ---- the C names ----------------------------------------------------------

def mc_create(L, xyz, types, pot, opts):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    types = np.ascontiguousarray(types, dtype=np.int32).reshape(-1)
    h = C.c_void_p()
    p = make_params(pot)
    _check(load().mc_create(C.byref(h), float(L), types.size // 3, _ptr(xyz), _ptr(types), C.byref(p), C.byref(opts)),
           "mc_create")
    return h


def mc_create_batch(Ls, n_mol, xyz, types, pot, opts):
    Ls = np.ascontiguousarray(Ls, dtype=np.float64)
    n_mol = np.ascontiguousarray(n_mol, dtype=np.int32)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    types = np.ascontiguousarray(types, dtype=np.int32).reshape(-1)
    h = C.c_void_p()
    p = make_params(pot)
    _check(load().mc_create_batch(C.byref(h), Ls.size, _ptr(Ls), _ptr(n_mol), _ptr(xyz), _ptr(types), C.byref(p),
                                  C.byref(opts)), "mc_create_batch")
    return h


def mc_destroy(h):
    load().mc_destroy(h)


def mc_set_stream(h, stream_ptr):
    _check(load().mc_set_stream(h, C.c_void_p(stream_ptr)), "mc_set_stream")


def mc_sweep(h, n, T, mix, seed):
    m = make_mix(mix)
    _check(load().mc_sweep(h, int(n), float(T), C.byref(m), int(seed)), "mc_sweep")


def mc_sweep_batch(h, n, Ts, mix, seeds):
    Ts = np.ascontiguousarray(Ts, dtype=np.float64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    m = make_mix(mix)
    _check(load().mc_sweep_batch(h, int(n), _ptr(Ts), C.byref(m), _ptr(seeds)), "mc_sweep_batch")


def mc_sweep_logged(h, n, Ts, mix, seeds, total_sites):
    Ts = np.ascontiguousarray(np.atleast_1d(Ts), dtype=np.float64)
    seeds = np.ascontiguousarray(np.atleast_1d(seeds), dtype=np.uint64)
    log = np.zeros(int(n) * int(total_sites), dtype=LOG_DTYPE)
    m = make_mix(mix)
    _check(load().mc_sweep_logged(h, int(n), _ptr(Ts), C.byref(m), _ptr(seeds), _ptr(log)), "mc_sweep_logged")
    return log


def mc_energy_device(h, dev_ptr):
    _check(load().mc_energy_device(h, C.c_void_p(dev_ptr)), "mc_energy_device")


def mc_sweep_timed(h, n, Ts, mix, seeds):
    Ts = np.ascontiguousarray(np.atleast_1d(Ts), dtype=np.float64)
    seeds = np.ascontiguousarray(np.atleast_1d(seeds), dtype=np.uint64)
    ms = np.zeros(3, dtype=np.float64)
    m = make_mix(mix)
    _check(load().mc_sweep_timed(h, int(n), _ptr(Ts), C.byref(m), _ptr(seeds), _ptr(ms)), "mc_sweep_timed")
    return ms


def mc_autotune(h, n, Ts, mix, seeds):
    Ts = np.ascontiguousarray(np.atleast_1d(Ts), dtype=np.float64)
    seeds = np.ascontiguousarray(np.atleast_1d(seeds), dtype=np.uint64)
    res = np.zeros(8, dtype=np.float64)
    m = make_mix(mix)
    _check(load().mc_autotune(h, int(n), _ptr(Ts), C.byref(m), _ptr(seeds), _ptr(res)), "mc_autotune")
    return res


def mc_sync(h):
    _check(load().mc_sync(h), "mc_sync")


def mc_energy(h, n_rep):
    e = np.zeros(n_rep, dtype=np.float64)
    _check(load().mc_energy(h, _ptr(e)), "mc_energy")
    return e


def mc_state(h, total_sites, n_rep):
    xyz = np.zeros((total_sites, 3), dtype=np.float64)
    t = np.zeros(total_sites, dtype=np.int32)
    st = (mc_stats * n_rep)()
    _check(load().mc_state(h, _ptr(xyz), _ptr(t), st), "mc_state")
    return xyz, t, [stats_dict(s) for s in st]


def mc_state_fixed(h, total_sites):
    q = np.zeros((total_sites, 3), dtype=np.uint32)
    X = np.zeros((total_sites, 3), dtype=np.int64)
    t = np.zeros(total_sites, dtype=np.int32)
    _check(load().mc_state_fixed(h, _ptr(q), _ptr(X), _ptr(t)), "mc_state_fixed")
    return q, X, t


def mc_set_state(h, xyz, types):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    types = np.ascontiguousarray(types, dtype=np.int32).reshape(-1)
    _check(load().mc_set_state(h, _ptr(xyz), _ptr(types)), "mc_set_state")


def mc_set_state_fixed(h, q, X, types):
    q = np.ascontiguousarray(q, dtype=np.uint32).reshape(-1, 3)
    X = None if X is None else np.ascontiguousarray(X, dtype=np.int64).reshape(-1, 3)
    types = np.ascontiguousarray(types, dtype=np.int32).reshape(-1)
    _check(load().mc_set_state_fixed(h, _ptr(q), _ptr(X), _ptr(types)), "mc_set_state_fixed")


def mc_set_sweep(h, sweep):
    _check(load().mc_set_sweep(h, int(sweep)), "mc_set_sweep")


def mc_reset_stats(h):
    _check(load().mc_reset_stats(h), "mc_reset_stats")


def mc_set_t0(h):
    _check(load().mc_set_t0(h), "mc_set_t0")


def mc_observables(h, qa, qc, n_rep, total_sites, per_particle=False):
    qa = np.ascontiguousarray(qa, dtype=np.float64).reshape(-1, 3)
    qc = np.ascontiguousarray(qc, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((n_rep, 3), dtype=np.float64)
    fs = fscm = c2 = None
    if per_particle:
        fs = np.zeros(total_sites)
        fscm = np.zeros(total_sites // 3)
        c2 = np.zeros(total_sites // 3)
    _check(load().mc_observables(h, _ptr(qa), len(qa), _ptr(qc), len(qc), _ptr(out), _ptr(fs), _ptr(fscm), _ptr(c2)),
           "mc_observables")
    return out, fs, fscm, c2


def mc_cell_grid(L, types, pot, request=0):
    """(n_c, interaction range) that mc_create picks for one replica (host only)."""
    types = np.ascontiguousarray(types, dtype=np.int32).reshape(-1)
    p = make_params(pot)
    nc = C.c_int(0)
    rng = C.c_double(0.0)
    _check(load().mc_cell_grid(float(L), types.size // 3, _ptr(types), C.byref(p), int(request), C.byref(nc),
                               C.byref(rng)), "mc_cell_grid")
    return nc.value, rng.value


def mc_pressure(h, T):
    T = np.ascontiguousarray(T, dtype=np.float64)
    out = np.zeros((T.size, 2), dtype=np.float64)
    _check(load().mc_pressure(h, _ptr(T), _ptr(out)), "mc_pressure")
    return out


def mc_structure_factor(h, qvec, n_rep):
    qvec = np.ascontiguousarray(qvec, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((n_rep, len(qvec)), dtype=np.float64)
    _check(load().mc_structure_factor(h, _ptr(qvec), len(qvec), _ptr(out)), "mc_structure_factor")
    return out


def mc_pair_histogram(h, dr, n_bins, n_rep):
    counts = np.zeros((n_rep, n_bins), dtype=np.uint64)
    g = np.zeros((n_rep, n_bins), dtype=np.float64)
    _check(load().mc_pair_histogram(h, float(dr), int(n_bins), _ptr(counts), _ptr(g)), "mc_pair_histogram")
    return counts, g


MC_CORR_NSUM = 16
MC_CORR_NRES = 11
CORR_RESULT_FIELDS = ("n", "F_s", "F_s_cm", "C_2", "chi4_F_s", "chi4_F_s_cm", "chi4_C_2", "chi4self_F_s",
                      "chi4self_F_s_cm", "chi4self_C_2", "rho")


def mc_corr_setup(h, lags, origin_every, max_origins, qa, qc):
    lags = np.ascontiguousarray(lags, dtype=np.int64).reshape(-1)
    qa = np.ascontiguousarray(qa, dtype=np.float64).reshape(-1, 3)
    qc = np.ascontiguousarray(qc, dtype=np.float64).reshape(-1, 3)
    _check(load().mc_corr_setup(h, len(lags), _ptr(lags), int(origin_every), int(max_origins), _ptr(qa), len(qa),
                                _ptr(qc), len(qc)), "mc_corr_setup")


def mc_corr_schedule(lags, origin_every, max_origins, n_sweeps):
    """Samples per lag after n_sweeps sweeps of mc_corr_run (host only)."""
    lags = np.ascontiguousarray(lags, dtype=np.int64).reshape(-1)
    counts = np.zeros(len(lags), dtype=np.int64)
    _check(load().mc_corr_schedule(len(lags), _ptr(lags), int(origin_every), int(max_origins), int(n_sweeps),
                                   _ptr(counts)), "mc_corr_schedule")
    return counts


def mc_corr_run(h, n, T, mix, seeds):
    T = np.ascontiguousarray(T, dtype=np.float64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    m = make_mix(mix)
    _check(load().mc_corr_run(h, int(n), _ptr(T), C.byref(m), _ptr(seeds)), "mc_corr_run")


def mc_corr_sums(h, n_rep, n_lags):
    out = np.zeros((n_rep, n_lags, MC_CORR_NSUM), dtype=np.float64)
    _check(load().mc_corr_sums(h, _ptr(out)), "mc_corr_sums")
    return out


def mc_corr_results(h, n_rep, n_lags):
    out = np.zeros((n_rep, n_lags, MC_CORR_NRES), dtype=np.float64)
    _check(load().mc_corr_results(h, _ptr(out)), "mc_corr_results")
    return out


def mc_corr_derive(sums, n_atoms):
    """Host-only derivation of the statistics from rows of sums (..., 16) with n_atoms per row."""
    sums = np.ascontiguousarray(sums, dtype=np.float64)
    rows = sums.reshape(-1, MC_CORR_NSUM)
    n_atoms = np.ascontiguousarray(np.broadcast_to(np.asarray(n_atoms, dtype=np.int32), (len(rows),)))
    out = np.zeros((len(rows), MC_CORR_NRES), dtype=np.float64)
    _check(load().mc_corr_derive(len(rows), _ptr(rows), _ptr(n_atoms), _ptr(out)), "mc_corr_derive")
    return out.reshape(sums.shape[:-1] + (MC_CORR_NRES,))


def mc_relaxation_time(lags, values, counts, level):
    lags = np.ascontiguousarray(lags, dtype=np.int64)
    values = np.ascontiguousarray(values, dtype=np.float64)
    counts = np.ascontiguousarray(counts, dtype=np.float64)
    tau = np.zeros(1, dtype=np.float64)
    _check(load().mc_relaxation_time(len(lags), _ptr(lags), _ptr(values), _ptr(counts), float(level), _ptr(tau)),
           "mc_relaxation_time")
    return float(tau[0])


def mc_corr_relaxation_time(h, which, level, n_rep):
    tau = np.zeros(n_rep, dtype=np.float64)
    _check(load().mc_corr_relaxation_time(h, int(which), float(level), _ptr(tau)), "mc_corr_relaxation_time")
    return tau


def mc_md_setup(h, dt, tau_T, T, v0, force_precision="fp64"):
    T = np.ascontiguousarray(T, dtype=np.float64)
    v0 = np.ascontiguousarray(v0, dtype=np.float64).reshape(-1)
    fp = MC_PREC_FP32 if force_precision == "fp32" else MC_PREC_FP64
    _check(load().mc_md_setup(h, float(dt), float(tau_T), _ptr(T), _ptr(v0), fp), "mc_md_setup")


def mc_md_run(h, n):
    _check(load().mc_md_run(h, int(n)), "mc_md_run")


def mc_md_state(h, n_sites, n_rep):
    v = np.zeros((n_sites, 3), dtype=np.float64)
    out = np.zeros((n_rep, 5), dtype=np.float64)
    _check(load().mc_md_state(h, _ptr(v), _ptr(out)), "mc_md_state")
    return v, out


def mc_get_info(h):
    i = mc_info()
    _check(load().mc_get_info(h, C.byref(i)), "mc_get_info")
    return {k: getattr(i, k) for k, _ in mc_info._fields_}


def mc_last_error():
    return load().mc_last_error().decode()


def mc_energy_noalloc(L, n_mol, dev_q_ptr, dev_types_ptr, pot, dev_out_ptr, stream_ptr=0):
    """Energy of a configuration in caller device memory, with no device
    allocation by the library (for callers that cannot allocate); raw device
    pointers in, one double written at dev_out_ptr.  Returns the C code."""
    p = make_params(pot)
    return load().mc_energy_noalloc(float(L), int(n_mol), C.c_void_p(dev_q_ptr), C.c_void_p(dev_types_ptr),
                                    C.byref(p), C.c_void_p(dev_out_ptr), C.c_void_p(stream_ptr))


def mc_test_fail_alloc(after):
    """Make the device allocation number `after` of the next handle creation
    fail (test hook of the library's failure paths; < 0 disarms)."""
    load().mc_test_fail_alloc(int(after))


def stats_dict(s):
    return {"attempts": list(s.attempts), "accepts": list(s.accepts), "rejected_geometry": s.rejected_geometry,
            "rejected_bond": s.rejected_bond, "pair_evals": s.pair_evals, "fp64_rechecks": s.fp64_rechecks,
            "pair_interactions": s.pair_interactions, "sweeps": s.sweeps, "e_run": s.e_run,
            "recomputes": s.recomputes, "drift_last": s.drift_last, "drift_max": s.drift_max}


class Handle:
    """One handle of the library (a batch of replicas; one replica by default)."""

    def __init__(self, L, xyz, types, pot, precision="fp32", n_cells=0, device=0, stencil_cap=0, recheck_gap=0.0,
                 n_mol=None, warps_per_cell=0, launch_mode=0, recompute_every=0, wait_limit_log2=0):
        opts = make_options(precision, n_cells, device, stencil_cap, recheck_gap, warps_per_cell, launch_mode,
                            recompute_every, wait_limit_log2)
        if np.ndim(L) == 0:
            self.h = mc_create(L, xyz, types, pot, opts)
        else:
            self.h = mc_create_batch(L, n_mol, xyz, types, pot, opts)
        self.info = mc_get_info(self.h)
        self.n_rep = self.info["n_rep"]
        self.N = self.info["total_sites"]

    def close(self):
        if self.h is not None:
            mc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n, T, mix, seed):
        if np.ndim(T) == 0 and np.ndim(seed) == 0:
            mc_sweep(self.h, n, T, mix, seed)
        else:
            Ts = np.broadcast_to(np.asarray(T, dtype=np.float64), (self.n_rep,))
            seeds = np.broadcast_to(np.asarray(seed, dtype=np.uint64), (self.n_rep,))
            mc_sweep_batch(self.h, n, Ts, mix, seeds)

    def sweep_logged(self, n, T, mix, seed):
        Ts = np.broadcast_to(np.asarray(T, dtype=np.float64), (self.n_rep,))
        seeds = np.broadcast_to(np.asarray(seed, dtype=np.uint64), (self.n_rep,))
        return mc_sweep_logged(self.h, n, Ts, mix, seeds, self.N)

    def sync(self):
        mc_sync(self.h)

    def sweep_timed(self, n, T, mix, seed):
        Ts = np.broadcast_to(np.asarray(T, dtype=np.float64), (self.n_rep,))
        seeds = np.broadcast_to(np.asarray(seed, dtype=np.uint64), (self.n_rep,))
        return mc_sweep_timed(self.h, n, Ts, mix, seeds)

    def autotune(self, n, T, mix, seed):
        """Time every cell schedule on a copy of the state and keep the fastest;
        returns ms per sweep [W=1, 2, 4, 8 persistent, W=1, 2, 4, 8 graphs] (-1: unavailable)."""
        Ts = np.broadcast_to(np.asarray(T, dtype=np.float64), (self.n_rep,))
        seeds = np.broadcast_to(np.asarray(seed, dtype=np.uint64), (self.n_rep,))
        res = mc_autotune(self.h, n, Ts, mix, seeds)
        self.info = mc_get_info(self.h)
        return res

    def energy_device(self, dev_ptr):
        mc_energy_device(self.h, dev_ptr)

    def energy(self):
        return mc_energy(self.h, self.n_rep)

    def state(self):
        return mc_state(self.h, self.N, self.n_rep)

    def state_fixed(self):
        return mc_state_fixed(self.h, self.N)

    def set_state(self, xyz, types):
        mc_set_state(self.h, xyz, types)

    def set_state_fixed(self, q, X, types):
        mc_set_state_fixed(self.h, q, X, types)

    def set_sweep(self, s):
        mc_set_sweep(self.h, s)

    def set_t0(self):
        mc_set_t0(self.h)

    def observables(self, qa, qc, per_particle=False):
        return mc_observables(self.h, qa, qc, self.n_rep, self.N, per_particle)

    def pressure(self, T):
        """(n_rep, 2): the pair virial sum W and the pressure N T / V + W / (3 V)."""
        return mc_pressure(self.h, np.broadcast_to(np.asarray(T, dtype=np.float64), (self.n_rep,)))

    def structure_factor(self, qvec):
        """(n_rep, n_q): |sum_i exp(i q . x_i)|^2 / N."""
        return mc_structure_factor(self.h, qvec, self.n_rep)

    def pair_histogram(self, dr, n_bins):
        """(counts, g): pair-distance counts per bin (pairs i < j) and g(r), each (n_rep, n_bins)."""
        return mc_pair_histogram(self.h, dr, n_bins, self.n_rep)

    def corr_setup(self, lags, origin_every, max_origins, qa, qc):
        """Multiple-origin correlations from the current state (time 0)."""
        self._corr_lags = len(np.asarray(lags).reshape(-1))
        mc_corr_setup(self.h, lags, origin_every, max_origins, qa, qc)

    def corr_run(self, n, T, mix, seed):
        Ts = np.broadcast_to(np.asarray(T, dtype=np.float64), (self.n_rep,))
        seeds = np.broadcast_to(np.asarray(seed, dtype=np.uint64), (self.n_rep,))
        mc_corr_run(self.h, n, Ts, mix, seeds)

    def corr_sums(self):
        return mc_corr_sums(self.h, self.n_rep, self._corr_lags)

    def corr_results(self):
        """(n_rep, n_lags, 11): see CORR_RESULT_FIELDS."""
        return mc_corr_results(self.h, self.n_rep, self._corr_lags)

    def corr_relaxation_time(self, which=0, level=float(np.exp(-1.0))):
        """Per replica: the time at which F_s (0), F_s^cm (1) or C_2 (2) reaches level."""
        return mc_corr_relaxation_time(self.h, which, level, self.n_rep)

    def md_setup(self, dt, tau_T, T, v0, force_precision="fp64"):
        """MD from the current positions: time step dt, thermostat time tau_T (<= 0: none), v0 (N, 3),
        pair forces in "fp64" or "fp32"."""
        mc_md_setup(self.h, dt, tau_T, np.broadcast_to(np.asarray(T, dtype=np.float64), (self.n_rep,)), v0,
                    force_precision)

    def md_run(self, n):
        mc_md_run(self.h, n)

    def md_state(self):
        """(v (N, 3), per replica [K, U, xi, eta, conserved energy])."""
        return mc_md_state(self.h, self.N, self.n_rep)

    def stats(self):
        return mc_state_stats(self.h, self.n_rep)

    def reset_stats(self):
        mc_reset_stats(self.h)

    def set_stream(self, stream_ptr):
        mc_set_stream(self.h, stream_ptr)


def mc_state_stats(h, n_rep):
    st = (mc_stats * n_rep)()
    _check(load().mc_state(h, None, None, st), "mc_state")
    return [stats_dict(s) for s in st]
