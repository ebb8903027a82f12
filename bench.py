#!/usr/bin/env python3
"""Throughput of the flip Monte Carlo sweep on GB300.

A step is `--sweeps-per-step` sweeps of the whole hot path (cell-list build,
8 checkerboard colour phases with translation and flip attempts, Metropolis,
commit, per-sweep energy bookkeeping) followed by one FP64 total-energy
recompute, over one synthetic configuration resident in HBM.  `value` is
attempted MC moves per second over all ranks in FP32 mode (FP32 pair Delta E,
FP64 totals); site-pair evaluations per second and their fraction of the FP32
peak are reported next to it, and the same workload is timed in FP64
oracle-match mode (`fp64`).  The default workload is 8000 molecules at
T = 0.75 (24000 atoms, 16^3 cells).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl native|reference]

N > 1 runs under torch.distributed.run, one independent replica set per GPU
(no data-path collective: replicas do not interact).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_21290_gb300 import workloads as W  # noqa: E402

METRIC = "MC attempted moves/sec and site-pair evals/sec (frac. FP32 peak), FP32 vs FP64"
UNIT = "attempted moves/s"
FLOPS_PER_PAIR_EVAL = 8      # per candidate distance: 3 scalings + r^2 (3 mul, 2 add)
FLOPS_PER_INTERACTION = 10   # per pair-potential evaluation in range: reciprocal, s^2, s^6, s^12, combine, add
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture of that kernel on that workload; keyed by (workload, kernel, sweeps
# per launch), so a timed launch that differs from the captured one reports null
NCU_TRAFFIC = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="single-8000", choices=sorted(W.WORKLOADS))
    ap.add_argument("--sweeps-per-step", type=int, default=0, help="0: workload default")
    ap.add_argument("--precision", default="", choices=["", "fp32", "fp64"])
    ap.add_argument("--launch-mode", type=int, default=0, choices=[0, 1, 2],
                    help="0 auto, 1 a CUDA graph per sweep, 2 one persistent launch per step")
    ap.add_argument("--warps-per-cell", type=int, default=0, choices=[0, 1, 2, 4, 8])
    ap.add_argument("--recheck-gap", type=float, default=0.0, help="FP32 decision margin (0: library default)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 oracle-match-mode leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--autotune", type=int, default=-1,
                    help="sweeps per schedule for mc_autotune when the schedule is automatic (0: off; -1: the "
                         "sweeps of one timed step, so that each trial is one launch of the shape timed)")
    ap.add_argument("--one-by-one", type=int, default=16,
                    help="batched workloads: replicas timed one by one on their own handles (0: off)")
    ap.add_argument("--md", type=int, default=0,
                    help="also time this many molecular-dynamics steps on the workload (0: off)")
    ap.add_argument("--corr", type=int, default=0,
                    help="also time the multiple-origin correlation sampling with this many origins "
                         "measured per event (0: off)")
    return ap.parse_args()


# sweeps per step (each step ends with an FP64 energy recompute): 20 for the
# single-8000 and batched workloads, 100 where the workload names that interval
DEFAULT_SPS = {"tiny-64": 100, "single-1000": 100, "single-8000": 20, "batched-256": 20, "large-64000": 100}


def combine_ranks(ms, attempts, pairs, dist=None, device="cpu"):
    """Whole-job numbers over the ranks of an N-GPU run: the slowest rank's time
    and the sum of every rank's attempts and pair evaluations (ranks run
    independent replica sets, so no data-path collective is involved)."""
    if dist is None:
        return float(ms), float(attempts), float(pairs)
    import torch
    tot = torch.tensor([float(ms), float(attempts), float(pairs)], dtype=torch.float64, device=device)
    mx = tot.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = tot.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(sm[2])


def config_of(name, wl, sps, precision, warmup, world):
    """The `config` object of a bench line (both arms)."""
    return {"workload": name, "molecules": wl["M_total"], "sites": 3 * wl["M_total"], "replicas": wl["replicas"],
            "T": wl["T"] if wl["replicas"] == 1 else "uniform [0.75, 3.0] per replica",
            "density": W.RHO, "sweeps_per_step": sps, "precision": precision,
            "move_mix": "atom translation 0.8 (d=0.1) / flip 0.2",
            "start": "simple-cubic lattice, random orientations, then %d warm-up steps" % warmup,
            "l2": "256 MiB buffer written between timed steps",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def make_workload(name, rank=0):
    spec = W.WORKLOADS[name]
    if "R" in spec:
        Ms, Ts = W.replica_mix(spec["R"], seed=spec["seed"])
        Ls = np.array([W.box_length(int(M)) for M in Ms])
        xyz, ts = [], []
        for k, M in enumerate(Ms):
            x, t = W.lattice_start(int(M), Ls[k], k)
            xyz.append(x)
            ts.append(t)
        seeds = np.arange(len(Ms), dtype=np.uint64) + np.uint64(1000 * rank)
        return dict(L=Ls, n_mol=Ms.astype(np.int32), xyz=np.concatenate(xyz), types=np.concatenate(ts), T=Ts,
                    seeds=seeds, M_total=int(Ms.sum()), replicas=len(Ms), precision=spec["precision"])
    M = spec["M"]
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, spec["seed"])
    return dict(L=L, n_mol=None, xyz=xyz, types=t, T=spec["T"], seeds=spec["seed"] + 1000 * rank, M_total=M,
                replicas=1, precision=spec["precision"])


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(device_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _cells_per_axis(L):
    """The cell grid the library picks (largest even n_c with cells >= 1.575 wide)."""
    nc = 2
    while math.floor(2 ** 32 / (nc + 2)) * L / 2 ** 32 >= 1.575:
        nc += 2
    return nc


def _oracle_replica(args):
    """Worker of the all-core CPU baseline: one replica's oracle chain, whole
    sweeps until `budget_s` has passed; returns (attempts, seconds)."""
    L, xyz, t, T, mix, budget_s, seed = args
    import oracle
    ch = oracle.Chain(L, xyz, t, W.PAPER_POT, nc=_cells_per_axis(L))
    n_sites = len(t)
    t0 = time.perf_counter()
    n = 0
    while True:
        ch.run(1, T, mix, seed=seed)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            return n * n_sites, dt


def cpu_baseline(wl, name, budget_s, T, mix):
    """The oracle, as it stands, on this host, on a bounded sample: one chain
    on one core for a single replica; for a batch, one replica per core on
    all cores at once (the first `cores` replicas), whole-job moves/s."""
    import oracle
    oracle.build()
    if wl["replicas"] > 1:
        import multiprocessing as mp
        cores = os.cpu_count() or 1
        n_mol = wl["n_mol"]
        offs = np.concatenate([[0], np.cumsum(3 * n_mol)])
        take = min(cores, len(n_mol))
        jobs = [(float(wl["L"][k]), wl["xyz"][offs[k]:offs[k + 1]], wl["types"][offs[k]:offs[k + 1]],
                 float(wl["T"][k]), mix, budget_s, int(wl["seeds"][k])) for k in range(take)]
        # spawn: a forked child of a process that has touched the GPU can hang
        with mp.get_context("spawn").Pool(take) as pool:
            res = pool.map(_oracle_replica, jobs)
        moves = sum(a for a, _ in res)
        wall = max(dt for _, dt in res)
        return {"value": moves / wall, "unit": UNIT, "cores": take, "kind": "oracle",
                "sample": "replicas 0..%d of the batch (%d-%d molecules), one per core at once, whole sweeps for "
                          "%.0f s each, FP64, O(N) Delta E per move" % (take - 1, int(n_mol[:take].min()),
                                                                       int(n_mol[:take].max()), budget_s),
                "cpu_model": _cpu_model()}
    L0, M0, xyz0, t0, T0 = wl["L"], wl["M_total"], wl["xyz"], wl["types"], T
    ch = oracle.Chain(L0, xyz0, t0, W.PAPER_POT, nc=_cells_per_axis(L0))
    t0w = time.perf_counter()
    ch.run(1, T0, mix, seed=1)
    one = time.perf_counter() - t0w
    n = max(1, int(budget_s / max(one, 1e-6)))
    t1 = time.perf_counter()
    ch.run(n, T0, mix, seed=1)
    dt = time.perf_counter() - t1
    return {"value": 3 * M0 * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d sweeps of %d molecules (%s), FP64, O(N) Delta E per move, after 1 untimed sweep"
                      % (n, M0, name), "cpu_model": _cpu_model()}


# Arm CPU part numbers of /proc/cpuinfo (Arm's published MIDR values)
ARM_PARTS = {"0xd0c": "Neoverse-N1", "0xd40": "Neoverse-V1", "0xd49": "Neoverse-N2", "0xd4f": "Neoverse-V2"}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        for key in ("model name", "CPU part"):
            for line in txt.splitlines():
                if line.startswith(key):
                    v = line.split(":", 1)[1].strip()
                    return "%s (%s)" % (ARM_PARTS.get(v, v), os.uname().machine)
    except OSError:
        pass
    return os.uname().machine


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args.workload)
    T = wl["T"] if wl["replicas"] == 1 else float(wl["T"][0])
    import oracle
    oracle.build()
    if wl["replicas"] > 1:
        M0 = int(wl["n_mol"][0])
        L0, xyz0, t0 = float(wl["L"][0]), wl["xyz"][: 3 * M0], wl["types"][: 3 * M0]
        sample = "one sweep of replica 0 (%d molecules) per step" % M0
    else:
        M0, L0, xyz0, t0 = wl["M_total"], wl["L"], wl["xyz"], wl["types"]
        sample = "one sweep of %d molecules per step" % M0
    ch = oracle.Chain(L0, xyz0, t0, W.PAPER_POT, nc=_cells_per_axis(L0))
    for _ in range(args.warmup):
        ch.run(1, T, W.PAPER_MIX, seed=1)
    t1 = time.perf_counter()
    for _ in range(args.steps):
        ch.run(1, T, W.PAPER_MIX, seed=1)
    dt = time.perf_counter() - t1
    v = 3 * M0 * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.workload, wl, args.sweeps_per_step or DEFAULT_SPS[args.workload],
                                wl["precision"], args.warmup, args.gpus),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "note": "each step times one oracle sweep (a bounded sample of the workload)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_one_by_one(F, wl, mix, sps, n_take, precision):
    """Moves/s of a sample of the batched replicas, each on its own handle and
    run one after the other (same sweeps per step, CUDA events per handle)."""
    import torch
    n_mol = wl["n_mol"]
    offs = np.concatenate([[0], np.cumsum(3 * n_mol)])
    take = np.linspace(0, len(n_mol) - 1, min(n_take, len(n_mol))).astype(int)
    total_ms, total_att = 0.0, 0
    for k in take:
        sl = slice(offs[k], offs[k + 1])
        hk = F.Handle(float(wl["L"][k]), wl["xyz"][sl], wl["types"][sl], W.PAPER_POT, precision=precision)
        st = torch.cuda.Stream()
        hk.set_stream(st.cuda_stream)
        hk.sweep(sps, float(wl["T"][k]), mix, int(wl["seeds"][k]))      # warm-up (first launch)
        a0 = sum(hk.stats()[0]["attempts"])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        hk.sweep(sps, float(wl["T"][k]), mix, int(wl["seeds"][k]))
        e1.record(st)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_att += sum(hk.stats()[0]["attempts"]) - a0
        hk.close()
    return {"value": total_att / (total_ms / 1000.0), "unit": UNIT, "replicas_timed": int(len(take)),
            "sweeps_each": sps, "what": "the same replicas, own handle each, one after the other"}


def run_corr(h, wl, mix, P, stream, n_events=10):
    """Cost of one correlation event with P (origin, lag) pairs over the whole
    state: lags 0..P-1, an origin every sweep, so that every sweep after the
    first P ends in an event of exactly P pairs.  Each timed sweep with its
    event is compared with the same sweep alone."""
    import torch
    rng = np.random.default_rng(2506)
    qa, qc = rng.normal(size=(12, 3)), rng.normal(size=(8, 3))
    qa *= 7.4 / np.linalg.norm(qa, axis=1, keepdims=True)
    qc *= 5.1 / np.linalg.norm(qc, axis=1, keepdims=True)
    h.corr_setup(np.arange(P), 1, P, qa, qc)
    h.corr_run(P + 2, wl["T"], mix, wl["seeds"])

    def timed(fn):
        tot = 0.0
        for _ in range(n_events):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / n_events

    with_ev = timed(lambda: h.corr_run(1, wl["T"], mix, wl["seeds"]))
    plain = timed(lambda: h.sweep(1, wl["T"], mix, wl["seeds"]))
    M = h.N // 3
    ev_ms = max(with_ev - plain, 1e-6)
    cos_per_pair = 3 * len(qa) + len(qc)
    return {"pairs_per_event": P, "event_ms": ev_ms, "sweep_plus_event_ms": with_ev, "sweep_ms": plain,
            "molecule_samples_per_s": P * M / (ev_ms * 1e-3),
            "fp64_cos_per_s": P * M * cos_per_pair / (ev_ms * 1e-3),
            "what": "per event: gather of the unwrapped positions, F_s (12 q), F_s^cm (8 q), C_2 per molecule "
                    "for each pair in FP64, fixed-order per-replica sums, one new origin"}


def run_md(h, wl, n_steps, stream):
    """Molecular dynamics on the workload's state after the MC measurement:
    dt = 0.001, Nose-Hoover with tau = 1 at the workload's temperature(s),
    with FP64 and with FP32 pair forces."""
    import torch
    T = np.broadcast_to(np.asarray(wl["T"], dtype=np.float64), (h.n_rep,))
    out = {"steps": n_steps,
           "what": "one step: thermostat half + kick, drift, cell-list rebuild (4 kernels), forces, kick + "
                   "thermostat half; one CUDA graph per step"}
    for prec in ("fp64", "fp32"):
        h.md_setup(0.001, 1.0, T, W.maxwell_velocities(h.N, float(np.mean(T)), 11), force_precision=prec)
        h.md_run(20)                      # warm-up, graphs instantiated
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.md_run(n_steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        out[prec + "_forces"] = {"ms_per_step": ms / n_steps, "steps_per_s": n_steps / (ms * 1e-3),
                                 "atom_steps_per_s": h.N * n_steps / (ms * 1e-3)}
    return out


def fp32_peak_tflops(sms, mhz):
    """FP32 peak: SMs x 128 FP32 lanes x 2 flop (fma) x clock."""
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def timed_steps(h, wl, mix, sps, steps, stream, flush, e_dev, drift=None):
    """`steps` timed steps (the sweeps, then the FP64 energy recompute), each
    bracketed by CUDA events on the library's stream, the L2 flushed before
    each.  Returns (total ms, sweep-only ms, stats before, stats after).  With
    `drift` (a list), after each step the relative drift of the running total
    against that step's recompute is appended (outside the events)."""
    import torch
    h.sync()
    torch.cuda.synchronize()
    st0 = h.stats()
    evs = []
    for _ in range(steps):
        flush.fill_(1)                 # evict the state from L2 between timed steps
        a = torch.cuda.Event(enable_timing=True)
        m = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.sweep(sps, wl["T"], mix, wl["seeds"])   # the sweep launch(es) of the step
        m.record(stream)
        h.energy_device(e_dev.data_ptr())         # FP64 energy recompute
        b.record(stream)
        evs.append((a, m, b))
        if drift is not None:
            b.synchronize()
            E = e_dev.cpu().numpy()
            er = np.array([s["e_run"] for s in h.stats()])
            drift.append(float(np.max(np.abs(er - E) / np.abs(E))))
    torch.cuda.synchronize()
    h.sync()
    ms = sum(a.elapsed_time(b) for a, m, b in evs)
    sweep_ms = sum(a.elapsed_time(m) for a, m, b in evs)
    return ms, sweep_ms, st0, h.stats()


def stat_delta(st0, st1, key):
    return sum(s1[key] - s0[key] for s0, s1 in zip(st0, st1))


def kernel_label(precision, info):
    persistent = info.get("launch_mode", 0) != 1
    return ("sweep_persistent" if persistent else "phase_kernel") + \
        ("<FP32,W=%d>" if precision == "fp32" else "<FP64,W=%d>") % info["warps_per_cell"]


def run_fp64_leg(F, wl, mix, sps, steps, warmup, autotune, stream, flush, sms):
    """The same workload from the same start in FP64 oracle-match mode (every
    Delta E the FP64 ordered sum, decisions bit-exact to the oracle's chain)."""
    import torch
    h = F.Handle(wl["L"], wl["xyz"], wl["types"], W.PAPER_POT, precision="fp64", n_mol=wl["n_mol"])
    if autotune > 0:
        h.autotune(autotune, wl["T"], mix, wl["seeds"])
    h.set_stream(stream.cuda_stream)
    e_dev = torch.zeros(h.n_rep, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        h.sweep(sps, wl["T"], mix, wl["seeds"])
        h.energy_device(e_dev.data_ptr())
    clocks = Clocks(torch.cuda.current_device())
    time.sleep(0.3)
    ms, sweep_ms, st0, st1 = timed_steps(h, wl, mix, sps, steps, stream, flush, e_dev)
    clk = clocks.stop()
    att = sum(sum(s1["attempts"]) - sum(s0["attempts"]) for s0, s1 in zip(st0, st1))
    pairs = stat_delta(st0, st1, "pair_evals")
    inter = stat_delta(st0, st1, "pair_interactions")
    flops = FLOPS_PER_PAIR_EVAL * pairs + FLOPS_PER_INTERACTION * inter
    info = h.info
    out = {"value": att / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "sweeps_per_step": sps, "pair_evals_per_s": pairs / (ms / 1000.0),
           "pair_interactions_per_s": inter / (ms / 1000.0),
           "fp32_peak_frac": flops / (ms / 1000.0) / (fp32_peak_tflops(sms, SM_MAX_MHZ) * 1e12),
           "kernel": kernel_label("fp64", info), "sweep_launch_ms": sweep_ms / steps,
           "schedule": {"warps_per_cell": info["warps_per_cell"],
                        "launch": "persistent" if info.get("launch_mode", 0) != 1 else "graph per sweep"},
           "what": "FP64 oracle-match mode: every Delta E the FP64 ordered sum (unfused, fixed order), FP64 "
                   "thresholds; same workload, start and timing as the FP32 line",
           "clocks": clk}
    h.close()
    return out, (ms, att)


def run_native(args):
    import torch
    from paper_2506_21290_gb300 import build as B
    from paper_2506_21290_gb300 import flipmc as F

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    F.load()
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    wl = make_workload(args.workload, rank)
    precision = args.precision or wl["precision"]
    sps = args.sweeps_per_step or DEFAULT_SPS[args.workload]
    mix = W.PAPER_MIX
    h = F.Handle(wl["L"], wl["xyz"], wl["types"], W.PAPER_POT, precision=precision, device=local, n_mol=wl["n_mol"],
                 launch_mode=args.launch_mode, warps_per_cell=args.warps_per_cell, recheck_gap=args.recheck_gap)
    N = h.N
    tuned = None
    trial = sps if args.autotune < 0 else args.autotune
    if trial > 0 and args.warps_per_cell == 0 and args.launch_mode == 0:
        # pick the cell schedule on a copy of the state (the chain is unchanged)
        res = h.autotune(trial, wl["T"], mix, wl["seeds"])
        tuned = {"ms_per_sweep": {"persistent": [float(x) for x in res[:4]], "graphs": [float(x) for x in res[4:]]},
                 "warps_per_cell": [1, 2, 4, 8], "sweeps_per_trial": trial}
    # a dedicated stream: the library enqueues on it, the events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    h.set_stream(stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    e_dev = torch.zeros(h.n_rep, dtype=torch.float64, device="cuda")

    for _ in range(args.warmup):
        h.sweep(sps, wl["T"], mix, wl["seeds"])
        h.energy_device(e_dev.data_ptr())
    h.sync()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    time.sleep(0.4)
    if dist is not None:
        dist.barrier()
    drift_series = []
    ms, sweep_ms, st0, st1 = timed_steps(h, wl, mix, sps, args.steps, stream, flush, e_dev, drift_series)
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    attempts = sum(sum(s1["attempts"]) - sum(s0["attempts"]) for s0, s1 in zip(st0, st1))
    pairs = stat_delta(st0, st1, "pair_evals")
    inter = stat_delta(st0, st1, "pair_interactions")
    rechecks = stat_delta(st0, st1, "fp64_rechecks")
    accepts = [sum(s1["accepts"][k] - s0["accepts"][k] for s0, s1 in zip(st0, st1)) for k in range(4)]
    att_k = [sum(s1["attempts"][k] - s0["attempts"][k] for s0, s1 in zip(st0, st1)) for k in range(4)]
    geom = stat_delta(st0, st1, "rejected_geometry")
    ms_max, attempts_all, pairs_all = combine_ranks(ms, attempts, pairs, dist, "cuda")
    _, inter_all, _ = combine_ranks(ms, inter, 0, dist, "cuda")
    value = attempts_all / (ms_max / 1000.0)
    pair_rate = pairs_all / (ms_max / 1000.0)
    flops_all = FLOPS_PER_PAIR_EVAL * pairs_all + FLOPS_PER_INTERACTION * inter_all

    # the dominant kernel is the sweep kernel: one persistent launch per step
    # (events around it in every timed step, on its stream); per-stage times of
    # the separate-kernel path are reported next to it
    info = h.info
    persistent = info.get("launch_mode", 0) != 1
    launch_ms = sweep_ms / args.steps
    flops_per_launch = (FLOPS_PER_PAIR_EVAL * pairs + FLOPS_PER_INTERACTION * inter) / args.steps
    achieved = flops_per_launch / (launch_ms / 1000.0) / 1e12
    n_prof = max(2, min(20, sps))
    stage_ms = h.sweep_timed(n_prof, wl["T"], mix, wl["seeds"])
    peak = fp32_peak_tflops(sms, SM_MAX_MHZ)
    peak_at_clock = fp32_peak_tflops(sms, clk["sm_mhz"]) if clk.get("sm_mhz") else None

    kernel_name = kernel_label(precision, info)
    traffic = NCU_TRAFFIC.get((args.workload, kernel_name, sps)) if persistent else None

    # drift of the FP64 running total (FP32 Delta E of the accepted moves)
    # against the step-end FP64 recomputes: cumulative, never re-based
    st_now = h.stats()
    energy_drift = {"sweeps_total": int(st_now[0]["sweeps"]), "sweeps_per_recompute": sps,
                    "series": drift_series, "max_rel": max(drift_series) if drift_series else None,
                    "final_rel": drift_series[-1] if drift_series else None,
                    "what": "|running FP64 total - FP64 recompute| / |recompute| at the end of each timed step "
                            "(worst replica), cumulative over the timed steps"}

    # the same replicas, each on its own handle and run one after the other
    one_by_one = None
    if wl["replicas"] > 1 and args.one_by_one > 0 and rank == 0:
        one_by_one = run_one_by_one(F, wl, mix, sps, args.one_by_one, precision)
        one_by_one["batched_over_one_by_one"] = value / one_by_one["value"]

    # FP64 oracle-match mode on the same workload
    fp64 = None
    if precision == "fp32" and not args.no_fp64:
        fp64, (ms64, att64) = run_fp64_leg(F, wl, mix, sps, args.steps, args.warmup, trial, stream, flush,
                                           sms)
        ms64_max, att64_all, _ = combine_ranks(ms64, att64, 0, dist, "cuda")
        fp64["value"] = att64_all / (ms64_max / 1000.0)
        fp64["fp32_over_fp64"] = value / fp64["value"]

    # end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        h.set_stream(0)
        torch.cuda.synchronize()
        xyz_h, t_h = wl["xyz"], wl["types"]
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h.set_state(xyz_h, t_h)
            h.sweep(sps, wl["T"], mix, wl["seeds"])
            E = h.energy()
            xyz_o, t_o, _s = h.state()
        dt = time.perf_counter() - t0
        e2e = {"value": N * sps * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(16 * N), "d2h_bytes_per_step": int(28 * N + 8 * h.n_rep + 144 * h.n_rep),
               "steps": args.e2e_steps,
               "path": "mc_set_state (host positions) + mc_sweep + mc_energy + mc_state (host positions)"}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(wl, args.workload, args.cpu_seconds, wl["T"] if wl["replicas"] == 1 else None, mix)
    # our kernels per timed step: the sweeps (one persistent launch, or per
    # sweep 4 cell-list + 8 colour + 1 finalisation kernels in a graph) and the
    # energy recompute (2 kernels)
    launches_per_step = (1 if persistent else 13 * sps) + 2
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "f64",
        "data": "synthetic",
        "config": config_of(args.workload, wl, sps, precision, args.warmup, world),
        "pair_evals_per_s": pair_rate,
        "pair_interactions_per_s": inter_all / (ms_max / 1000.0),
        "pair_evals_fp32_peak_frac": flops_all / (ms_max / 1000.0) / (peak * 1e12),
        "fp64": fp64,
        "fp64_recheck_rate": rechecks / max(attempts, 1),
        "acceptance": [accepts[k] / att_k[k] if att_k[k] else None for k in range(4)],
        "geometry_reject_rate": geom / max(attempts, 1),
        "roofline": {"bound": "alu",
                     "kernel": kernel_name,
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_unit": "B per launch (ncu dram__bytes_read + write)",
                     "peak_basis": "%d SMs x 128 FP32 lanes x 2 x 2070 MHz (max clock); derived, not measured" % sms,
                     "peak_at_measured_clock": peak_at_clock,
                     "launch_ms": launch_ms, "flops_per_launch": flops_per_launch,
                     "flops_basis": "%d per site-pair evaluation (2 or 6 x neighbourhood atoms per evaluated "
                                    "attempt) + %d per pair-potential evaluation in range"
                                    % (FLOPS_PER_PAIR_EVAL, FLOPS_PER_INTERACTION),
                     "separate_kernel_stage_ms_per_sweep": {"cell_list": stage_ms[0] / n_prof,
                                                            "8_phases": stage_ms[1] / n_prof,
                                                            "finalize": stage_ms[2] / n_prof}},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "energy_drift": energy_drift,
        "schedule": {"warps_per_cell": info["warps_per_cell"],
                     "launch": "persistent" if persistent else "graph per sweep",
                     "autotune": tuned},
        "one_by_one": one_by_one,
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clk,
    }
    if args.corr > 0:
        line["corr"] = run_corr(h, wl, mix, args.corr, stream)
    if args.md > 0:
        line["md"] = run_md(h, wl, args.md, stream)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
