"""Relaxation-time measurement of flip MC against local MC (Sec. III.C-D).

For each temperature, R replicas of M molecules at the paper's density run
from the lattice start with the flip mix (p_flip = 0.2) and with the local mix
(atom translations only, p_flip = 0; the paper's stand-in for the physical
dynamics, Sec. II.D).  After n_eq sweeps of equilibration the library's
multiple-origin correlator records F_s(q = 7.4, t) at log-spaced lags and each
replica's tau_alpha is the time at which F_s reaches e^-1 (Sec. III.C).  The
ratio tau(local) / tau(flip) at one temperature is the measurable part of the
speedup claim: how much faster flips decorrelate the liquid than
translations alone.

    python -m paper_2506_21290_gb300.speedup --T 2.5 2.0 1.6

prints one JSON line per (T, mix) and one per T with the ratio.  Every sweep
and every correlation sample runs in the CUDA library; this module only picks
the schedule and prints.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import flipmc as F
from . import workloads as W


def log_lags(lag_max: int, per_decade: int = 8) -> np.ndarray:
    """0 and about per_decade lags per decade up to lag_max (distinct integers)."""
    n = int(math.ceil(per_decade * math.log10(max(lag_max, 2)))) + 1
    lags = np.unique(np.round(np.logspace(0, math.log10(lag_max), n)).astype(np.int64))
    return np.concatenate([[0], lags])


def measure(T: float, mix, M: int, R: int, lag_max: int, n_eq: int, n_run: int, seed: int,
            precision: str = "fp32") -> dict:
    L = W.box_length(M)
    starts = [W.lattice_start(M, L, seed + r) for r in range(R)]
    h = F.Handle(np.full(R, L), np.concatenate([s[0] for s in starts]), np.concatenate([s[1] for s in starts]),
                 W.PAPER_POT, precision=precision, n_mol=np.full(R, M))
    Ts = np.full(R, T)
    seeds = np.arange(seed, seed + R, dtype=np.uint64)
    h.sweep(n_eq, Ts, mix, seeds)
    lags = log_lags(lag_max)
    every = max(1, lag_max // 8)
    h.corr_setup(lags, every, 16, W.qvectors(L, 7.4), W.qvectors(L, 5.1))
    h.corr_run(n_run, Ts, mix, seeds)
    tau = h.corr_relaxation_time(0)
    res = h.corr_results()
    fs = res[:, :, 1].mean(axis=0)
    ok = np.isfinite(tau)
    return {"T": T, "M": M, "replicas": R, "sweeps_equilibration": n_eq, "sweeps_measured": n_run,
            "tau_alpha": float(np.mean(tau[ok])) if ok.any() else None,
            "tau_alpha_sem": float(np.std(tau[ok]) / math.sqrt(ok.sum())) if ok.sum() > 1 else None,
            "replicas_crossed": int(ok.sum()),
            "lags": lags.tolist(), "F_s": [round(float(x), 5) for x in fs],
            "samples_at_last_lag": int(res[0, -1, 0])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--T", type=float, nargs="+", default=[2.5, 2.0, 1.6])
    ap.add_argument("--M", type=int, default=1000)
    ap.add_argument("--replicas", type=int, default=8)
    ap.add_argument("--lag-max", type=int, nargs="+", default=[2000, 5000, 20000],
                    help="largest lag per temperature (the last value repeats)")
    ap.add_argument("--seed", type=int, default=100)
    args = ap.parse_args()
    F.load()
    for k, T in enumerate(args.T):
        lag_max = args.lag_max[min(k, len(args.lag_max) - 1)]
        out = {}
        for name, mix in (("flip", W.PAPER_MIX), ("local", W.LOCAL_MIX)):
            r = measure(T, mix, args.M, args.replicas, lag_max, n_eq=lag_max, n_run=3 * lag_max, seed=args.seed)
            r["mix"] = name
            out[name] = r
            print(json.dumps(r), flush=True)
        a, b = out["flip"]["tau_alpha"], out["local"]["tau_alpha"]
        print(json.dumps({"T": T, "tau_local_over_tau_flip": (b / a) if (a and b) else None}), flush=True)


if __name__ == "__main__":
    main()
