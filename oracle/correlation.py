"""Multiple-origin time correlations and their statistics, plain numpy FP64.

Test infrastructure only (see the package docstring): the library's mc_corr_*
calls are checked against this.

Per time origin t_o and lag l the per-particle values are those of Eq. 5-7
(oracle.observables): fs_i per atom, fcm_i and c2_i per molecule, with the
instantaneous averages F_s, F_s^cm, C_2 of one sample.  Over the samples of a
lag:
  - the averages of F_s, F_s^cm, C_2 (the time-correlation series);
  - chi_4 = P (<C^2> - <C>^2), <> over samples, P = N atoms for F_s and
    M molecules for F_s^cm and C_2 (Eq. chi4, Sec. III.E);
  - chi_4^self = <C_i^2> - <C_i>^2 over the particles of all samples
    (Sec. III.E);
  - rho = Pearson coefficient of (c2_i, fcm_i) over the molecules of all
    samples (Eq. pearson, Sec. III.F).
Here the statistics are taken from the stored per-particle arrays with numpy's
var and corrcoef.

The origin schedule is an interface choice of the library, not the paper's:
the clock t starts at 0 at construction and counts sweeps; at each t,
(1) every live origin with t - t_o in lags is sampled, (2) origins with
t - t_o >= lags[-1] retire, (3) if t % every == 0 and fewer than max_origins
are live, the state becomes an origin, sampled at once if lags[0] == 0.
"""
from __future__ import annotations

import numpy as np

from . import observables as O

NSUM = 16
NRES = 11


class Correlator:
    def __init__(self, chain, lags, every, max_origins, qvec_atom, qvec_cm):
        self.ch = chain
        self.lags = [int(x) for x in lags]
        self.every = int(every)
        self.max_origins = int(max_origins)
        self.qa = np.asarray(qvec_atom, dtype=np.float64).reshape(-1, 3)
        self.qc = np.asarray(qvec_cm, dtype=np.float64).reshape(-1, 3)
        self.t = 0
        self.origins = []                        # live origins: dicts with t0, X0, u0, kref
        self.samples = [[] for _ in self.lags]   # per lag: list of (fs_i, fcm_i, c2_i)
        self._events()

    def run(self, n_sweeps, T, mix, seed):
        for _ in range(int(n_sweeps)):
            self.ch.run(1, T, mix, seed=seed)
            self.t += 1
            self._events()

    def _sample(self, o, li):
        ch = self.ch
        r = O.observables(ch.L, ch.X, o["X0"], ch.q, o["u0"], o["kref"], self.qa, self.qc)
        self.samples[li].append((r["F_s_i"], r["F_s_cm_i"], r["C_2_i"]))

    def _events(self):
        for o in self.origins:
            lag = self.t - o["t0"]
            if lag in self.lags:
                self._sample(o, self.lags.index(lag))
        self.origins = [o for o in self.origins if self.t - o["t0"] < self.lags[-1]]
        if self.t % self.every == 0 and len(self.origins) < self.max_origins:
            ch = self.ch
            kref = O.reference_sites(ch.t)
            o = {"t0": self.t, "X0": ch.X.copy(), "kref": kref, "u0": O.orientation(ch.q, ch.L, kref)}
            self.origins.append(o)
            if self.lags[0] == 0:
                self._sample(o, 0)

    def counts(self):
        return np.array([len(s) for s in self.samples], dtype=np.int64)

    def sums(self):
        return np.array([sums_of_samples(ss) for ss in self.samples]).reshape(len(self.lags), NSUM)

    def results(self):
        return np.array([stats_of_samples(ss) for ss in self.samples]).reshape(len(self.lags), NRES)


def sums_of_samples(ss):
    """The library's 16 sums of one lag from its samples [(fs_i, fcm_i, c2_i), ...]."""
    out = np.zeros(NSUM)
    for fs, fcm, c2 in ss:
        out[0] += 1
        out[1] += fs.mean()
        out[2] += fs.mean() ** 2
        out[3] += fs.sum()
        out[4] += (fs * fs).sum()
        out[5] += fcm.mean()
        out[6] += fcm.mean() ** 2
        out[7] += fcm.sum()
        out[8] += (fcm * fcm).sum()
        out[9] += c2.mean()
        out[10] += c2.mean() ** 2
        out[11] += c2.sum()
        out[12] += (c2 * c2).sum()
        out[13] += (c2 * fcm).sum()
    return out


def stats_of_samples(ss):
    """n, F_s, F_s^cm, C_2, chi_4 (3), chi_4^self (3), rho of one lag's samples."""
    out = np.full(NRES, np.nan)
    out[0] = len(ss)
    if not ss:
        return out
    fs = [s[0] for s in ss]
    fcm = [s[1] for s in ss]
    c2 = [s[2] for s in ss]
    N, M = fs[0].size, fcm[0].size
    means = [np.array([a.mean() for a in arrs]) for arrs in (fs, fcm, c2)]
    out[1:4] = [m.mean() for m in means]
    out[4:7] = [P * m.var() for P, m in zip((N, M, M), means)]
    pooled = [np.concatenate(arrs) for arrs in (fs, fcm, c2)]
    out[7:10] = [p.var() for p in pooled]
    if pooled[1].var() > 0 and pooled[2].var() > 0:
        out[10] = np.corrcoef(pooled[2], pooled[1])[0, 1]
    return out


def relaxation_time(lags, series, counts, level):
    """The time at which a lag series first reaches level (Sec. III.C, level
    e^-1): lags without samples are skipped; between the bracketing lags the
    crossing is placed linearly in ln t (linearly in t from lag 0); the first
    sampled lag itself when the series starts at or below level; NaN if it
    never crosses."""
    pts = [(float(t), float(f)) for t, f, n in zip(lags, series, counts) if n > 0]
    for k, (t, f) in enumerate(pts):
        if f <= level:
            if k == 0:
                return t
            t0, f0 = pts[k - 1]
            a = (f0 - level) / (f0 - f)
            if t0 > 0:
                return float(np.exp(np.log(t0) + a * (np.log(t) - np.log(t0))))
            return t0 + a * (t - t0)
    return float("nan")
