"""Static observables of a configuration, plain numpy FP64: the pair virial
and pressure (Sec. II.C quotes P = 30 at T = 1, rho = 1.2), the structure
factor (Eq. sq) and the pair-distance histogram behind g(r) (Eq. gr).

Test infrastructure only (see the package docstring).

Virial: W = sum over pairs i < j of -r dphi/dr, with phi the WCA term (Eq. 1)
for every pair inside its cutoff and, for two atoms of one molecule, the FENE
term (Eq. 2):
  WCA:  -r dphi/dr = 24 eps s6 (2 s6 - 1),  s6 = (sigma_ab^2 / r^2)^3
  FENE: -r dphi/dr = -2 K eps x / (1 - x),  x = r^2 / (R0 sigma_ab)^2
Pressure: P = N T / V + W / (3 V), N atoms, V = L^3.
Pairs use the minimum image from the int32 difference of the 32-bit
fixed-point coordinates (x = q L / 2^32).
Structure factor: S(q) = |sum_i exp(i q . x_i)|^2 / N over the wrapped
positions; the double sum of Eq. sq with the i = j terms, so the i != j sum is
S - 1.
Pair histogram: the pairs i < j per bin floor(r / dr), r from the FP64
minimum-image distance computed as ((x^2 + y^2) + z^2) of the rounded
products dx h, then sqrt, then the division by dr, so that the same FP64
operations take the same bin decision as the library's.
"""
from __future__ import annotations

import numpy as np


def _h(L):
    return float(L) / 4294967296.0


def pair_vectors(L, q, i):
    """Minimum-image vectors (length units) from atom i to atoms j > i."""
    q = np.asarray(q, dtype=np.uint32).reshape(-1, 3)
    d = (q[i + 1:] - q[i]).view(np.int32).astype(np.float64) * _h(L)
    return d


def pair_w(r2, sab, bonded, pot):
    """-r dphi/dr of pairs at squared distances r2 with mixed diameters sab
    (arrays), FENE included where bonded."""
    eps, K, R0 = float(pot[3]), float(pot[4]), float(pot[5])
    s6 = (sab * sab / r2) ** 3
    inside = r2 < 2.0 ** (1.0 / 3.0) * sab * sab
    w = np.where(inside, 24.0 * eps * s6 * (2.0 * s6 - 1.0), 0.0)
    x = np.where(bonded, r2 / (R0 * sab) ** 2, 0.0)
    return w + np.where(bonded, -2.0 * K * eps * x / (1.0 - x), 0.0)


def virial(L, q, t, pot) -> float:
    sig = np.asarray(pot[:3], dtype=np.float64)
    t = np.asarray(t).reshape(-1)
    N = t.size
    W = 0.0
    for i in range(N - 1):
        d = pair_vectors(L, q, i)
        r2 = (d * d).sum(axis=1)
        sab = 0.5 * (sig[t[i]] + sig[t[i + 1:]])
        same = (np.arange(i + 1, N) // 3) == (i // 3)
        W += pair_w(r2, sab, same, pot).sum()
    return float(W)


def pressure(L, q, t, pot, T) -> float:
    N = np.asarray(t).size
    V = float(L) ** 3
    return N * float(T) / V + virial(L, q, t, pot) / (3.0 * V)


def structure_factor(L, q, qvec) -> np.ndarray:
    x = np.asarray(q, dtype=np.uint32).reshape(-1, 3).astype(np.float64) * _h(L)
    qv = np.asarray(qvec, dtype=np.float64).reshape(-1, 3)
    rho = np.exp(1j * (x @ qv.T)).sum(axis=0)
    return (rho.real ** 2 + rho.imag ** 2) / x.shape[0]


def pair_histogram(L, q, dr, n_bins) -> np.ndarray:
    q = np.asarray(q, dtype=np.uint32).reshape(-1, 3)
    h = _h(L)
    counts = np.zeros(n_bins, dtype=np.int64)
    for i in range(q.shape[0] - 1):
        d = (q[i + 1:] - q[i]).view(np.int32).astype(np.float64)
        x, y, z = d[:, 0] * h, d[:, 1] * h, d[:, 2] * h
        r2 = (x * x + y * y) + z * z
        b = np.floor(np.sqrt(r2) / dr)
        b = b[b < n_bins].astype(np.int64)
        counts += np.bincount(b, minlength=n_bins)
    return counts


def pair_correlation(L, counts, N, dr) -> np.ndarray:
    """g(r) per bin: 2 counts / (N rho V_shell), rho = N / L^3."""
    r0 = np.arange(len(counts)) * dr
    shell = 4.0 / 3.0 * np.pi * ((r0 + dr) ** 3 - r0 ** 3)
    return 2.0 * np.asarray(counts, dtype=np.float64) / (N * (N / float(L) ** 3) * shell)
