"""Molecular dynamics of the model (Sec. II.D), plain numpy FP64.

Test infrastructure only (see the package docstring).  m = 1, forces
F = -grad U over all pairs (WCA on every pair inside its cutoff, Eq. 1; FENE on
the three bonds of a molecule, Eq. 2), minimum image from the int32
difference of the 32-bit fixed-point coordinates.  One step is the symmetric
splitting of velocity Verlet and a Nose-Hoover thermostat (g = 3N degrees of
freedom, Q = g T tau^2):
  xi += dt/2 (2K - gT)/Q; eta += dt/2 xi; v = v exp(-xi dt/2) + dt/2 F
  q += rint(v dt / h)      (h = L / 2^32; positions stay fixed point)
  F(q)
  v = (v + dt/2 F) exp(-xi dt/2); xi += dt/2 (2K - gT)/Q; eta += dt/2 xi
with K = sum v^2 / 2.  The conserved energy is K + U + Q xi^2 / 2 + g T eta.
Without a thermostat (tau <= 0) xi stays 0 and K + U is conserved.
"""
from __future__ import annotations

import numpy as np

from . import structure as S

TWO32 = 4294967296.0


def forces(L, q, t, pot) -> np.ndarray:
    q = np.asarray(q, dtype=np.uint32).reshape(-1, 3)
    t = np.asarray(t).reshape(-1)
    N = t.size
    sig = np.asarray(pot[:3], dtype=np.float64)
    h = float(L) / TWO32
    d = (q[None, :, :] - q[:, None, :]).view(np.int32).astype(np.float64) * h    # x_j - x_i
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    np.fill_diagonal(r2, 1.0)
    sab = 0.5 * (sig[t][:, None] + sig[t][None, :])
    mol = np.arange(N) // 3
    bonded = mol[:, None] == mol[None, :]
    np.fill_diagonal(bonded, False)
    w = S.pair_w(r2, sab, bonded, pot) / r2
    np.fill_diagonal(w, 0.0)
    return -(w[..., None] * d).sum(axis=1)


def kinetic(v) -> float:
    v = np.asarray(v, dtype=np.float64)
    return 0.5 * float(((v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]).sum())


class MD:
    def __init__(self, L, q, X, t, pot, dt, tau, T, v0):
        self.L, self.pot, self.T = float(L), pot, float(T)
        self.q = np.asarray(q, dtype=np.uint32).reshape(-1, 3).copy()
        self.X = np.asarray(X, dtype=np.int64).reshape(-1, 3).copy()
        self.t = np.asarray(t, dtype=np.int32).reshape(-1)
        self.dt, self.hdt = float(dt), 0.5 * float(dt)
        self.g = 3.0 * self.t.size
        self.Q = self.g * self.T * tau * tau if tau > 0 else np.inf
        self.v = np.asarray(v0, dtype=np.float64).reshape(-1, 3).copy()
        self.xi = 0.0
        self.eta = 0.0
        self.F = forces(self.L, self.q, self.t, pot)

    def _thermostat(self):
        if np.isfinite(self.Q):
            self.xi = self.xi + self.hdt * ((2.0 * kinetic(self.v) - self.g * self.T) / self.Q)
            self.eta = self.eta + self.hdt * self.xi

    def step(self, n=1):
        s = self.dt * (TWO32 / self.L)
        for _ in range(int(n)):
            self._thermostat()
            self.v = self.v * np.exp(-self.xi * self.hdt) + self.hdt * self.F
            self.X = self.X + np.rint(self.v * s).astype(np.int64)
            self.q = (self.X & 0xFFFFFFFF).astype(np.uint32)
            self.F = forces(self.L, self.q, self.t, self.pot)
            self.v = (self.v + self.hdt * self.F) * np.exp(-self.xi * self.hdt)
            self._thermostat()

    def conserved(self, U) -> float:
        extra = 0.5 * self.Q * self.xi ** 2 + self.g * self.T * self.eta if np.isfinite(self.Q) else 0.0
        return kinetic(self.v) + U + extra
