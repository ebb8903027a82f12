"""Time-correlation observables of Sec. III.B, written out in plain numpy FP64.

Test infrastructure only (see the package docstring).  Definitions:
  - F_s(q,t)   = 1/N sum_j <cos(q . (r_j(t) - r_j(0)))>_q           (Eq. 5)
  - F_s^cm(q,t)= 1/M sum_j <cos(q . (r_j^cm(t) - r_j^cm(0)))>_q     (Eq. 6)
  - C_l(t)     = 1/M sum_j P_l(u_j(t) . u_j(0)),  l = 2               (Eq. 7)
Positions are indexed by site index, which a flip does not change (Sec. III.B);
r_j(t) - r_j(0) uses the unwrapped trajectory.  u_j points from the molecule's
centre of mass (equal masses) to the atom of index k_j, the atom of type B at
t = 0, whatever its type later.  The wavevectors are an input (a list of
3-vectors); the paper averages over vectors of modulus near 7.4 (atoms) and
5.1 (centres of mass).
"""
from __future__ import annotations

import numpy as np


def _h(L):
    return float(L) / 4294967296.0


def reference_sites(t0: np.ndarray) -> np.ndarray:
    """Per molecule, the site index that holds type B (=1) at t = 0."""
    t3 = np.asarray(t0).reshape(-1, 3)
    M = t3.shape[0]
    slot = np.argmax(t3 == 1, axis=1)
    has_b = (t3 == 1).any(axis=1)
    slot = np.where(has_b, slot, 0)
    return (3 * np.arange(M) + slot).astype(np.int64)


def orientation(q: np.ndarray, L: float, kref: np.ndarray) -> np.ndarray:
    """Unit vectors centre-of-mass -> site kref, from wrapped fixed-point q (N,3)."""
    q3 = np.asarray(q, dtype=np.uint32).reshape(-1, 3, 3)
    M = q3.shape[0]
    rel = (q3 - q3[:, :1, :]).view(np.int32).astype(np.float64) * _h(L)
    cm = ((rel[:, 0] + rel[:, 1]) + rel[:, 2]) / 3.0
    u = rel[np.arange(M), np.asarray(kref) - 3 * np.arange(M)] - cm
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def observables(L, X, X0, q, u0, kref, qvec_atom, qvec_cm):
    """Return dict with F_s, F_s_cm, C_2 and per-particle contributions.

    X, X0: (N,3) int64 unwrapped fixed point at t and 0; q: (N,3) wrapped at t;
    u0: (M,3) orientation at 0; kref: (M,) reference site index; qvec_*: (nq,3).
    """
    h = _h(L)
    dX = (np.asarray(X, dtype=np.int64) - np.asarray(X0, dtype=np.int64)).astype(np.float64) * h
    qa = np.asarray(qvec_atom, dtype=np.float64).reshape(-1, 3)
    qc = np.asarray(qvec_cm, dtype=np.float64).reshape(-1, 3)
    fs_i = np.cos(dX @ qa.T).mean(axis=1)
    d3 = dX.reshape(-1, 3, 3)
    dcm = ((d3[:, 0] + d3[:, 1]) + d3[:, 2]) / 3.0
    fscm_i = np.cos(dcm @ qc.T).mean(axis=1)
    u = orientation(q, L, kref)
    x = np.sum(u * np.asarray(u0, dtype=np.float64), axis=1)
    c2_i = 1.5 * x * x - 0.5
    return {
        "F_s": float(fs_i.mean()),
        "F_s_cm": float(fscm_i.mean()),
        "C_2": float(c2_i.mean()),
        "F_s_i": fs_i,
        "F_s_cm_i": fscm_i,
        "C_2_i": c2_i,
    }
