"""Ensemble statistics over ranks (replicas only: one independent replica set
per GPU).

The correlation sums of replicas at one state point add (the layout of
mc_corr_sums), so an ensemble over ranks is a sum reduction of those rows
followed by the library's host-only derivation (mc_corr_derive).  The
reduction is the only collective; the sweeps never exchange data.
"""
from __future__ import annotations

import numpy as np

from . import flipmc as F


def allreduce_sums(sums: np.ndarray, dist=None) -> np.ndarray:
    """Sum of every rank's correlation-sum rows (any shape ending in 16); the
    rows themselves when dist is None or the world has one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return np.array(sums, dtype=np.float64, copy=True)
    import torch
    t = torch.from_numpy(np.ascontiguousarray(sums, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def ensemble_results(sums: np.ndarray, n_atoms, dist=None) -> np.ndarray:
    """Statistics (MC_CORR_NRES per row) of the sums reduced over all ranks."""
    return F.mc_corr_derive(allreduce_sums(sums, dist), n_atoms)
