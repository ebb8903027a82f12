"""Seeded synthetic inputs for the flip Monte Carlo library and its tests.

This module only generates inputs (initial configurations, temperatures,
wavevector lists, replica size mixes).  It holds none of the method's
arithmetic and imports neither the CUDA binding nor the oracle, so both can
consume exactly the same data.

Constants follow arXiv 2506.21290 Sec. II: sigma_A = 0.9, sigma_B = 1,
sigma_C = 1.1, eps = 1 (Sec. II.A), FENE prefactor 33.75 and range 1.5 sigma
(Eq. 2), number density rho = N/V = 1.2 with N = 3M atoms (Sec. II.A),
p_flip = 0.2 (Sec. II.B), temperatures from T = 3 down to 0.75 (Fig. 4).
The atom step size, the rigid-move widths and the initial lattice are not
given in the paper; the values here are this library's defaults.
"""
from __future__ import annotations

import math

import numpy as np

SIGMA = (0.9, 1.0, 1.1)
EPS = 1.0
FENE_K = 33.75
FENE_R0 = 1.5
RHO = 1.2
P_FLIP = 0.2
T_HIGH, T_MID, T_LOW = 3.0, 1.1, 0.75

#: potential parameters {sigma_A, sigma_B, sigma_C, eps, fene_K, fene_R0}
PAPER_POT = (SIGMA[0], SIGMA[1], SIGMA[2], EPS, FENE_K, FENE_R0)
#: move mix {p_atom, p_flip, p_mol_trans, p_mol_rot, d_atom, d_mol, rot_a}
PAPER_MIX = (1.0 - P_FLIP, P_FLIP, 0.0, 0.0, 0.1, 0.05, 0.05)
#: a mix that also uses the rigid-body moves
RIGID_MIX = (0.5, 0.2, 0.15, 0.15, 0.1, 0.05, 0.05)
#: local MC: atom translations only (Sec. II.C)
LOCAL_MIX = (1.0, 0.0, 0.0, 0.0, 0.1, 0.05, 0.05)

# bond lengths of the template triangle: 0.96 sigma_ab, near the WCA+FENE minimum
_BOND_SCALE = 0.96


def box_length(M: int, rho: float = RHO) -> float:
    """Side of the cubic box holding M three-site molecules at atom density rho."""
    return (3.0 * M / rho) ** (1.0 / 3.0)


def _template() -> np.ndarray:
    """Triangle A, B, C with sides 0.96 sigma_ab, centroid at the origin."""
    s = SIGMA
    ab = _BOND_SCALE * 0.5 * (s[0] + s[1])
    bc = _BOND_SCALE * 0.5 * (s[1] + s[2])
    ac = _BOND_SCALE * 0.5 * (s[0] + s[2])
    cx = (ab * ab + ac * ac - bc * bc) / (2.0 * ab)
    cy = math.sqrt(max(ac * ac - cx * cx, 0.0))
    tri = np.array([[0.0, 0.0, 0.0], [ab, 0.0, 0.0], [cx, cy, 0.0]])
    return tri - tri.mean(axis=0)


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniform random rotation matrices (Shoemake's quaternion method)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    x = a * np.cos(2 * np.pi * u2)
    y = b * np.sin(2 * np.pi * u3)
    z = b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def lattice_start(M: int, L: float, seed: int, candidates: int = 24, passes: int = 3):
    """Molecule centroids on a simple cubic lattice, uniform random orientations.

    The lattice has m = ceil(M^(1/3)) points per axis; molecules take the first M
    points in index order.  Each molecule's orientation is the best of
    `candidates` uniform random rotations (plus its current one after the first
    pass), "best" meaning the largest smallest distance, in units of
    sigma_ab, to the atoms of its face- and edge-neighbour molecules on the
    lattice.  Molecules are visited by lattice colour class (no two lattice
    neighbours share a class), so that the choice vectorises; `passes` rounds
    are made.  Returns (xyz (3M,3) float64,
    types (3M,) int32) with types A, B, C at slots 0, 1, 2 of every molecule.
    """
    rng = np.random.default_rng(seed)
    m = max(1, int(math.ceil(M ** (1.0 / 3.0) - 1e-9)))
    a = L / m
    idx = np.arange(M)
    lat = np.stack([idx % m, (idx // m) % m, idx // (m * m)], axis=1)
    centres = (lat + 0.5) * a
    tpl = _template()
    sig = np.asarray(SIGMA)
    inv_sab = 1.0 / (0.5 * (sig[:, None] + sig[None, :]))
    occ = -np.ones((m, m, m), dtype=np.int64)
    occ[lat[:, 0], lat[:, 1], lat[:, 2]] = idx
    offs = np.array([(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
                     if 0 < abs(dx) + abs(dy) + abs(dz) <= 2])
    nb = occ[(lat[:, None, 0] + offs[None, :, 0]) % m, (lat[:, None, 1] + offs[None, :, 1]) % m,
             (lat[:, None, 2] + offs[None, :, 2]) % m]                  # (M, 18), -1 = empty
    nb = np.where(nb == idx[:, None], -1, nb)
    # parity classes per axis; with m odd the last layer gets a class of its own
    # so that no two lattice neighbours (periodic) share a colour
    cls = np.where((m % 2 == 1) & (lat == m - 1), 2, lat & 1)
    colour = cls[:, 0] + 3 * cls[:, 1] + 9 * cls[:, 2]
    xyz = np.zeros((M, 3, 3))
    placed = np.zeros(M, dtype=bool)
    chunk = 512
    for p in range(passes):
        for col in range(27):
            ids_all = idx[colour == col]
            for c0 in range(0, ids_all.size, chunk):
                ids = ids_all[c0:c0 + chunk]
                R = _random_rotations(rng, ids.size * candidates).reshape(ids.size, candidates, 3, 3)
                cand = centres[ids][:, None, None, :] + np.einsum("ckij,sj->cksi", R, tpl)  # (c,K,3,3)
                if p > 0:
                    cand = np.concatenate([xyz[ids][:, None], cand], axis=1)
                nbi = nb[ids]                                                 # (c,18)
                valid = (nbi >= 0) & placed[np.maximum(nbi, 0)]
                other = xyz[np.maximum(nbi, 0)]                               # (c,18,3,3)
                d = (cand[:, :, :, None, None, :] - other[:, None, None, :, :, :]).astype(np.float32)
                d -= np.float32(L) * np.round(d / np.float32(L))             # (c,K,3,18,3,3)
                r = np.sqrt((d * d).sum(-1)) * inv_sab[None, None, :, None, :].astype(np.float32)
                r = np.where(valid[:, None, None, :, None], r, np.inf)
                best = np.argmax(r.min(axis=(2, 3, 4)), axis=1)
                xyz[ids] = cand[np.arange(ids.size), best]
                placed[ids] = True
    types = np.tile(np.array([0, 1, 2], dtype=np.int32), M)
    return np.ascontiguousarray(xyz.reshape(-1, 3)), types


def qvectors(L: float, q0: float, dq: float = 0.1, max_n: int = 48) -> np.ndarray:
    """Wavevectors 2 pi n / L of modulus within dq of q0 (one of each +-n pair),
    ordered by (|n|^2, n_x, n_y, n_z), at most max_n of them.  If no lattice
    vector lies in that shell (small boxes), the shell closest to q0 is used."""
    k = 2.0 * math.pi / L
    nmax = int(math.ceil((q0 + dq) / k)) + 1
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    # one representative of each +-n pair: first nonzero component positive
    first = np.where(n[:, 0] != 0, n[:, 0], np.where(n[:, 1] != 0, n[:, 1], n[:, 2]))
    n = n[first > 0]
    mod = k * np.sqrt((n * n).sum(1))
    dist = np.abs(mod - q0)
    n = n[dist <= max(dq, dist.min() + 1e-12)]
    order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], (n * n).sum(1)))
    n = n[order][:max_n]
    return np.ascontiguousarray(n.astype(np.float64) * k)


def replica_mix(R: int = 256, seed: int = 0, m_lo: int = 256, m_hi: int = 2000,
                t_lo: float = T_LOW, t_hi: float = T_HIGH):
    """Replica sizes M_r uniform in [m_lo, m_hi] and temperatures uniform in [t_lo, t_hi]."""
    rng = np.random.default_rng(0xBA7C + seed)
    Ms = rng.integers(m_lo, m_hi + 1, size=R)
    Ts = rng.uniform(t_lo, t_hi, size=R)
    return Ms.astype(np.int64), Ts


WORKLOADS = {
    # name: (M, T, seed, sweeps the paper-shaped run would take)
    "tiny-64": dict(M=64, T=T_HIGH, seed=0, sweeps=1000, precision="fp64"),
    "single-1000": dict(M=1000, T=T_MID, seed=1, sweeps=10_000, precision="fp32"),
    "single-8000": dict(M=8000, T=T_LOW, seed=2, sweeps=10_000, precision="fp32"),
    "batched-256": dict(R=256, T=None, seed=0, sweeps=1000, precision="fp32"),
    "large-64000": dict(M=64000, T=T_LOW, seed=3, sweeps=1000, precision="fp32"),
}


def maxwell_velocities(n_sites: int, T: float, seed: int) -> np.ndarray:
    """Initial MD velocities: each component normal with variance T (m = 1),
    then the mean velocity removed (seeded, numpy)."""
    v = np.random.default_rng(seed).normal(scale=math.sqrt(T), size=(n_sites, 3))
    return v - v.mean(axis=0, keepdims=True)
