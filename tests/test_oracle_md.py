"""Pins of the oracle's molecular dynamics (no GPU).

The forces are checked against the energy of the C oracle (separate code) by
central differences; the integrator by what it must conserve: K + U without a
thermostat, and K + U + Q xi^2/2 + g T eta with the Nose-Hoover thermostat.
"""
import numpy as np
import pytest

import oracle
from oracle import md as MD
from paper_2506_21290_gb300 import workloads as W

POT = W.PAPER_POT


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _state(M=64, T=2.0, sweeps=10, seed=1):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    ch = oracle.Chain(L, xyz, t, POT)
    n = 2
    while np.floor(2 ** 32 / (n + 2)) * L / 2 ** 32 >= 1.575:
        n += 2
    ch.run(sweeps, T, W.PAPER_MIX, seed=seed, nc=n)
    return L, ch


def test_forces_are_minus_the_energy_gradient():
    L, ch = _state()
    F = MD.forces(L, ch.q, ch.t, POT)
    h = L / 2 ** 32
    k = 2 ** 12                           # displacement in fixed-point units (about 1.3e-6 sigma)
    for i in (0, 5, 77, 191):
        for ax in range(3):
            qp, qm = ch.q.copy(), ch.q.copy()
            qp[i, ax] += np.uint32(k)
            qm[i, ax] -= np.uint32(k)
            dU = (oracle.energy(L, qp, ch.t, POT) - oracle.energy(L, qm, ch.t, POT)) / (2 * k * h)
            assert F[i, ax] == pytest.approx(-dU, rel=1e-5, abs=1e-4), (i, ax)
    assert np.allclose(F.sum(axis=0), 0.0, atol=1e-9)                 # Newton's third law


# the configurations start near equilibrium (300 MC sweeps at T = 1.5); the
# drifts measured at dt = 0.001 over 1000 steps are a few 1e-6 relative


def test_constant_energy_without_thermostat():
    L, ch = _state(T=1.5, sweeps=300)
    v0 = W.maxwell_velocities(ch.t.size, 1.5, 3)
    m = MD.MD(L, ch.q, ch.X, ch.t, POT, 0.001, 0.0, 1.5, v0)
    E0 = m.conserved(oracle.energy(L, m.q, m.t, POT))
    m.step(1000)
    E1 = m.conserved(oracle.energy(L, m.q, m.t, POT))
    assert abs(E1 - E0) < 5e-5 * abs(E0)
    assert m.xi == 0.0


def test_nose_hoover_conserved_energy():
    L, ch = _state(T=1.5, sweeps=300)
    v0 = W.maxwell_velocities(ch.t.size, 2.0, 4)         # start hotter than the bath: the thermostat has work to do
    m = MD.MD(L, ch.q, ch.X, ch.t, POT, 0.001, 1.0, 1.5, v0)
    H0 = m.conserved(oracle.energy(L, m.q, m.t, POT))
    m.step(1000)
    H1 = m.conserved(oracle.energy(L, m.q, m.t, POT))
    assert m.xi > 0.1                                     # friction switched on to cool the system
    assert abs(H1 - H0) < 5e-5 * abs(H0)
