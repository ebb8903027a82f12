"""GPU molecular dynamics (mc_md_*) against the oracle's numpy MD.

The start is a state the FP64 MC chain reaches identically on both sides; the
velocities are the same seeded input.  The two MD trajectories agree to
rounding: CUDA's and numpy's exp and the order of the force sums differ in the
last bit, which 200 steps do not amplify beyond the tolerances below.
"""
import numpy as np
import pytest

import oracle
from oracle import md as OMD
from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.PAPER_POT


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21290_gb300 import build as B
    B.build()
    oracle.build()


@pytest.mark.parametrize("M,tau,seed", [(64, 1.0, 1), (125, 1.0, 2), (125, 0.0, 3)])
def test_md_matches_oracle(M, tau, seed):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    h = F.Handle(L, xyz, t, POT, precision="fp64")
    ch = oracle.Chain(L, xyz, t, POT, nc=h.info["max_cells_per_axis"])
    h.sweep(60, 1.5, W.PAPER_MIX, seed)
    ch.run(60, 1.5, W.PAPER_MIX, seed=seed)
    q, X, tt = h.state_fixed()
    assert np.array_equal(q, ch.q)
    v0 = W.maxwell_velocities(3 * M, 2.0, seed)
    h.md_setup(0.001, tau, 1.5, v0)
    m = OMD.MD(L, ch.q, ch.X, ch.t, POT, 0.001, tau, 1.5, v0)
    for _ in range(4):
        h.md_run(50)
        m.step(50)
        q, X, tt = h.state_fixed()
        assert np.max(np.abs(X - m.X)) <= 2                      # fixed-point units (h = L / 2^32)
        v, st = h.md_state()
        assert np.allclose(v, m.v, rtol=1e-9, atol=1e-9)
        assert st[0, 2] == pytest.approx(m.xi, abs=1e-10)
        U = oracle.energy(L, m.q, m.t, POT)
        assert st[0, 1] == pytest.approx(U, rel=1e-10)
        assert st[0, 4] == pytest.approx(m.conserved(U), rel=1e-10)


def test_md_conservation_and_temperature_at_M1000():
    M, T = 1000, 1.5
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, 4)
    h = F.Handle(L, xyz, t, POT, precision="fp32")
    h.sweep(500, T, W.PAPER_MIX, 4)
    # constant energy without a thermostat
    h.md_setup(0.001, 0.0, T, W.maxwell_velocities(3 * M, T, 5))
    E0 = h.md_state()[1][0, 4]
    h.md_run(5000)
    E1 = h.md_state()[1][0, 4]
    assert abs(E1 - E0) < 1e-4 * abs(E0)
    # Nose-Hoover: the conserved energy stays, the kinetic temperature settles at T
    h.md_setup(0.001, 1.0, T, W.maxwell_velocities(3 * M, 2.5, 6))
    H0 = h.md_state()[1][0, 4]
    temps = []
    for k in range(40):
        h.md_run(250)
        st = h.md_state()[1][0]
        temps.append(2.0 * st[0] / (3.0 * 3 * M))
    H1 = h.md_state()[1][0, 4]
    print("MD: E drift %.2e, H' drift %.2e, <T_kin> last 20 blocks %.4f" %
          ((E1 - E0) / abs(E0), (H1 - H0) / abs(H0), np.mean(temps[20:])))
    assert abs(H1 - H0) < 1e-4 * abs(H0)
    assert np.mean(temps[20:]) == pytest.approx(T, rel=0.03)
    # MC sweeps continue from the MD configuration with a consistent running energy
    h.sweep(5, T, W.PAPER_MIX, 7)
    assert h.stats()[0]["e_run"] == pytest.approx(h.energy()[0], rel=1e-6)


def test_md_argument_errors():
    L = W.box_length(64)
    xyz, t = W.lattice_start(64, L, 8)
    h = F.Handle(L, xyz, t, POT)
    with pytest.raises(F.McError):
        h.md_run(1)
    v0 = np.zeros((192, 3))
    for dt, T in ((0.0, 1.0), (0.001, -1.0)):
        with pytest.raises(F.McError) as e:
            h.md_setup(dt, 1.0, T, v0)
        assert e.value.code == F.MC_ERR_INVALID_ARG


def test_fp32_forces_follow_the_fp64_trajectory():
    """FP32 pair terms (one rounding per axis of the exact differences, about
    1e-6 relative per force) against the FP64 path from the same start: over
    100 steps (t = 0.1) the velocities stay within 1e-3 and the positions
    within 1e-4 sigma; without a thermostat the energy drifts by less than
    1e-3 over 2000 steps."""
    M, T = 216, 1.5
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, 9)
    a = F.Handle(L, xyz, t, POT, precision="fp32")
    a.sweep(300, T, W.PAPER_MIX, 9)
    q, X, tt = a.state_fixed()
    b = F.Handle(L, xyz, t, POT, precision="fp32")
    b.set_state_fixed(q, X, tt)
    v0 = W.maxwell_velocities(3 * M, T, 10)
    a.md_setup(0.001, 0.0, T, v0, force_precision="fp64")
    b.md_setup(0.001, 0.0, T, v0, force_precision="fp32")
    a.md_run(100)
    b.md_run(100)
    va, sa = a.md_state()
    vb, sb = b.md_state()
    Xa, Xb = a.state_fixed()[1], b.state_fixed()[1]
    h = L / 2 ** 32
    assert np.max(np.abs(va - vb)) < 1e-3
    assert np.max(np.abs(Xa - Xb)) * h < 1e-4
    E0 = sb[0, 4]
    b.md_run(2000)
    E1 = b.md_state()[1][0, 4]
    print("FP32 forces: max |dv| %.2e, max |dx| %.2e, energy drift %.2e over 2000 steps"
          % (np.max(np.abs(va - vb)), np.max(np.abs(Xa - Xb)) * h, (E1 - E0) / abs(E0)))
    assert abs(E1 - E0) < 1e-3 * abs(E0)


def test_md_of_a_batch_equals_each_replica_alone():
    """Replicas of different size and temperature advanced together give, bit
    for bit, what each gives on its own handle: the kinetic-energy chunks and
    the forces are per replica."""
    Ms, Ts = [64, 125], [1.2, 2.0]
    Ls = [W.box_length(m) for m in Ms]
    st = [W.lattice_start(m, l, 20 + k) for k, (m, l) in enumerate(zip(Ms, Ls))]
    v0 = [W.maxwell_velocities(3 * m, T, 30 + k) for k, (m, T) in enumerate(zip(Ms, Ts))]
    hb = F.Handle(np.array(Ls), np.concatenate([s[0] for s in st]), np.concatenate([s[1] for s in st]), POT,
                  precision="fp32", n_mol=np.array(Ms))
    hb.md_setup(0.001, 1.0, np.array(Ts), np.concatenate(v0), force_precision="fp32")
    hb.md_run(150)
    vb, sb = hb.md_state()
    qb, Xb, tb = hb.state_fixed()
    off = 0
    for k, M in enumerate(Ms):
        h = F.Handle(Ls[k], st[k][0], st[k][1], POT, precision="fp32")
        h.md_setup(0.001, 1.0, Ts[k], v0[k], force_precision="fp32")
        h.md_run(150)
        v, s1 = h.md_state()
        q, X, t = h.state_fixed()
        sl = slice(off, off + 3 * M)
        assert np.array_equal(vb[sl], v) and np.array_equal(Xb[sl], X), k
        assert sb[k, 2] == s1[0, 2]                                    # xi
        off += 3 * M
