"""The state's host entry points at sizes that spread their work over several
host threads (more than 8192 molecules per call).

mc_set_state stores every position as a 32-bit fixed-point fraction of the
box, q = floor(frac(x / L) 2^32), and mc_state returns q L / 2^32: the round
trip is checked bit for bit against that rule written out in numpy.  When the
input is invalid, mc_set_state reports the error the serial order meets first
(replicas in order; within a replica every site, in order, before any bond),
whichever host thread finds it, and leaves the state as it was.
"""
import numpy as np
import pytest

from paper_2506_21290_gb300 import flipmc as F
from paper_2506_21290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POT = W.PAPER_POT


def _start(M, seed):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed=seed, candidates=1, passes=1)
    return L, xyz, t


def _quantised(xyz, L):
    t = xyz / L
    t = t - np.floor(t)
    v = np.floor(t * 2.0 ** 32)
    v[v >= 2.0 ** 32] = 0.0
    return v * (L / 2.0 ** 32)


def _stretch(xyz, mol):
    """Move atom 1 of molecule `mol` 3 sigma along each axis: its bonds (about
    1 sigma_ab long) pass 1.5 sigma_ab whatever their direction."""
    out = xyz.copy()
    out[3 * mol + 1] += 3.0
    return out


def _expect(h, xyz, t, code, text):
    with pytest.raises(F.McError) as e:
        h.set_state(xyz, t)
    assert e.value.code == code
    assert text in str(e.value)


def test_round_trip_is_the_fixed_point_rule():
    M = 20000
    L, xyz, t = _start(M, 5)
    h = F.Handle(L, xyz, t, POT)
    moved = xyz + np.array([0.31, -7.7, 2.0 * L + 0.05])     # wraps across the box in y and z
    h.set_state(moved, t)
    out, types, _ = h.state()
    assert np.array_equal(out, _quantised(moved, L))
    assert np.array_equal(types, t)


def test_first_error_in_serial_order_one_replica():
    M = 20000
    L, xyz, t = _start(M, 6)
    h = F.Handle(L, xyz, t, POT)
    before, _, _ = h.state()
    # a bond error early and a non-finite position late: every site comes first
    bad = _stretch(xyz, 1500)
    bad[3 * 18000, 2] = np.nan
    _expect(h, bad, t, F.MC_ERR_BAD_STATE, "non-finite position")
    # a type error after a bond error in the same replica
    bad_t = t.copy()
    bad_t[3 * 19999 + 2] = 3
    _expect(h, _stretch(xyz, 100), bad_t, F.MC_ERR_INVALID_ARG, "type outside {0,1,2}")
    # two bond errors in different thread chunks: the lower molecule
    _expect(h, _stretch(_stretch(xyz, 17000), 3000), t, F.MC_ERR_BAD_STATE, "molecule 3000)")
    # nothing was taken
    after, _, _ = h.state()
    assert np.array_equal(after, before)


def test_first_error_in_serial_order_two_replicas():
    M = 9000
    La, xa, ta = _start(M, 7)
    Lb, xb, tb = _start(M, 8)
    L = np.array([La, Lb])
    xyz = np.concatenate([xa, xb])
    t = np.concatenate([ta, tb])
    h = F.Handle(L, xyz, t, POT, n_mol=[M, M])
    off = 3 * M
    # replica 0's last site before replica 1's first bond
    bad = xyz.copy()
    bad[off - 1, 0] = np.inf
    bad[off + 1] += 3.0
    _expect(h, bad, t, F.MC_ERR_BAD_STATE, "non-finite position")
    # bond errors in both replicas: replica 0's
    bad = xyz.copy()
    bad[3 * 8000 + 1] += 3.0
    bad[off + 3 * 5 + 1] += 3.0
    _expect(h, bad, t, F.MC_ERR_BAD_STATE, "(replica 0, molecule 8000)")
    # a bond error in replica 1 only
    bad = xyz.copy()
    bad[off + 3 * 8999 + 1] += 3.0
    _expect(h, bad, t, F.MC_ERR_BAD_STATE, "(replica 1, molecule 8999)")
    h.set_state(xyz, t)
    out, _, _ = h.state()
    assert np.array_equal(out[:off], _quantised(xa, La))
    assert np.array_equal(out[off:], _quantised(xb, Lb))
