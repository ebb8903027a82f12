"""Pins of the numpy observables of Sec. III.B (Eq. 5-7) on constructed
trajectories whose correlation values are known in closed form."""
import math

import numpy as np
import pytest

import oracle
from oracle import observables as O
from paper_2506_21290_gb300 import workloads as W


def _state(M=27, seed=0):
    L = W.box_length(M)
    xyz, t = W.lattice_start(M, L, seed)
    q = oracle.quantize(xyz, L)
    return L, q, t


def test_qvectors_have_the_requested_modulus():
    L = W.box_length(1000)
    for q0 in (7.4, 5.1):
        qv = W.qvectors(L, q0)
        assert 3 <= len(qv) <= 48
        mod = np.linalg.norm(qv, axis=1)
        assert np.all(np.abs(mod - q0) <= 0.1 + 1e-12)
        n = qv * L / (2 * math.pi)
        assert np.allclose(n, np.round(n), atol=1e-9)      # on the box's reciprocal lattice


def test_correlations_are_one_at_the_time_origin():
    L, q, t = _state()
    X = q.astype(np.int64)
    kref = O.reference_sites(t)
    assert np.all(t[kref] == 1)
    u0 = O.orientation(q, L, kref)
    ob = O.observables(L, X, X, q, u0, kref, W.qvectors(L, 7.4), W.qvectors(L, 5.1))
    assert ob["F_s"] == 1.0 and ob["F_s_cm"] == 1.0
    assert ob["C_2"] == pytest.approx(1.0, abs=1e-15)


def test_uniform_translation():
    """Every atom displaced by the same d: F_s = F_s^cm = <cos(q.d)>_q, C_2 = 1."""
    L, q, t = _state()
    X0 = q.astype(np.int64)
    dfix = np.array([123456789, -987654321, 4000000000], dtype=np.int64)   # crosses the box
    X = X0 + dfix
    qt = (X & 0xFFFFFFFF).astype(np.uint32)
    kref = O.reference_sites(t)
    u0 = O.orientation(q, L, kref)
    qa, qc = W.qvectors(L, 7.4), W.qvectors(L, 5.1)
    ob = O.observables(L, X, X0, qt, u0, kref, qa, qc)
    d = dfix * (L / 2 ** 32)
    assert ob["F_s"] == pytest.approx(np.cos(qa @ d).mean(), abs=1e-12)
    assert ob["F_s_cm"] == pytest.approx(np.cos(qc @ d).mean(), abs=1e-12)
    assert ob["C_2"] == pytest.approx(1.0, abs=1e-9)


def test_orientation_reversal_and_quarter_turn():
    """u -> -u leaves P_2 = 1; a rotation by 90 degrees about an axis normal to
    u gives P_2(0) = -1/2 (Eq. 7 with l = 2)."""
    L = 10.0
    M = 4
    tri = W._template()
    xyz0 = np.concatenate([tri + np.array([2.0 + 2 * m, 3.0, 4.0]) for m in range(M)])
    t = np.tile(np.array([0, 1, 2], dtype=np.int32), M)
    q0 = oracle.quantize(xyz0, L)
    kref = O.reference_sites(t)
    u0 = O.orientation(q0, L, kref)
    # template lies in the xy plane: rotate by 90 degrees about z about each centroid
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    xyz1 = np.concatenate([tri @ Rz.T + np.array([2.0 + 2 * m, 3.0, 4.0]) for m in range(M)])
    q1 = oracle.quantize(xyz1, L)
    ob = O.observables(L, q1.astype(np.int64), q0.astype(np.int64), q1, u0, kref, W.qvectors(L, 7.4),
                       W.qvectors(L, 5.1))
    assert ob["C_2"] == pytest.approx(-0.5, abs=1e-7)
    xyz2 = np.concatenate([-tri + np.array([2.0 + 2 * m, 3.0, 4.0]) for m in range(M)])
    q2 = oracle.quantize(xyz2, L)
    ob = O.observables(L, q2.astype(np.int64), q0.astype(np.int64), q2, u0, kref, W.qvectors(L, 7.4),
                       W.qvectors(L, 5.1))
    assert ob["C_2"] == pytest.approx(1.0, abs=1e-7)
    # the centroid did not move: F_s^cm = 1
    assert ob["F_s_cm"] == pytest.approx(1.0, abs=1e-9)


def test_flip_leaves_orientation_vector_unchanged():
    """A flip swaps types, not indices; u follows index k (Sec. III.B)."""
    L, q, t = _state()
    kref = O.reference_sites(t)
    u0 = O.orientation(q, L, kref)
    t2 = t.reshape(-1, 3)[:, [1, 0, 2]].reshape(-1)     # swap types of slots 0 and 1
    X = q.astype(np.int64)
    ob = O.observables(L, X, X, q, u0, kref, W.qvectors(L, 7.4), W.qvectors(L, 5.1))
    assert ob["C_2"] == pytest.approx(1.0, abs=1e-15)
    assert not np.array_equal(O.reference_sites(t2), kref)
