"""Pins of the oracle's multi-sweep accumulation (orc_accumulate, orc_project,
Sec. IV-A.1) against scipy's rotations, the identity pose and the round trip
sensor -> world -> body of the same pose."""
import numpy as np
import pytest


def _q(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def test_accumulate_is_pose_transform(orc):
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(0)
    ps = rng.normal(0, 8, (500, 3))
    for _ in range(5):
        q, p = _q(rng), rng.normal(0, 20, 3)
        ref = p + Rot.from_quat([q[1], q[2], q[3], q[0]]).apply(ps)   # scipy is (x, y, z, w)
        assert np.abs(orc.accumulate(ps, p, q) - ref).max() < 1e-12
        # a non-unit quaternion is normalised first
        assert np.abs(orc.accumulate(ps, p, 3.7 * q) - ref).max() < 1e-12


def test_identity_pose_and_round_trip(orc):
    rng = np.random.default_rng(1)
    ps = rng.normal(0, 8, (300, 3))
    assert np.array_equal(orc.accumulate(ps, [0, 0, 0], [1, 0, 0, 0]), ps)
    q, p = _q(rng), rng.normal(0, 20, 3)
    back = orc.project(orc.accumulate(ps, p, q), p, q)
    assert np.abs(back - ps).max() < 1e-12
    # projecting into another pose equals composing the relative transform
    q2, p2 = _q(rng), rng.normal(0, 20, 3)
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    r1 = Rot.from_quat([q[1], q[2], q[3], q[0]])
    r2 = Rot.from_quat([q2[1], q2[2], q2[3], q2[0]])
    ref = (r2.inv() * r1).apply(ps) + r2.inv().apply(p - p2)
    assert np.abs(orc.project(orc.accumulate(ps, p, q), p2, q2) - ref).max() < 1e-11
