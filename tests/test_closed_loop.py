"""CPU parts of the closed loop: the simulated quadrotor against the oracle's
rollout (same Eq. dynamics and RK4), and the exact scene distance against
brute force over densely sampled surfaces."""
import numpy as np

from paper_2509_17340_gb300 import closed_loop as L
from paper_2509_17340_gb300 import inputs as I


def test_simulated_drone_matches_oracle_rollout(orc):
    rng = np.random.default_rng(0)
    P = I.workload_params("ensemble")
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    x = np.concatenate([[1.0, -2.0, 1.5], q, [2.0, 0.5, -0.3]])
    U = np.tile([P["g"], 0, 0, 0], (30, 1)) + rng.normal(0, [2, 1.5, 1.5, 1.5], (30, 4))
    X = orc.rollout(x, U, P["dt"], P["mass"], P["g"])
    y = x.copy()
    for j in range(30):
        y = L.rk4(y, U[j], P["dt"], P["mass"], P["g"])
        assert np.abs(y - X[j + 1]).max() < 1e-12
    assert np.abs(L.rotation(q) - orc.rotation(q)).max() < 1e-15


def _surface_samples(scene, n=4000, rng=None):
    rng = rng or np.random.default_rng(0)
    out = []
    for (cx, cy, r, z0, z1) in scene.cylinders:
        th, z = rng.uniform(0, 2 * np.pi, n), rng.uniform(z0, z1, n)
        out.append(np.stack([cx + r * np.cos(th), cy + r * np.sin(th), z], 1))
        for zz in (z0, z1):   # caps
            rr, th = r * np.sqrt(rng.uniform(0, 1, n // 4)), rng.uniform(0, 2 * np.pi, n // 4)
            out.append(np.stack([cx + rr * np.cos(th), cy + rr * np.sin(th), np.full(n // 4, zz)], 1))
    for (c, a1, a2, s1, s2) in scene.rects:
        u, v = rng.uniform(-s1, s1, n), rng.uniform(-s2, s2, n)
        out.append(np.asarray(c) + u[:, None] * np.asarray(a1) + v[:, None] * np.asarray(a2))
    for c, r in scene.spheres:
        d = rng.normal(size=(n, 3))
        out.append(np.asarray(c) + r * d / np.linalg.norm(d, axis=1, keepdims=True))
    for lo, hi in scene.boxes:
        lo, hi = np.asarray(lo, float), np.asarray(hi, float)
        for ax in range(3):
            for side in (lo, hi):
                p = rng.uniform(lo, hi, (n // 6, 3))
                p[:, ax] = side[ax]
                out.append(p)
    return np.concatenate(out)


def test_scene_distance_against_sampled_surfaces():
    rng = np.random.default_rng(1)
    for scene in (I.scene_plain(0)[1], I.scene_walls(np.random.default_rng(2)),
                  I.scene_inclines(np.random.default_rng(3))):
        rects = [(c, a1, a2, min(s1, 3.0), min(s2, 3.0)) for (c, a1, a2, s1, s2) in scene.rects[:3]]
        scene = I.Scene(scene.cylinders[:6], scene.boxes[:4], rects, scene.spheres[:4], False)
        surf = _surface_samples(scene, rng=rng)
        q = rng.uniform(surf.min(0) - 2, surf.max(0) + 2, (300, 3))
        d = I.scene_distance(scene, q)
        brute = np.min(np.linalg.norm(q[:, None, :] - surf[None], axis=2), axis=1)
        outside = d > 0
        # the exact distance is a lower bound of the sampled one and close to it
        assert np.all(d[outside] <= brute[outside] + 1e-9)
        assert np.all(brute[outside] - d[outside] < 0.25)
    # the ground half-space
    g = I.Scene(ground=True)
    assert np.allclose(I.scene_distance(g, [[0, 0, 2.5], [1, 1, -1]]), [2.5, 0.0])
