"""Seeded synthetic inputs: planner parameters and LiDAR-like point clouds.

This module is the only code shared by the CUDA path's tests/bench and the CPU
oracle.  It holds none of the planning method's arithmetic: it only builds
parameter dictionaries (the values of Table I of the paper and the workload
sizes) and synthetic scenes (ray-cast LiDAR sweeps or surface samples of
cylinders, walls, inclined planes and spheres), all from numpy's seeded PCG64
generator.

Scene shapes follow the paper's simulation scenes (Sec. V-B: forests of
cylinders, vertical obstacles, inclines) at the sizes of the benchmark
workloads:

* ``plain``     – 10 vertical cylinders, 2,000 surface points, single MPPI.
* ``ensemble``  – forest of 60 cylinders + ground, one 1024x32 LiDAR sweep.
* ``large``     – 60x60x10 m clutter, 3 merged sweeps resampled to 200,000 pts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

G = 9.81

# Table I (Sec. V-A): MPPI and AERO-MPPI parameters.  sigma holds standard
# deviations; Table I lists the covariance diagonal, so its std is sqrt(Sigma).
TABLE_I = dict(
    mass=1.0, g=G,
    u_min=[0.3, -3.0, -3.0, -2.0], u_max=[16.35, 3.0, 3.0, 2.0],
    sigma=[1.0, 1.0, 1.0, math.sqrt(0.5)],
    dt=0.05, K=128, T=25, lam=0.1,
    Q_p=3.0, Q_v=0.25, Q_q=1.0, Q_vnorm=0.15, Q_track=15.0, Q_c=0.5, Q_cd=0.5,
    ell=5.0, C_col=1.0e6, a_col=5.0, d_min=0.4, d_max=1.0,
)


def default_params() -> dict:
    """Planner parameters with Table I defaults and the paper's partition.

    Partition: 3 degree fine cells (120 x 60 over the full sphere), 6x6 pooling
    to 18 degree coarse cells (20 x 10), M_h x M_v = 5 x 3 anchors, r_max = 10 m
    (Sec. IV-A, Sec. V-A).
    """
    p = dict(TABLE_I)
    p.update(
        E=15, iters=1, v_end=0.0, r_max=10.0,
        fine_az=120, fine_el=60, pool_az=6, pool_el=6, M_h=5, M_v=3,
        el_lo=-math.pi / 2, el_hi=math.pi / 2,
        collision_set=0,
        v_goal=[0.0, 0.0, 0.0], q_goal=[1.0, 0.0, 0.0, 0.0],
        seed=0, step_id=0, debug_samples=0,
        refine_steps=0, refine_step=0.05,
    )
    return p


def workload_params(name: str) -> dict:
    """Parameters of the named benchmark workload.

    plain    : E=1, K=256, T=20, dt=0.05, lambda=1, sigma=(2,1.5,1.5,1.5),
               thrust in [0, 2g], rates in [-6, 6]; no guide tracking.
    ensemble : E=8 (4x2 anchors), K=1024, T=40, dt=0.05, fine 128x64 pooled
               8x16 to a 16x4 coarse grid.
    large    : E=32 (8x4 anchors), K=8192, T=64, dt=0.03, fine 256x64 pooled
               4x8 to a 64x8 coarse grid, r_max=20 m.
    refined  : the ensemble sizes with 5 gradient-refinement steps of 0.05 on
               every updated nominal before Stage II (on the plain scene).
    """
    p = default_params()
    common = dict(lam=1.0, sigma=[2.0, 1.5, 1.5, 1.5],
                  u_min=[0.0, -6.0, -6.0, -6.0], u_max=[2 * G, 6.0, 6.0, 6.0])
    if name == "plain":
        p.update(common)
        p.update(E=1, K=256, T=20, dt=0.05, M_h=1, M_v=1, Q_track=0.0)
    elif name == "ensemble":
        p.update(common)
        p.update(E=8, K=1024, T=40, dt=0.05, fine_az=128, fine_el=64,
                 pool_az=8, pool_el=16, M_h=4, M_v=2)
    elif name == "large":
        p.update(common)
        p.update(E=32, K=8192, T=64, dt=0.03, fine_az=256, fine_el=64,
                 pool_az=4, pool_el=8, M_h=8, M_v=4, r_max=20.0)
    elif name == "refined":
        p.update(common)
        p.update(E=8, K=1024, T=40, dt=0.05, fine_az=128, fine_el=64,
                 pool_az=8, pool_el=16, M_h=4, M_v=2, refine_steps=5, refine_step=0.05)
    else:
        raise KeyError(name)
    return p


# --------------------------------------------------------------------------
# Scene primitives and ray casting (input synthesis only)
# --------------------------------------------------------------------------

@dataclass
class Scene:
    cylinders: list = field(default_factory=list)   # (cx, cy, r, z0, z1)
    boxes: list = field(default_factory=list)       # (lo[3], hi[3])
    rects: list = field(default_factory=list)       # (centre[3], a1[3], a2[3], s1, s2)
    spheres: list = field(default_factory=list)     # (centre[3], r)
    ground: bool = False


def _hit_cylinders(o, d, cyls, t_best):
    for (cx, cy, r, z0, z1) in cyls:
        ox, oy = o[0] - cx, o[1] - cy
        a = d[:, 0] ** 2 + d[:, 1] ** 2
        b = 2 * (ox * d[:, 0] + oy * d[:, 1])
        c = ox * ox + oy * oy - r * r
        disc = b * b - 4 * a * c
        ok = (disc >= 0) & (a > 1e-12)
        with np.errstate(invalid="ignore", divide="ignore"):
            t = (-b - np.sqrt(np.where(ok, disc, 0))) / (2 * a)
        z = o[2] + t * d[:, 2]
        ok &= (t > 1e-6) & (z >= z0) & (z <= z1)
        np.minimum(t_best, np.where(ok, t, np.inf), out=t_best)


def _hit_ground(o, d, t_best):
    with np.errstate(invalid="ignore", divide="ignore"):
        t = -o[2] / d[:, 2]
    ok = (d[:, 2] < 0) & (t > 1e-6)
    np.minimum(t_best, np.where(ok, t, np.inf), out=t_best)


def _hit_boxes(o, d, boxes, t_best):
    for lo, hi in boxes:
        lo, hi = np.asarray(lo), np.asarray(hi)
        with np.errstate(invalid="ignore", divide="ignore"):
            inv = 1.0 / d
            t0 = (lo - o) * inv
            t1 = (hi - o) * inv
        tmin = np.nanmax(np.minimum(t0, t1), axis=1)
        tmax = np.nanmin(np.maximum(t0, t1), axis=1)
        ok = (tmax >= tmin) & (tmin > 1e-6)
        np.minimum(t_best, np.where(ok, tmin, np.inf), out=t_best)


def _hit_rects(o, d, rects, t_best):
    for (c, a1, a2, s1, s2) in rects:
        c, a1, a2 = (np.asarray(v, dtype=np.float64) for v in (c, a1, a2))
        n = np.cross(a1, a2)
        dn = d @ n
        with np.errstate(invalid="ignore", divide="ignore"):
            t = ((c - o) @ n) / dn
        h = o + t[:, None] * d - c
        ok = (np.abs(dn) > 1e-12) & (t > 1e-6) & (np.abs(h @ a1) <= s1) & (np.abs(h @ a2) <= s2)
        np.minimum(t_best, np.where(ok, t, np.inf), out=t_best)


def _hit_spheres(o, d, spheres, t_best):
    for c, r in spheres:
        oc = o - np.asarray(c)
        b = d @ oc
        cc = oc @ oc - r * r
        disc = b * b - cc
        ok = disc >= 0
        t = -b - np.sqrt(np.where(ok, disc, 0))
        ok &= t > 1e-6
        np.minimum(t_best, np.where(ok, t, np.inf), out=t_best)


def scene_distance(scene: Scene, p) -> np.ndarray:
    """Exact distance from points p (M x 3) to the scene's solid primitives
    (cylinders, boxes, spheres, the ground half-space z <= 0) and surfaces
    (rectangles); zero inside a solid.  Clearance of a simulated flight."""
    p = np.atleast_2d(np.asarray(p, np.float64))
    d = np.full(len(p), np.inf)
    for (cx, cy, r, z0, z1) in scene.cylinders:
        dr = np.maximum(np.hypot(p[:, 0] - cx, p[:, 1] - cy) - r, 0.0)
        dz = np.maximum(np.maximum(z0 - p[:, 2], p[:, 2] - z1), 0.0)
        np.minimum(d, np.hypot(dr, dz), out=d)
    if scene.ground:
        np.minimum(d, np.maximum(p[:, 2], 0.0), out=d)
    for lo, hi in scene.boxes:
        e = np.maximum(np.maximum(np.asarray(lo) - p, p - np.asarray(hi)), 0.0)
        np.minimum(d, np.linalg.norm(e, axis=1), out=d)
    for (c, a1, a2, s1, s2) in scene.rects:
        c, a1, a2 = (np.asarray(v, dtype=np.float64) for v in (c, a1, a2))
        h = p - c
        u, v, w = h @ a1, h @ a2, h @ np.cross(a1, a2)
        du, dv = u - np.clip(u, -s1, s1), v - np.clip(v, -s2, s2)
        np.minimum(d, np.sqrt(du * du + dv * dv + w * w), out=d)
    for c, r in scene.spheres:
        np.minimum(d, np.maximum(np.linalg.norm(p - np.asarray(c), axis=1) - r, 0.0), out=d)
    return d


def lidar_sweep(scene: Scene, origin, n_az: int, n_el: int, el_min_deg: float,
                el_max_deg: float, max_range: float, range_sigma: float,
                rng: np.random.Generator, chunk: int = 8192) -> np.ndarray:
    """Ray-cast one 360 degree sweep; returns the hit points (float64, Mx3)."""
    o = np.asarray(origin, dtype=np.float64)
    az = np.arange(n_az) * (2 * np.pi / n_az)
    el = np.deg2rad(np.linspace(el_min_deg, el_max_deg, n_el))
    A, B = np.meshgrid(az, el, indexing="ij")
    dirs = np.stack([np.cos(B) * np.cos(A), np.cos(B) * np.sin(A), np.sin(B)], -1).reshape(-1, 3)
    out = []
    for s in range(0, len(dirs), chunk):
        d = dirs[s:s + chunk]
        t = np.full(len(d), np.inf)
        _hit_cylinders(o, d, scene.cylinders, t)
        if scene.ground:
            _hit_ground(o, d, t)
        _hit_boxes(o, d, scene.boxes, t)
        _hit_rects(o, d, scene.rects, t)
        _hit_spheres(o, d, scene.spheres, t)
        ok = t <= max_range
        tt = t[ok] + rng.normal(0.0, range_sigma, size=int(ok.sum()))
        out.append(o + tt[:, None] * d[ok])
    return np.concatenate(out, 0) if out else np.zeros((0, 3))


def _forest(rng, n, half, r_lo, r_hi, h, keep_out, centre=(0.0, 0.0)):
    cyl = []
    while len(cyl) < n:
        cx = rng.uniform(centre[0] - half, centre[0] + half)
        cy = rng.uniform(centre[1] - half, centre[1] + half)
        r = rng.uniform(r_lo, r_hi)
        if any(math.hypot(cx - kx, cy - ky) < r + kr for (kx, ky, kr) in keep_out):
            continue
        cyl.append((cx, cy, r, 0.0, h))
    return cyl


@dataclass
class Workload:
    name: str
    params: dict
    cloud: np.ndarray       # float32 N x 3, world frame
    p0: np.ndarray          # float32 3
    q0: np.ndarray          # float32 4 (w, x, y, z)
    v0: np.ndarray          # float32 3
    goal: np.ndarray        # float32 3
    note: str = ""

    def hover_nominal(self) -> np.ndarray:
        """Warm start u_nom = hover thrust, zero body rates (E x T x 4, float32)."""
        p = self.params
        u = np.zeros((p["E"], p["T"], 4), np.float32)
        u[..., 0] = p["mass"] * p["g"]
        return u


def scene_plain(seed: int = 0) -> tuple[np.ndarray, Scene]:
    """10 vertical cylinders (r ~ U(0.2,0.5) m, h = 5 m, x ~ U(0,20), y ~ U(-10,10)),
    200 surface points each (theta ~ U(0, 2pi), z ~ U(0, 5))."""
    rng = np.random.default_rng(seed)
    keep = [(0.0, 0.0, 1.5), (18.0, 0.0, 1.5)]
    cyl = []
    while len(cyl) < 10:
        cx, cy, r = rng.uniform(0, 20), rng.uniform(-10, 10), rng.uniform(0.2, 0.5)
        if any(math.hypot(cx - a, cy - b) < r + k for (a, b, k) in keep):
            continue
        cyl.append((cx, cy, r, 0.0, 5.0))
    pts = []
    for (cx, cy, r, _, h) in cyl:
        th = rng.uniform(0, 2 * np.pi, 200)
        z = rng.uniform(0, h, 200)
        pts.append(np.stack([cx + r * np.cos(th), cy + r * np.sin(th), z], 1))
    return np.concatenate(pts, 0), Scene(cylinders=cyl)


def scene_ensemble(seed: int = 0) -> tuple[np.ndarray, Scene]:
    """Forest: 60 cylinders r ~ U(0.2,0.5) m, h = 6 m, in a 40x40 m square centred
    at the start, plus ground; one LiDAR sweep at (0,0,1.5): 1024 azimuths x 32
    beams over +-15 deg, range <= 30 m, N(0, 0.02 m) range noise."""
    rng = np.random.default_rng(seed)
    cyl = _forest(rng, 60, 20.0, 0.2, 0.5, 6.0, keep_out=[(0.0, 0.0, 2.0), (18.0, 0.0, 1.5)])
    sc = Scene(cylinders=cyl, ground=True)
    pts = lidar_sweep(sc, (0.0, 0.0, 1.5), 1024, 32, -15.0, 15.0, 30.0, 0.02, rng)
    return pts, sc


def scene_large(seed: int = 0) -> tuple[np.ndarray, Scene]:
    """60x60x10 m clutter centred at x=20: 300 thin cylinders (r 0.1-0.3 m, h 10 m),
    8 vertical wall slabs, 4 inclined planes (10-25 deg), ground.  Three sweeps
    (1800 az x 64 beams, +-30 deg, range <= 40 m) from x = 0, 3, 6 m, merged and
    resampled to exactly 200,000 points."""
    rng = np.random.default_rng(seed)
    keep = [(x, 0.0, 1.5) for x in (0.0, 3.0, 6.0)]
    cyl = _forest(rng, 300, 30.0, 0.1, 0.3, 10.0, keep_out=keep, centre=(20.0, 0.0))
    boxes = []
    for _ in range(8):
        cx, cy = rng.uniform(12, 48), rng.uniform(-25, 25)
        L, H = rng.uniform(4, 8), rng.uniform(3, 8)
        if rng.uniform() < 0.5:
            boxes.append(([cx - 0.15, cy - L / 2, 0.0], [cx + 0.15, cy + L / 2, H]))
        else:
            boxes.append(([cx - L / 2, cy - 0.15, 0.0], [cx + L / 2, cy + 0.15, H]))
    rects = []
    for _ in range(4):
        cx, cy = rng.uniform(15, 45), rng.uniform(-25, 25)
        tilt = np.deg2rad(rng.uniform(10, 25))
        yaw = rng.uniform(0, 2 * np.pi)
        a1 = np.array([np.cos(yaw) * np.cos(tilt), np.sin(yaw) * np.cos(tilt), np.sin(tilt)])
        a2 = np.array([-np.sin(yaw), np.cos(yaw), 0.0])
        s1, s2 = rng.uniform(3, 6), rng.uniform(3, 6)
        c = np.array([cx, cy, s1 * np.sin(tilt)])
        rects.append((c, a1, a2, s1, s2))
    sc = Scene(cylinders=cyl, boxes=boxes, rects=rects, ground=True)
    sweeps = [lidar_sweep(sc, (x, 0.0, 2.0), 1800, 64, -30.0, 30.0, 40.0, 0.02, rng)
              for x in (0.0, 3.0, 6.0)]
    pts = np.concatenate(sweeps, 0)
    n = 200_000
    idx = rng.choice(len(pts), size=n, replace=len(pts) < n)
    return pts[idx], sc


def scene_walls(rng: np.random.Generator) -> Scene:
    """Three rows of 6 m walls across the flight direction (x = 6, 12, 18 m),
    each spanning y in [-15, 15] with three 1.5 m gaps at random places, plus
    ground and a few cylinders."""
    boxes = []
    for x in (6.0, 12.0, 18.0):
        gaps = np.sort(rng.uniform(-13, 13, 3))
        y = -15.0
        for gy in gaps:
            if gy - 0.75 > y:
                boxes.append(([x - 0.15, y, 0.0], [x + 0.15, gy - 0.75, 6.0]))
            y = max(y, gy + 0.75)
        if y < 15.0:
            boxes.append(([x - 0.15, y, 0.0], [x + 0.15, 15.0, 6.0]))
    cyl = _forest(rng, 10, 15.0, 0.2, 0.5, 6.0, keep_out=[(0.0, 0.0, 2.0)], centre=(10.0, 0.0))
    return Scene(cylinders=cyl, boxes=boxes, ground=True)


def scene_inclines(rng: np.random.Generator) -> Scene:
    """Ground tilted by 10-25 degrees under the flight path, plus spherical
    boulders (r 0.3-1.0 m) and a few inclined slabs."""
    tilt = np.deg2rad(rng.uniform(10, 25))
    yaw = rng.uniform(0, 2 * np.pi)
    a1 = np.array([np.cos(yaw) * np.cos(tilt), np.sin(yaw) * np.cos(tilt), np.sin(tilt)])
    a2 = np.array([-np.sin(yaw), np.cos(yaw), 0.0])
    rects = [(np.array([10.0, 0.0, -2.0]), a1, a2, 25.0, 25.0)]
    for _ in range(3):
        t2 = np.deg2rad(rng.uniform(10, 25))
        y2 = rng.uniform(0, 2 * np.pi)
        b1 = np.array([np.cos(y2) * np.cos(t2), np.sin(y2) * np.cos(t2), np.sin(t2)])
        b2 = np.array([-np.sin(y2), np.cos(y2), 0.0])
        rects.append((np.array([rng.uniform(5, 20), rng.uniform(-8, 8), 2.0]), b1, b2,
                      rng.uniform(2, 4), rng.uniform(2, 4)))
    spheres = []
    while len(spheres) < 25:
        c = np.array([rng.uniform(2, 25), rng.uniform(-12, 12), rng.uniform(0.5, 4.0)])
        r = rng.uniform(0.3, 1.0)
        if np.linalg.norm(c - [0, 0, 2.0]) > r + 2.0:
            spheres.append((c, r))
    return Scene(rects=rects, spheres=spheres)


BATCH_E = {4: (2, 2), 8: (4, 2), 16: (4, 4)}


def batch_workloads(n: int = 64, seed: int = 1) -> list:
    """Independent planners of uneven sizes: E in {4, 8, 16}, K in {256, 1024,
    4096}, T in {20, 40, 60}; scene forest / walls with 1.5 m gaps / inclines
    with boulders; 5k-100k points (log-uniform) from a 1024 x 32 LiDAR sweep at
    (0, 0, 2), resampled to the drawn size.  All sizes from `seed`."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        E = int(rng.choice([4, 8, 16]))
        K = int(rng.choice([256, 1024, 4096]))
        T = int(rng.choice([20, 40, 60]))
        kind = ["forest", "walls", "inclines"][int(rng.integers(3))]
        npts = int(np.exp(rng.uniform(np.log(5000), np.log(100000))))
        srng = np.random.default_rng([seed, i])
        if kind == "forest":
            sc = Scene(cylinders=_forest(srng, 60, 20.0, 0.2, 0.5, 6.0, keep_out=[(0.0, 0.0, 2.0)]),
                       ground=True)
        elif kind == "walls":
            sc = scene_walls(srng)
        else:
            sc = scene_inclines(srng)
        pts = lidar_sweep(sc, (0.0, 0.0, 2.0), 1024, 32, -15.0, 15.0, 30.0, 0.02, srng)
        if len(pts) == 0:
            pts = np.zeros((1, 3)) + [20.0, 0.0, 2.0]
        pts = pts[srng.choice(len(pts), size=npts, replace=len(pts) < npts)]
        p = workload_params("ensemble")
        Mh, Mv = BATCH_E[E]
        p.update(E=E, M_h=Mh, M_v=Mv, K=K, T=T, seed=seed * 1000 + i)
        w = Workload(f"batch{i}:{kind}", p, np.ascontiguousarray(pts, np.float32),
                     np.array([0, 0, 2], np.float32), np.array([1, 0, 0, 0], np.float32),
                     np.array([rng.uniform(0, 3), 0, 0], np.float32),
                     np.array([25, rng.uniform(-5, 5), 2], np.float32), note=kind)
        out.append(w)
    return out


def make_workload(name: str, seed: int = 0) -> Workload:
    """Build the named workload (params + scene + start state + goal)."""
    p = workload_params(name)
    p["seed"] = seed
    q0 = np.array([1, 0, 0, 0], np.float32)
    if name in ("plain", "refined"):
        pts, _ = scene_plain(seed)
        p0, v0, goal = (0, 0, 1.5), (0, 0, 0), (18, 0, 1.5)
    elif name == "ensemble":
        pts, _ = scene_ensemble(seed)
        p0, v0, goal = (0, 0, 1.5), (0, 0, 0), (18, 0, 1.5)
    elif name == "large":
        pts, _ = scene_large(seed)
        rng = np.random.default_rng(seed + 1000)
        p0, v0, goal = (6, 0, 2), (rng.uniform(7, 10), 0, 0), (56, 0, 2)
    else:
        raise KeyError(name)
    return Workload(name, p, np.ascontiguousarray(pts, np.float32),
                    np.array(p0, np.float32), q0, np.array(v0, np.float32),
                    np.array(goal, np.float32))


def random_cloud(n: int, seed: int, centre=(0.0, 0.0, 1.5), spread: float = 8.0) -> np.ndarray:
    """Uniform random points in a cube (small parity cases and edge cases)."""
    rng = np.random.default_rng(seed)
    return (np.asarray(centre) + rng.uniform(-spread, spread, size=(n, 3))).astype(np.float32)


def random_unit_quaternion(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    if q[0] < 0:
        q = -q
    return q.astype(np.float32)
