"""Receding-horizon flight on synthetic scenes (Sec. III-B receding horizon,
Sec. IV-A.1 accumulation, Sec. V-C.1 replanning rates).

Every planning cycle: a LiDAR sweep is ray-cast from the drone's true pose
(CPU), expressed in the sensor frame and pushed into the GPU accumulator; the
planner plans on the accumulated ring from the true state; the first
`round(1 / (plan_hz dt))` controls of the selected sequence drive a CPU
simulation of the quadrotor model (Eq. dynamics, RK4 at the planner's dt,
float64); the nominals are shifted by the executed steps on the GPU (warm
start) and the next cycle draws new noise (step_id).  A flight ends at the goal
(within goal_radius), on a collision (clearance below drone_radius) or at
max_time.  Synthetic scenes stand in for the paper's simulators.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I


@dataclass
class LoopConfig:
    plan_hz: float = 10.0        # replanning rate (the hardware experiments replan at 10 Hz)
    frames: int = 10             # accumulated sweeps (Sec. IV-A.1)
    sweep_az: int = 512
    sweep_el: int = 36
    el_min_deg: float = -60.0    # down-looking enough to see the ground under the drone
    el_max_deg: float = 30.0
    max_range: float = 30.0
    range_sigma: float = 0.02
    max_time: float = 15.0
    goal_radius: float = 1.0
    drone_radius: float = 0.25


@dataclass
class FlightResult:
    success: bool
    crashed: bool
    time: float
    path_length: float
    min_clearance: float
    mean_speed: float
    cycles: int
    plan_ms: list = field(default_factory=list)
    sense_ms: list = field(default_factory=list)
    positions: np.ndarray | None = None

    def summary(self) -> dict:
        return {"success": self.success, "crashed": self.crashed, "time_s": round(self.time, 3),
                "path_m": round(self.path_length, 3), "min_clearance_m": round(self.min_clearance, 3),
                "mean_speed_mps": round(self.mean_speed, 3), "cycles": self.cycles,
                "plan_ms_median": round(float(np.median(self.plan_ms)), 4) if self.plan_ms else None,
                "sense_ms_median": round(float(np.median(self.sense_ms)), 2) if self.sense_ms else None}


# ---------------------------------------------------------------------------
# The simulated quadrotor (Eq. dynamics), float64
# ---------------------------------------------------------------------------

def rotation(q) -> np.ndarray:
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def dynamics(x, u, m, g) -> np.ndarray:
    """x = (p, q, v), u = (F, w): p' = v, q' = 1/2 q (x) [0, w], v' = R(q)[0, 0, F]/m - g e3."""
    q, v = x[3:7], x[7:10]
    w, wx, wy, wz = q[0], u[1], u[2], u[3]
    qd = 0.5 * np.array([-q[1] * wx - q[2] * wy - q[3] * wz,
                         w * wx + q[2] * wz - q[3] * wy,
                         w * wy - q[1] * wz + q[3] * wx,
                         w * wz + q[1] * wy - q[2] * wx])
    a = rotation(q)[:, 2] * (u[0] / m) - np.array([0.0, 0.0, g])
    return np.concatenate([v, qd, a])


def rk4(x, u, dt, m, g) -> np.ndarray:
    k1 = dynamics(x, u, m, g)
    k2 = dynamics(x + 0.5 * dt * k1, u, m, g)
    k3 = dynamics(x + 0.5 * dt * k2, u, m, g)
    k4 = dynamics(x + dt * k3, u, m, g)
    xn = x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    xn[3:7] /= np.linalg.norm(xn[3:7])
    return xn


# ---------------------------------------------------------------------------
# The loop
# ---------------------------------------------------------------------------

def fly(scene: I.Scene, params: dict, start, goal, cfg: LoopConfig = LoopConfig(), v0=(0, 0, 0),
        seed: int = 0, planner=None, accumulator=None) -> FlightResult:
    """Fly from `start` to `goal` through `scene` with the GPU planner."""
    import torch

    from . import aero
    P = dict(params)
    E, K, T, dt = P["E"], P["K"], P["T"], P["dt"]
    m_exec = max(1, int(round(1.0 / (cfg.plan_hz * dt))))
    n_sweep = cfg.sweep_az * cfg.sweep_el
    own_pl, own_acc = planner is None, accumulator is None
    if own_pl:
        planner = aero.Planner(E_max=E, K_max=K, T_max=T, fine_cells_max=P["fine_az"] * P["fine_el"],
                               n_points_max=cfg.frames * n_sweep)
    if own_acc:
        accumulator = aero.Accumulator(cfg.frames, n_sweep)
    rng = np.random.default_rng(seed)
    dev = torch.device("cuda")
    x = np.concatenate([np.asarray(start, np.float64), [1.0, 0.0, 0.0, 0.0], np.asarray(v0, np.float64)])
    goal = np.asarray(goal, np.float32)
    hover = np.tile(np.array([P["mass"] * P["g"], 0.0, 0.0, 0.0], np.float32), (E, T, 1))
    un = torch.from_numpy(hover).to(dev)
    scratch = torch.empty_like(un)
    ub = torch.empty((T, 4), device=dev)
    cand = torch.empty((E,), device=dev)
    best = torch.empty((1,), dtype=torch.int32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = FlightResult(False, False, 0.0, 0.0, math.inf, 0.0, 0)
    positions = [x[:3].copy()]
    t_sim = 0.0
    max_cycles = int(math.ceil(cfg.max_time * cfg.plan_hz))
    for cycle in range(max_cycles):
        # sense: one sweep from the true pose, in the sensor frame, into the ring
        t0 = time.perf_counter()
        pw = I.lidar_sweep(scene, x[:3], cfg.sweep_az, cfg.sweep_el, cfg.el_min_deg, cfg.el_max_deg,
                           cfg.max_range, cfg.range_sigma, rng)
        ps = ((pw - x[:3]) @ rotation(x[3:7])).astype(np.float32)
        accumulator.push(torch.from_numpy(np.ascontiguousarray(ps)).to(dev), x[:3], x[3:7])
        res.sense_ms.append(1e3 * (time.perf_counter() - t0))
        # plan on the accumulated frames from the true state
        ring, _ = accumulator.view()
        P["step_id"] = cycle
        state = aero.state_struct(x[:3].astype(np.float32), x[3:7].astype(np.float32),
                                  x[7:10].astype(np.float32))
        ev0.record()
        planner.plan_step(state, ring, goal, aero.params_struct(P), un, ub, cand, best)
        ev1.record()
        u_exec = ub.cpu().numpy().astype(np.float64)       # synchronises
        res.plan_ms.append(ev0.elapsed_time(ev1))
        # execute the first controls on the simulated drone
        for j in range(m_exec):
            x = rk4(x, u_exec[min(j, T - 1)], dt, P["mass"], P["g"])
            t_sim += dt
            positions.append(x[:3].copy())
            clear = float(I.scene_distance(scene, x[:3])[0])
            res.min_clearance = min(res.min_clearance, clear)
            if clear < cfg.drone_radius:
                res.crashed = True
                break
            if np.linalg.norm(x[:3] - goal) < cfg.goal_radius:
                res.success = True
                break
        res.cycles = cycle + 1
        if res.crashed or res.success:
            break
        # warm start for the next cycle
        aero.shift_nominal(un, m_exec, scratch)
    pos = np.array(positions)
    res.positions = pos
    res.time = t_sim
    res.path_length = float(np.linalg.norm(np.diff(pos, axis=0), axis=1).sum())
    res.mean_speed = res.path_length / t_sim if t_sim > 0 else 0.0
    if own_pl:
        planner.close()
    if own_acc:
        accumulator.close()
    return res


def scenario(kind: str, seed: int, cfg: LoopConfig = LoopConfig()):
    """A scene, start, goal and workload parameters for a closed-loop flight.

    The partition covers the whole sphere in 3 degree cones, so accumulated
    points below the sweep's field of view (the ground the drone flies over)
    still enter the collision set; its coarse rows are 15 degrees and the
    anchors take the two rows around the goal's elevation, which the sweep
    (-60 to +30 degrees) observes: an unobserved cone is empty (range r_max) and would
    pass for free space as an anchor direction.  Q_c is 0.02 instead of Table
    I's 0.5: on |u|^2 with the thrust in m/s^2 the Table I weight makes hovering
    cost about 48 per step, more than any progress term, so a planner that
    cannot advance would rather cut the thrust and fall."""
    rng = np.random.default_rng(seed)
    P = I.workload_params("ensemble")
    P.update(K=512, T=30, seed=seed, E=8, M_h=4, M_v=2, fine_az=120, pool_az=6,
             fine_el=60, pool_el=5, el_lo=-math.pi / 2, el_hi=math.pi / 2, Q_c=0.02)
    if kind == "forest":
        _, scene = I.scene_ensemble(seed)
        start, goal = (0.0, 0.0, 1.5), (18.0, 0.0, 1.5)
    elif kind == "walls":
        scene = I.scene_walls(rng)
        start, goal = (0.0, 0.0, 2.0), (24.0, 0.0, 2.0)
    elif kind == "inclines":
        scene = I.scene_inclines(rng)
        start, goal = (0.0, 0.0, 2.5), (25.0, 0.0, 2.5)
    else:
        raise KeyError(kind)
    return scene, P, start, goal


def main():
    ap = argparse.ArgumentParser(description="closed-loop flights on synthetic scenes")
    ap.add_argument("--kind", default="forest", choices=["forest", "walls", "inclines"])
    ap.add_argument("--flights", type=int, default=4)
    ap.add_argument("--iters", type=int, default=1)
    ap.add_argument("--max-time", type=float, default=15.0)
    args = ap.parse_args()
    from . import build
    build.build()
    out = []
    for s in range(args.flights):
        scene, P, start, goal = scenario(args.kind, s)
        P["iters"] = args.iters
        r = fly(scene, P, start, goal, LoopConfig(max_time=args.max_time), seed=s)
        out.append(dict(r.summary(), seed=s))
        print(json.dumps(out[-1]), flush=True)
    ok = [o for o in out if o["success"]]
    print(json.dumps({"kind": args.kind, "flights": len(out), "success": len(ok),
                      "crashes": sum(o["crashed"] for o in out),
                      "min_clearance_m": min(o["min_clearance_m"] for o in out),
                      "mean_time_s": float(np.mean([o["time_s"] for o in ok])) if ok else None}))


if __name__ == "__main__":
    main()
