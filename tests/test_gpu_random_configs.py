"""Seeded random planning steps against the FP64 oracle: ragged sample
counts, horizons from 1 step, uneven anchor grids and partitions, both
collision sets, both Stage I passes (and the automatic choice), random start
attitudes and velocities, goals at rest and moving, clouds from empty to a few thousand points with the
start anywhere in them.  One planner (no debug buffers, room for the
every-point set) plans them all in a row, so nothing of one step may leak into
the next.  Checked per step: the partition's decisions and the anchor cells
exactly, anchors and guides within 1e-4 m; every sample's S(1) within 1e-4
relative but for at most 1% (the samples on a jump of J_col); each instance's
update fed the GPU's own sample costs within 1e-4; Stage II of the GPU's own
nominals (states and S(2) against the oracle's rollout and cost of them) and
the selection.  Inside a dense cloud the costs reach 1e7 with lambda = 1, where
FP32's rounding of S(1) alone moves the softmax weights, so the end-to-end
nominal is compared through the update from the GPU's costs, not against the
oracle's nominal."""
import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I
from gpu_util import JUMP_BAND, TOL_COST_REL, TOL_POS, TOL_QUAT, TOL_U
from test_gpu_bench_planner import _run

pytestmark = pytest.mark.gpu

N_CASES = 24


@pytest.fixture(scope="module")
def aero():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero as A
    return A


def _divisors(n, choices):
    return [d for d in choices if n % d == 0]


def random_case(i: int) -> I.Workload:
    rng = np.random.default_rng(9000 + i)
    p = I.workload_params("plain")
    M_h, M_v = int(rng.integers(1, 5)), int(rng.integers(1, 3))
    fine_az = int(rng.choice([24, 48, 64, 120]))
    fine_el = int(rng.choice([8, 16, 30]))
    pool_az = int(rng.choice(_divisors(fine_az, [2, 3, 4, 6, 8])))
    pool_el = int(rng.choice(_divisors(fine_el, [2, 4, 5, 8])))
    p.update(E=M_h * M_v, M_h=M_h, M_v=M_v, K=int(rng.integers(20, 700)),
             T=int(rng.integers(1, 49)), fine_az=fine_az, fine_el=fine_el, pool_az=pool_az,
             pool_el=pool_el, lanes_per_sample=int(rng.choice([0, 1, 4])),
             collision_set=int(rng.integers(0, 2)), Q_track=float(rng.choice([0.0, 15.0])),
             seed=int(rng.integers(1, 1 << 40)), step_id=int(rng.integers(0, 1000)))
    n = int(rng.choice([0, 40, 900, 4000]))
    if i % 3 == 1:  # a goal with a velocity and an attitude (drawn apart: the rest stays)
        grng = np.random.default_rng(9500 + i)
        p.update(v_goal=[float(v) for v in grng.uniform(-2.0, 2.0, 3)],
                 q_goal=[float(v) for v in I.random_unit_quaternion(grng)])
        if i % 9 == 4:
            p.update(lanes_per_sample=1)
    if i % 6 == 0:  # the every-point set with one lane per sample, a dense cloud
        p.update(collision_set=1, lanes_per_sample=1)
        n = 4000
    cloud = I.random_cloud(n, 9100 + i, spread=float(rng.uniform(2.0, 9.0)))
    p0 = rng.uniform(-1.5, 1.5, 3).astype(np.float32) + np.array([0, 0, 1.5], np.float32)
    q0 = I.random_unit_quaternion(rng)
    v0 = rng.uniform(-2.0, 2.0, 3).astype(np.float32)
    goal = np.array([rng.uniform(5, 20), rng.uniform(-6, 6), rng.uniform(0.5, 3)], np.float32)
    return I.Workload(f"random{i}", p, cloud, p0, q0, v0, goal)


def _check(orc, w, P, u0, g, o):
    win, _ = orc.coarse(o["keys"], P)
    assert np.array_equal(g["coarse"][:len(win)], win)
    gc = orc.goal_fine_cell(w.goal, w.p0, w.q0, P)
    assert g["goal_cell"] == gc
    assert np.array_equal(g["anchor_cells"][:P["E"]], orc.anchor_cells(gc, P))
    assert np.abs(g["anchors"] - o["anchors"]).max() < TOL_POS
    assert np.abs(g["guides"] - o["guides"]).max() < TOL_POS
    off = np.abs(g["S1"] - o["S1"]) > TOL_COST_REL * np.abs(o["S1"])
    assert off.mean() <= 0.01, int(off.sum())
    lo, hi = np.array(P["u_min"]), np.array(P["u_max"])
    for e in range(P["E"]):
        d = orc.noise_range(P, e, 0, P["K"])
        un0 = u0[e].astype(np.float64)
        dU = (np.clip(un0 + d, lo, hi) - un0).reshape(P["K"], -1)
        u_ref, _ = orc.mppi_update(g["S1"][e], dU, P["lam"], un0)
        assert np.abs(g["u_nom"][e] - u_ref).max() < TOL_U, e
    pts = orc.collision_set(w.cloud, w.p0, w.q0, o["keys"], P)
    x0 = np.concatenate([w.p0, w.q0, w.v0]).astype(np.float64)
    for e in range(P["E"]):
        X = orc.rollout(x0, g["u_nom"][e], P["dt"], P["mass"], P["g"])
        t = orc.cost_terms(X, g["u_nom"][e], None, w.goal.astype(np.float64), pts, P, stage=2,
                           want_dist=True)
        jump = np.min(np.minimum(np.abs(t["dist"] - P["d_min"]), np.abs(t["dist"] - P["d_max"])))
        if jump > JUMP_BAND:
            assert abs(g["cand"][e] - t["S"]) <= TOL_COST_REL * abs(t["S"]), e
    cand = g["cand"]
    c = np.sort(cand)
    if len(c) > 1 and (c[1] - c[0]) < TOL_COST_REL * abs(c[0]):
        assert cand[g["best"]] <= c[0] * (1 + TOL_COST_REL)
    else:
        assert g["best"] == int(np.argmin(cand))
    assert np.array_equal(g["u_best"], g["u_nom"][g["best"]].astype(np.float32))


def test_random_steps_match_oracle(aero, orc):
    cases = [random_case(i) for i in range(N_CASES)]
    assert {c.params["lanes_per_sample"] for c in cases} == {0, 1, 4}
    assert {c.params["collision_set"] for c in cases} == {0, 1}
    n_max = max(1, max(len(c.cloud) for c in cases))
    pl = aero.Planner(E_max=8, K_max=700, T_max=48, fine_cells_max=120 * 30, n_points_max=n_max,
                      raw_points_max=0)
    for w in cases:
        P = w.params
        u0 = w.hover_nominal()
        g = _run(aero, pl, w, P, u0)
        o = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, u0)
        _check(orc, w, P, u0, g, o)
    pl.close()
