"""The planner exactly as the benchmark creates it (no debug buffers, no
every-point collision set: the scatter pass empties the fine keys it reads, so
a step needs no key fill) against the FP64 oracle, end to end, over
consecutive steps on different clouds; and the full-size large clutter (E=32,
K=8192, T=64, 200,000 points) end to end against the oracle's whole planning
step.

Per step: coarse winners, goal cone and anchor cells bit-exact; anchors and
guides within 1e-4 m; every instance's update fed the GPU's own sample costs
within 1e-4 (Eq. mppi_update_simplified); the end-to-end nominal equal to the
oracle's plus the first-order shift its measured cost error predicts (as in
test_gpu_parity); S(2) within 1e-4 relative; the selected index equal (ties
within 1e-4 relative checked by membership)."""
import os

import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I
from gpu_util import TOL_COST_REL, TOL_POS, TOL_U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aero():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero as A
    return A


def _bench_planner(aero, P, n_points):
    """Created as bench.py creates its planners."""
    return aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                        fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=n_points,
                        raw_points_max=-1)


def _run(aero, pl, w, P, u0):
    import torch
    dev = torch.device("cuda")
    c = torch.from_numpy(np.ascontiguousarray(w.cloud, np.float32)).to(dev)
    un = torch.from_numpy(np.ascontiguousarray(u0, np.float32)).to(dev)
    u_best, cand, best = aero.plan_step(pl, w.p0, w.q0, w.v0, c, w.goal, P, un)
    torch.cuda.synchronize()
    assert pl.sync_status() == 0
    E, K, T = P["E"], P["K"], P["T"]
    p0 = w.p0.astype(np.float64)
    return dict(u_nom=un.cpu().numpy().astype(np.float64), u_best=u_best.cpu().numpy(),
                cand=cand.cpu().numpy().astype(np.float64), best=int(best.cpu().numpy()[0]),
                coarse=pl.debug("COARSE_WIN"), goal_cell=int(pl.debug("GOAL_CELL")[0]),
                anchor_cells=pl.debug("ANCHOR_CELLS"),
                anchors=pl.debug("ANCHORS")[:E * 3].reshape(E, 3) + p0,
                guides=pl.debug("GUIDES")[:E * T * 3].reshape(E, T, 3) + p0,
                S1=pl.debug("SAMPLE_COSTS")[:E * K].reshape(E, K).astype(np.float64))


def _check_step(orc, w, P, u0, g, o):
    win, _ = orc.coarse(o["keys"], P)
    assert np.array_equal(g["coarse"][:len(win)], win)
    gc = orc.goal_fine_cell(w.goal, w.p0, w.q0, P)
    assert g["goal_cell"] == gc
    assert np.array_equal(g["anchor_cells"][:P["E"]], orc.anchor_cells(gc, P))
    assert np.abs(g["anchors"] - o["anchors"]).max() < TOL_POS
    assert np.abs(g["guides"] - o["guides"]).max() < TOL_POS
    lo, hi = np.array(P["u_min"]), np.array(P["u_max"])
    lam = P["lam"]
    for e in range(P["E"]):
        d = orc.noise_range(P, e, 0, P["K"])
        un0 = u0[e].astype(np.float64)
        dU = (np.clip(un0 + d, lo, hi) - un0).reshape(P["K"], -1)
        # the update from the GPU's own costs
        u_ref, _ = orc.mppi_update(g["S1"][e], dU, lam, un0)
        assert np.abs(g["u_nom"][e] - u_ref).max() < TOL_U, e
        # end to end: the oracle's nominal plus the first-order shift of the cost error
        S = o["S1"][e]
        eps = np.exp(-(S - S.min()) / lam)
        eps /= eps.sum()
        dS = g["S1"][e] - S
        shift = (eps * (eps @ dS - dS) / lam) @ dU
        pred = o["u_nom"][e].reshape(-1) + shift
        assert np.abs(g["u_nom"][e].reshape(-1) - pred).max() < TOL_U, e
    assert np.all(np.abs(g["cand"] - o["cand"]) <= TOL_COST_REL * np.abs(o["cand"]))
    c = np.sort(o["cand"])
    if len(c) > 1 and (c[1] - c[0]) < TOL_COST_REL * abs(c[0]):
        assert o["cand"][g["best"]] <= c[0] * (1 + TOL_COST_REL)
    else:
        assert g["best"] == o["best"]
    assert np.array_equal(g["u_best"], g["u_nom"][g["best"]].astype(np.float32))


def _sequence():
    ens = I.make_workload("ensemble")
    plain = I.make_workload("plain")
    empty = I.make_workload("plain", seed=4)
    empty.cloud = np.zeros((0, 3), np.float32)
    empty.params.update(E=3, M_h=3, M_v=1, K=512, T=30)
    ens2 = I.make_workload("ensemble", seed=2)
    ens2.params["step_id"] = 9
    return [ens, plain, empty, ens2]


@pytest.mark.parametrize("lanes", [0, 1])
def test_bench_planner_consecutive_clouds_match_oracle(aero, orc, lanes):
    """One planner, created as the benchmark creates it for the ensemble, plans
    the ensemble scene, the plain scene, an empty cloud and another ensemble
    scene in a row: each step equals the oracle's step on its own inputs, so
    nothing of an earlier step (keys, counts, lists, the update launch's
    finished-CTA count and tickets, the warm-up scratch) leaks into the next.
    Both Stage I passes: the split pass these sizes select, and one lane per
    sample with its own update launch."""
    seq = _sequence()
    P0 = seq[0].params
    pl = _bench_planner(aero, P0, max(len(w.cloud) for w in seq))
    for w in seq:
        P = dict(w.params, lanes_per_sample=lanes)
        u0 = w.hover_nominal()
        g = _run(aero, pl, w, P, u0)
        o = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, u0)
        _check_step(orc, w, P, u0, g, o)
    pl.close()


def test_large_clutter_end_to_end(aero, orc):
    """The full-size large clutter (the benchmark's headline workload, in the
    launch configuration it times) against the oracle's whole planning step
    (OpenMP over the samples; results do not depend on the thread count)."""
    w = I.make_workload("large")
    P = w.params
    pl = _bench_planner(aero, P, len(w.cloud))
    u0 = w.hover_nominal()
    g = _run(aero, pl, w, P, u0)
    pl.close()
    orc.set_threads(os.cpu_count() or 1)
    try:
        o = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, u0)
    finally:
        orc.set_threads(1)
    _check_step(orc, w, P, u0, g, o)
