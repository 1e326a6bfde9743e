"""Batched planning (aero_batch_plan): one launch per stage over the work units of
many planners.  Every slot is checked against a separate aero_plan_step from
the same nominal (integer decisions exactly, floating point to rounding) and
its update against the oracle's update from the slot's own sample costs, over
consecutive calls (the batch leaves its keys and counts clean for the next
call), mixed iteration counts, both collision sets, both cell sizes, both
queue modes and degenerate items; the autotuner leaves the items' buffers
alone."""
import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I
from gpu_util import JUMP_BAND, TOL_COST_REL, TOL_U, x0_of

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


def _buffers(w, dev):
    import torch
    P = w.params
    return (torch.from_numpy(w.cloud).to(dev), torch.from_numpy(w.hover_nominal()).to(dev),
            torch.empty((P["T"], 4), device=dev), torch.empty((P["E"],), device=dev),
            torch.empty((1,), dtype=torch.int32, device=dev))


def _limits(ws):
    return dict(E_max=16, K_max=4096, T_max=60, fine_cells_max=128 * 64,
                n_points_max=max(1, max(len(w.cloud) for w in ws)))


def _items(aero, ws, bufs):
    return [aero.Batch.item(aero.state_struct(w.p0, w.q0, w.v0), b[0], w.goal,
                            aero.params_struct(w.params), b[1], b[2], b[3], b[4])
            for w, b in zip(ws, bufs)]


def _planner_step(aero, pl, w, u_in, dev):
    import torch
    c, _, ub, cand, best = _buffers(w, dev)
    un = u_in.clone()
    pl.plan_step(aero.state_struct(w.p0, w.q0, w.v0), c, w.goal, aero.params_struct(w.params),
                 un, ub, cand, best)
    torch.cuda.synchronize()
    return un, ub, cand, best


def _check_slot(aero, orc, batch, pl, slot, w, b, u_in, dev, oracle_budget=1_000_000):
    """Slot `slot` of the last batched call.  Against a separate aero_plan_step
    from the same nominal: the integer decisions exactly, anchors and guides to
    rounding, the sample costs to rounding except for the few samples whose
    trajectory meets the jump of J_col at d_max (the two paths compile the same
    unit code in different contexts, so states differ by rounding).  Against the
    oracle, for items of up to `oracle_budget` sample-steps: the update from the
    slot's own sample costs (one-iteration items), the Stage II rollout of the
    slot's own nominal and its costs (instances clear of the jump band), the
    selection."""
    import torch
    P = w.params
    un, ub, cand, best = _planner_step(aero, pl, w, u_in, dev)
    for what in ("GOAL_CELL", "ANCHOR_CELLS", "COARSE_WIN", "POINT_COUNTS"):
        assert np.array_equal(batch.debug(slot, what), pl.debug(what)), (slot, what)
    for what in ("ANCHORS", "GUIDES"):
        np.testing.assert_allclose(batch.debug(slot, what), pl.debug(what), rtol=1e-6, atol=1e-5)
    S_b = batch.debug(slot, "SAMPLE_COSTS").astype(np.float64)
    S_p = pl.debug("SAMPLE_COSTS").astype(np.float64)
    off = np.abs(S_b - S_p) > 2e-5 * np.abs(S_p)
    if P["iters"] == 1:
        assert off.mean() <= 0.01, (slot, int(off.sum()))
    c_b = b[3].cpu().numpy().astype(np.float64)
    bi = int(b[4].cpu()[0])
    assert bi == int(np.argmin(c_b)), slot      # ties to the lower index
    assert torch.equal(b[2], b[1][bi]), slot
    if P["E"] * P["K"] * P["T"] * P["iters"] > oracle_budget:
        return
    u_gpu = b[1].cpu().numpy().astype(np.float64)
    if P["iters"] == 1:
        S = S_b.reshape(P["E"], P["K"])
        lo, hi = np.array(P["u_min"]), np.array(P["u_max"])
        u0s = u_in.cpu().numpy().astype(np.float64)
        for e in range(P["E"]):
            dU = np.clip(u0s[e] + orc.noise_range(P, e, 0, P["K"]), lo, hi) - u0s[e]
            ref, _ = orc.mppi_update(S[e], dU.reshape(P["K"], -1), P["lam"], u0s[e])
            assert np.abs(u_gpu[e] - ref).max() < TOL_U, (slot, e)
    keys = orc.partition(w.cloud, w.p0, w.q0, P)[0]
    pts = orc.collision_set(w.cloud, w.p0, w.q0, keys, P)
    x0 = x0_of(w)
    for e in range(P["E"]):
        X = orc.rollout(x0, u_gpu[e], P["dt"], P["mass"], P["g"])
        t = orc.cost_terms(X, u_gpu[e], None, w.goal.astype(np.float64), pts, P, stage=2,
                           want_dist=True)
        jump = np.min(np.abs(t["dist"] - P["d_max"])) if len(t["dist"]) else np.inf
        if jump > JUMP_BAND:
            assert abs(c_b[e] - t["S"]) <= TOL_COST_REL * abs(t["S"]), (slot, e)


def _batch_calls(aero, orc, batch, pl, ws, bufs, calls=2, oracle_budget=1_000_000):
    """`calls` consecutive batched calls (warm-started), every slot checked."""
    import torch
    dev = torch.device("cuda")
    for call in range(calls):
        for w in ws:
            w.params["step_id"] = call
        u_in = [b[1].clone() for b in bufs]
        batch.plan(_items(aero, ws, bufs))
        torch.cuda.synchronize()
        for i, (w, b) in enumerate(zip(ws, bufs)):
            _check_slot(aero, orc, batch, pl, i, w, b, u_in[i], dev,
                        oracle_budget if call == 0 else 0)


def test_batch_slots_match_planner_steps_and_oracle(aero, orc):
    import torch
    dev = torch.device("cuda")
    ws = I.batch_workloads(64, seed=1)
    for i, w in enumerate(ws):
        w.params["lanes_per_sample"] = 1 if i % 3 else 4
    lim = _limits(ws)
    batch = aero.Batch(len(ws), **lim)
    pl = aero.Planner(debug_samples_max=0, **lim)
    bufs = [_buffers(w, dev) for w in ws]
    _batch_calls(aero, orc, batch, pl, ws, bufs, calls=2)
    assert batch.sync_status() == 0
    pl.close()
    batch.close()


def test_batch_mixed_iterations_collision_sets_and_degenerate_items(aero, orc):
    import torch
    dev = torch.device("cuda")
    ws = I.batch_workloads(12, seed=3)
    for i, w in enumerate(ws):
        w.params["iters"] = 1 + i % 3
        w.params["collision_set"] = 1 if i % 4 == 1 else 0
        w.params["lanes_per_sample"] = 4 if i % 2 else 1
    ws[6].cloud = ws[6].cloud[:0]                       # no points at all
    ws[9].params.update(K=1, T=1)                       # one sample, one step
    lim = _limits(ws)
    batch = aero.Batch(len(ws), **lim)
    batch.set_config(coarse_cells=1)
    pl = aero.Planner(debug_samples_max=0, **lim)
    bufs = [_buffers(w, dev) for w in ws]
    _batch_calls(aero, orc, batch, pl, ws, bufs, calls=2, oracle_budget=200_000)
    # a smaller call on the same batch afterwards, other configuration
    batch.set_config(quad_max_samples=32768, rollout_ctas_per_sm=6, dynamic_queue=0)
    _batch_calls(aero, orc, batch, pl, ws[:5], bufs[:5], calls=1, oracle_budget=200_000)
    pl.close()
    batch.close()


@pytest.mark.parametrize("spc", [64, 256])
def test_batch_samples_per_cta(aero, orc, spc):
    """The one-lane Stage I pass with 64 or 256 samples per CTA (the autotuner's
    choices besides 128): the partial rows are laid out for the CTA size, and
    every slot still matches the planner's step and the oracle."""
    import torch
    dev = torch.device("cuda")
    ws = I.batch_workloads(10, seed=6)
    for w in ws:
        w.params["lanes_per_sample"] = 1
    ws[3].params.update(K=1, T=1)                       # a CTA with one active sample
    ws[5].params.update(K=300, T=60)                    # ragged last CTA, T above 64
    lim = _limits(ws)
    batch = aero.Batch(len(ws), **lim)
    batch.set_config(samples_per_cta=spc)
    assert batch.config()["samples_per_cta"] == spc
    pl = aero.Planner(debug_samples_max=0, **lim)
    bufs = [_buffers(w, dev) for w in ws]
    _batch_calls(aero, orc, batch, pl, ws, bufs, calls=1, oracle_budget=300_000)
    assert batch.sync_status() == 0
    with pytest.raises(aero.AeroError):
        batch.set_config(samples_per_cta=96)
    pl.close()
    batch.close()


def test_batch_tune_then_plan_agrees_with_oracle(aero, orc):
    import torch
    dev = torch.device("cuda")
    ws = I.batch_workloads(16, seed=4)
    lim = _limits(ws)
    batch = aero.Batch(len(ws), **lim)
    bufs = [_buffers(w, dev) for w in ws]
    items = _items(aero, ws, bufs)
    before = [tuple(t.clone() for t in b[1:]) for b in bufs]
    cfg, ms = batch.tune(items, repeats=2)
    torch.cuda.synchronize()
    assert ms > 0 and cfg == batch.config()
    for b, old in zip(bufs, before):   # the tuner wrote only its scratch
        assert torch.equal(b[1], old[0])
    batch.plan(items)
    torch.cuda.synchronize()
    checked = 0
    for i, (w, b) in enumerate(zip(ws, bufs)):
        P = w.params
        if P["E"] * P["K"] * P["T"] > 400_000 or checked >= 2:
            continue
        # Stage II costs of the tuned launch against the oracle; the selection is
        # their argmin (the update itself is compared bitwise in the tests above)
        o = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, w.hover_nominal())
        g_cand = b[3].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(g_cand - o["cand"]) <= TOL_COST_REL * np.abs(o["cand"])), i
        assert int(b[4].cpu()[0]) == int(np.argmin(g_cand)), i
        checked += 1
    assert checked >= 1
    batch.close()


def test_batch_rejects_an_invalid_item_before_enqueuing(aero):
    import torch
    dev = torch.device("cuda")
    ws = I.batch_workloads(3, seed=2)
    batch = aero.Batch(3, **_limits(ws))
    bufs = [_buffers(w, dev) for w in ws]
    before = [b[1].clone() for b in bufs]
    items = _items(aero, ws, bufs)
    items[2].params.K = 8192        # beyond the batch's limits
    with pytest.raises(aero.AeroError) as ei:
        batch.plan(items)
    assert ei.value.code == aero.ERR_EXCEEDS_LIMITS
    items[2].params.K = 256
    items[1].params.debug_samples = 4   # batches carry no debug buffers
    with pytest.raises(aero.AeroError) as ei:
        batch.plan(items)
    assert ei.value.code == aero.ERR_INVALID_ARG
    with pytest.raises(aero.AeroError):
        batch.set_config(quad_max_samples=-1)
    torch.cuda.synchronize()
    for b, u in zip(bufs, before):
        assert torch.equal(b[1], u)   # nothing ran
    batch.close()
