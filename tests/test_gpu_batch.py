"""Batched planning (aero_batch_plan): 64 independent planners of uneven sizes
and scenes in one call give bitwise the results of 64 separate aero_plan_step
calls, and sampled planners agree with the oracle."""
import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I
from gpu_util import TOL_COST_REL, TOL_U

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


def test_batch_equals_individual_steps_and_oracle(aero, orc):
    import torch
    dev = torch.device("cuda")
    ws = I.batch_workloads(64, seed=1)
    lim = dict(E_max=16, K_max=4096, T_max=60, fine_cells_max=128 * 64,
               n_points_max=max(len(w.cloud) for w in ws))
    batch = aero.Batch(len(ws), **lim)
    bufs = [_buffers(w, dev) for w in ws]
    items = [aero.Batch.item(aero.state_struct(w.p0, w.q0, w.v0), b[0], w.goal,
                             aero.params_struct(w.params), b[1], b[2], b[3], b[4])
             for w, b in zip(ws, bufs)]
    batch.plan(items)
    torch.cuda.synchronize()
    pl = aero.Planner(debug_samples_max=0, **lim)
    checked = 0
    for i, (w, b) in enumerate(zip(ws, bufs)):
        c, un, ub, cand, best = _buffers(w, dev)
        pl.plan_step(aero.state_struct(w.p0, w.q0, w.v0), c, w.goal, aero.params_struct(w.params),
                     un, ub, cand, best)
        torch.cuda.synchronize()
        assert torch.equal(un, b[1]) and torch.equal(cand, b[3]) and torch.equal(best, b[4]), i
        assert torch.equal(ub, b[2]), i
        P = w.params
        if P["K"] == 256 and P["T"] == 20 and checked < 3:
            # oracle: Stage II costs, selection, and the update from the GPU's sample costs
            o = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, w.hover_nominal())
            S = pl.debug("SAMPLE_COSTS").reshape(P["E"], P["K"]).astype(np.float64)
            lo, hi = np.array(P["u_min"]), np.array(P["u_max"])
            u_gpu = un.cpu().numpy()
            for e in range(P["E"]):
                u0 = w.hover_nominal()[e].astype(np.float64)
                dU = np.clip(u0 + orc.noise_range(P, e, 0, P["K"]), lo, hi) - u0
                ref, _ = orc.mppi_update(S[e], dU.reshape(P["K"], -1), P["lam"], u0)
                assert np.abs(u_gpu[e] - ref).max() < TOL_U, (i, e)
            assert np.array_equal(pl.debug("FINE_KEYS"), o["keys"])
            g_cand = cand.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(g_cand - o["cand"]) <= TOL_COST_REL * np.abs(o["cand"])), i
            checked += 1
    assert checked >= 1
    pl.close()
    batch.close()


def test_batch_rejects_an_invalid_item_before_enqueuing(aero):
    import torch
    dev = torch.device("cuda")
    ws = I.batch_workloads(3, seed=2)
    batch = aero.Batch(3, E_max=16, K_max=4096, T_max=60, fine_cells_max=128 * 64,
                       n_points_max=max(len(w.cloud) for w in ws))
    bufs = [_buffers(w, dev) for w in ws]
    before = [b[1].clone() for b in bufs]
    items = [aero.Batch.item(aero.state_struct(w.p0, w.q0, w.v0), b[0], w.goal,
                             aero.params_struct(w.params), b[1], b[2], b[3], b[4])
             for w, b in zip(ws, bufs)]
    items[2].params.K = 8192        # beyond the batch's limits
    with pytest.raises(aero.AeroError) as ei:
        batch.plan(items)
    assert ei.value.code == aero.ERR_EXCEEDS_LIMITS
    torch.cuda.synchronize()
    for b, u in zip(bufs, before):
        assert torch.equal(b[1], u)   # nothing ran
    batch.close()
