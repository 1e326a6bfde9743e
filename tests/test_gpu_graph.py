"""aero_plan_step enqueues without allocating or synchronising, so a step can
be captured in a CUDA graph (programmatic launch edges included) and
replayed: every replay equals a direct step on the same inputs, bit for bit,
for both Stage I passes and with the gradient refinement."""
import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I

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


@pytest.mark.parametrize("variant", ["split", "one_lane", "refined"])
def test_graph_replay_equals_direct_steps(aero, variant):
    import torch
    w = I.make_workload("ensemble")
    P = dict(w.params, K=512, T=24)
    if variant == "one_lane":
        P["lanes_per_sample"] = 1
    if variant == "refined":
        P.update(refine_steps=2, refine_step=0.02)
    dev = torch.device("cuda")
    pl = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"], fine_cells_max=P["fine_az"] * P["fine_el"],
                      n_points_max=len(w.cloud))
    cloud = torch.from_numpy(w.cloud).to(dev)
    u0 = torch.from_numpy(np.ascontiguousarray(w.hover_nominal()[:, :P["T"]])).to(dev)
    state, ps = aero.state_struct(w.p0, w.q0, w.v0), aero.params_struct(P)

    def buffers():
        return (u0.clone(), torch.empty((P["T"], 4), device=dev), torch.empty((P["E"],), device=dev),
                torch.empty((1,), dtype=torch.int32, device=dev))

    # direct: two consecutive steps from u0 (the second warm-started by the first)
    un, ub, cand, best = buffers()
    ref = []
    for _ in range(2):
        pl.plan_step(state, cloud, w.goal, ps, un, ub, cand, best)
        torch.cuda.synchronize()
        ref.append((un.clone(), ub.clone(), cand.clone(), best.clone()))
    assert pl.sync_status() == 0
    # captured once, replayed twice on the same buffers
    g_un, g_ub, g_cand, g_best = buffers()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        graph.capture_begin()
        pl.plan_step(state, cloud, w.goal, ps, g_un, g_ub, g_cand, g_best, stream=side)
        graph.capture_end()
    torch.cuda.current_stream().wait_stream(side)
    for r in ref:
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip((g_un, g_ub, g_cand, g_best), r):
            assert torch.equal(a, b), variant
    assert pl.sync_status() == 0
    # a fresh planner's very first call captured (its workspace clears included)
    pl2 = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                       fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=len(w.cloud))
    f_un, f_ub, f_cand, f_best = buffers()
    graph2 = torch.cuda.CUDAGraph()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        graph2.capture_begin()
        pl2.plan_step(state, cloud, w.goal, ps, f_un, f_ub, f_cand, f_best, stream=side)
        graph2.capture_end()
    torch.cuda.current_stream().wait_stream(side)
    for r in ref:
        graph2.replay()
        torch.cuda.synchronize()
        for a, b in zip((f_un, f_ub, f_cand, f_best), r):
            assert torch.equal(a, b), variant
    assert pl2.sync_status() == 0
    pl2.close()
    pl.close()
