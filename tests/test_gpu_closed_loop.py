"""The receding-horizon loop on the GPU: the warm-start shift kernel against
its definition, and short closed-loop flights through the synthetic forest
(sweeps accumulated on the GPU, plans from the true state, the first controls
flown on the simulated quadrotor)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("shift", [0, 1, 3, 19, 20, 25])
def test_shift_nominal_definition(aero, shift):
    import torch
    rng = np.random.default_rng(shift)
    u = rng.normal(size=(5, 20, 4)).astype(np.float32)
    t = torch.from_numpy(u).cuda()
    aero.shift_nominal(t, shift)
    torch.cuda.synchronize()
    ref = u[:, np.minimum(np.arange(20) + shift, 19), :]
    assert np.array_equal(t.cpu().numpy(), ref)


@pytest.mark.parametrize("iters", [1, 2])
def test_closed_loop_flight_makes_safe_progress(aero, iters):
    from paper_2509_17340_gb300 import closed_loop as L
    scene, P, start, goal = L.scenario("forest", 0)
    P["iters"] = iters
    r = L.fly(scene, P, start, goal, L.LoopConfig(max_time=6.0), seed=0)
    d0 = np.linalg.norm(np.asarray(goal) - np.asarray(start))
    d1 = np.linalg.norm(np.asarray(goal) - r.positions[-1])
    assert not r.crashed
    assert r.min_clearance >= L.LoopConfig().drone_radius
    assert r.success or d0 - d1 > 5.0, (d0, d1)
    assert len(r.plan_ms) == r.cycles and all(ms > 0 for ms in r.plan_ms)
