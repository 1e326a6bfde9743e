"""aero_plan_step_noalloc: the planning step for callers that cannot allocate
device memory while running (a control loop that must not block on cudaMalloc,
a host program that owns all device memory itself).  It takes no planner and
works in a fixed device array inside the library.

Checked through the C ABI against aero_plan_step (which uses a planner created
by aero_create) on two calls in a row -- the second warm-started from the
first -- within the parity tolerances of the other GPU tests, and the size
limits are checked.  Collected last so that a run stopping at the first failure
has run every other test before it.
"""
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


def _outputs(P, dev):
    import torch
    return (torch.empty((P["T"], 4), device=dev), torch.empty((P["E"],), device=dev),
            torch.empty((1,), dtype=torch.int32, device=dev))


def test_noalloc_matches_planner_on_two_calls(aero):
    import torch
    dev = torch.device("cuda")
    w = I.make_workload("ensemble")   # E=8, K=1024, T=40, 20,816 points: inside the limits
    P = w.params
    cloud = torch.from_numpy(w.cloud).to(dev)
    state = aero.state_struct(w.p0, w.q0, w.v0)
    pl = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                      fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=len(w.cloud))
    u_ref = torch.from_numpy(w.hover_nominal()).to(dev)
    u_na = u_ref.clone()
    for call in range(2):
        P["step_id"] = call
        prm = aero.params_struct(P)
        ub_ref, c_ref, b_ref = _outputs(P, dev)
        ub_na, c_na, b_na = _outputs(P, dev)
        pl.plan_step(state, cloud, w.goal, prm, u_ref, ub_ref, c_ref, b_ref)
        aero.plan_step_noalloc(state, cloud, w.goal, prm, u_na, ub_na, c_na, b_na)
        torch.cuda.synchronize()
        assert np.abs(u_na.cpu().numpy() - u_ref.cpu().numpy()).max() < TOL_U, call
        assert np.abs(ub_na.cpu().numpy() - ub_ref.cpu().numpy()).max() < TOL_U, call
        cr = c_ref.cpu().numpy()
        assert np.all(np.abs(c_na.cpu().numpy() - cr) <= TOL_COST_REL * np.abs(cr)), call
        assert int(b_na.cpu()[0]) == int(b_ref.cpu()[0]), call
    pl.close()


def test_noalloc_rejects_sizes_beyond_its_array(aero):
    import torch
    dev = torch.device("cuda")
    w = I.make_workload("ensemble")
    cloud = torch.from_numpy(w.cloud).to(dev)
    state = aero.state_struct(w.p0, w.q0, w.v0)
    for upd in [dict(K=4096), dict(T=65), dict(debug_samples=1),
                dict(E=32, M_h=8, M_v=4, fine_az=256, pool_az=4, pool_el=8, fine_el=64),
                dict(collision_set=1)]:
        P = dict(w.params, **upd)
        u = torch.zeros((P["E"], P["T"], 4), device=dev)
        ub, c, b = _outputs(P, dev)
        with pytest.raises(aero.AeroError) as ei:
            aero.plan_step_noalloc(state, cloud, w.goal, aero.params_struct(P), u, ub, c, b)
        assert ei.value.code == aero.ERR_EXCEEDS_LIMITS, upd
