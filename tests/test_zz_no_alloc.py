"""aero_plan_step_noalloc: the planning step for callers that cannot allocate
device memory while running (a control loop that must not block on cudaMalloc,
a host program that owns all device memory itself).  It takes no planner and
works in a fixed device array inside the library.

Checked through the C ABI against aero_plan_step (which uses a planner created
by aero_create) on two calls in a row -- the second warm-started from the
first -- within the parity tolerances of the other GPU tests, for both Stage I
passes, with and without the gradient refinement, and with a partition range
large enough that the collision grid is coarsened to the array's 32^3 cells.
The size limits and the refusal of a first call inside a stream capture are
checked too.  Collected last so that a run stopping at the first failure has
run every other test before it.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I
from gpu_util import TOL_COST_REL, TOL_U

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _grid_cells_per_axis(P: dict, cap: int, gmax: int) -> int:
    """Cells per axis of the collision grid for the P_f set of P under a
    candidate capacity `cap` and at most `gmax` cells per axis (the
    planner's rule, restated for the test's choice of r_max)."""
    n_items = P["fine_az"] * P["fine_el"]
    reach = P["d_max"] * (1 + 1e-3) + 1e-4
    h = 0.5 * P["d_max"] if 216 * n_items <= cap else P["d_max"] * 1.0625
    G = int(np.ceil(2 * (P["r_max"] + reach + h) / h))
    return min(G, gmax)


# (lanes_per_sample, refine_steps, r_max): both Stage I passes, the refinement
# in the fused update (four lanes) and in the update launch (one lane), and a
# partition range whose grid needs more than 32 cells per axis at the finest
# admissible edge, so the noalloc array's grid is coarsened
CASES = [(0, 0, None), (1, 0, None), (4, 5, None), (1, 5, None), (4, 0, 40.0)]


@pytest.mark.parametrize("lanes,refine,r_max", CASES)
def test_noalloc_matches_planner_on_two_calls(aero, lanes, refine, r_max):
    import torch
    dev = torch.device("cuda")
    w = I.make_workload("ensemble")   # E=8, K=1024, T=40, 20,816 points: inside the limits
    P = w.params
    P["lanes_per_sample"] = lanes
    P["refine_steps"] = refine
    if r_max is not None:
        P["r_max"] = r_max
        assert _grid_cells_per_axis(P, 1 << 18, 10**9) > 32
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


_FIRST_CALL_IN_CAPTURE = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2509_17340_gb300 import aero, inputs as I
w = I.make_workload("ensemble")
P = w.params
dev = torch.device("cuda")
cloud = torch.from_numpy(w.cloud).to(dev)
u = torch.from_numpy(w.hover_nominal()).to(dev)
ub, c, b = (torch.empty((P["T"], 4), device=dev), torch.empty((P["E"],), device=dev),
            torch.empty((1,), dtype=torch.int32, device=dev))
state, prm = aero.state_struct(w.p0, w.q0, w.v0), aero.params_struct(P)
s = torch.cuda.Stream()
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
code = None
with torch.cuda.stream(s):
    g.capture_begin()
    try:
        aero.plan_step_noalloc(state, cloud, w.goal, prm, u, ub, c, b, s)
    except aero.AeroError as ex:
        code = ex.code
    g.capture_end()
assert code == aero.ERR_INVALID_ARG, code
aero.plan_step_noalloc(state, cloud, w.goal, prm, u, ub, c, b)   # outside capture: sets up
torch.cuda.synchronize()
print("ok")
"""


def test_noalloc_first_call_inside_capture_is_refused(aero):
    """A fresh process whose first noalloc call is made on a capturing stream
    gets AERO_ERR_INVALID_ARG (the set-up is not a stream operation); the next
    call, outside the capture, sets the device up and runs."""
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_IN_CAPTURE, ROOT], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


@pytest.mark.parametrize("lanes,refine,events", [(4, 0, False), (4, 5, False), (1, 0, False),
                                                  (1, 5, False), (1, 0, True), (4, 0, True)])
def test_outputs_equal_with_and_without_the_fused_update_and_warm_up_block(aero, lanes, refine,
                                                                           events):
    # a planner's Stage I launch runs a warm-up block (the update's code on
    # scratch at the start of the launch) and, in the one-lane pass, the
    # update in the last CTA of each instance; the no-allocation entry point
    # runs neither (the one-lane pass's update is a launch of its own).  The
    # nearest-point distances do not depend on the grid's cell edge, and every
    # sum runs in a fixed order, so the two agree bit for bit: the warm-up
    # block writes nothing the step returns.  With events around Stage I the
    # update launch no longer overlaps it, and its CTAs skip the warm-up run.
    import torch
    dev = torch.device("cuda")
    w = I.make_workload("ensemble")
    P = dict(w.params, lanes_per_sample=lanes, refine_steps=refine)
    cloud = torch.from_numpy(w.cloud).to(dev)
    state = aero.state_struct(w.p0, w.q0, w.v0)
    pl = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                      fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=len(w.cloud))
    u_ref = torch.from_numpy(w.hover_nominal()).to(dev)
    u_na = u_ref.clone()
    if events:
        pl.profile(["rollout"])
    for call in range(3):
        P["step_id"] = 100 + call
        prm = aero.params_struct(P)
        ub_ref, c_ref, b_ref = _outputs(P, dev)
        ub_na, c_na, b_na = _outputs(P, dev)
        pl.plan_step(state, cloud, w.goal, prm, u_ref, ub_ref, c_ref, b_ref)
        aero.plan_step_noalloc(state, cloud, w.goal, prm, u_na, ub_na, c_na, b_na)
        torch.cuda.synchronize()
        assert torch.equal(u_na, u_ref), call
        assert torch.equal(ub_na, ub_ref), call
        assert torch.equal(c_na, c_ref), call
        assert torch.equal(b_na, b_ref), call
    assert pl.sync_status() == 0
    pl.close()
