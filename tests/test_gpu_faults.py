"""Failure paths of the boundary, driven on the host: every allocation of the
create functions is made to fail in turn (aero_test_fail_alloc); each failure
is reported as AERO_ERR_ALLOC and frees everything the call had allocated,
and the library stays usable afterwards.  Nothing here faults the device."""
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
    yield A
    A.inject_alloc_failure(-1)


SMALL = dict(E_max=4, K_max=256, T_max=16, fine_cells_max=64 * 16, n_points_max=5000)


def _makers(aero):
    return {
        "planner": lambda: aero.Planner(**SMALL),
        "planner_debug": lambda: aero.Planner(**SMALL, debug_samples_max=4),
        "batch": lambda: aero.Batch(2, **SMALL),
        "accumulator": lambda: aero.Accumulator(3, 1000),
    }


@pytest.mark.parametrize("kind", ["planner", "planner_debug", "batch", "accumulator"])
def test_each_failed_allocation_is_reported_and_nothing_leaks(aero, kind):
    make = _makers(aero)[kind]
    total0, live0 = aero.alloc_stats()
    obj = make()
    total1, live1 = aero.alloc_stats()
    n = total1 - total0
    assert n >= 1 and live1 - live0 == n
    obj.close()
    assert aero.alloc_stats()[1] == live0
    for k in range(n):
        aero.inject_alloc_failure(k)
        with pytest.raises(aero.AeroError) as err:
            make()
        assert err.value.code == aero.ERR_ALLOC, (kind, k)
        assert aero.alloc_stats()[1] == live0, (kind, k)
    # the countdown fired: the next create succeeds
    obj = make()
    assert aero.alloc_stats()[1] == live0 + n
    obj.close()


def test_cancelled_failure_does_not_fire(aero):
    _, live0 = aero.alloc_stats()
    aero.inject_alloc_failure(0)
    aero.inject_alloc_failure(-1)
    pl = aero.Planner(**SMALL)
    pl.close()
    assert aero.alloc_stats()[1] == live0


def test_planning_after_failed_creates(aero):
    """After a run of failed creates the same process plans the small
    ensemble workload to a finite, valid result."""
    import torch
    w = I.make_workload("ensemble")
    P = dict(w.params, K=256, T=16, E=4, M_h=2, M_v=2, fine_az=64, fine_el=16, pool_az=8, pool_el=4)
    for k in range(3):
        aero.inject_alloc_failure(k)
        with pytest.raises(aero.AeroError):
            aero.Planner(**SMALL)
    cloud = torch.from_numpy(w.cloud[:SMALL["n_points_max"]]).cuda()
    pl = aero.Planner(**SMALL)
    un = torch.from_numpy(np.ascontiguousarray(w.hover_nominal()[:P["E"], :P["T"]])).cuda()
    ub, cand, best = aero.plan_step(pl, w.p0, w.q0, w.v0, cloud, w.goal, P, un)
    torch.cuda.synchronize()
    pl.sync_status()
    assert torch.isfinite(ub).all() and torch.isfinite(cand).all()
    assert 0 <= int(best.cpu()[0]) < P["E"]
    pl.close()


@pytest.mark.parametrize("lanes", [1, 4])
def test_non_finite_costs_select_the_first_instance(aero, lanes):
    # an infinite control weight makes every cost non-finite: the step still
    # selects an instance in range (the first), the status word reports it,
    # and the planner is usable afterwards
    import torch
    w = I.make_workload("ensemble")
    P = dict(w.params, K=256, lanes_per_sample=lanes)
    pl = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                      fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=len(w.cloud))
    cloud = torch.from_numpy(w.cloud).cuda()
    u0 = torch.from_numpy(w.hover_nominal()).cuda()
    bad = dict(P, Q_c=float("inf"))
    u_best, cand, best = aero.plan_step(pl, w.p0, w.q0, w.v0, cloud, w.goal, bad, u0.clone())
    assert pl.sync_status() == aero.ERR_DEVICE_CHECK
    assert int(best.item()) == 0
    assert not torch.isfinite(cand).any()
    u_best, cand, best = aero.plan_step(pl, w.p0, w.q0, w.v0, cloud, w.goal, P, u0.clone())
    assert pl.sync_status() == 0
    assert torch.isfinite(cand).all() and 0 <= int(best.item()) < P["E"]
    assert int(best.item()) == int(torch.argmin(cand).item())
    pl.close()
