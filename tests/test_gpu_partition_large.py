"""The partition of clouds of four million points and more (Sec. IV-A: the
cloud binned into fine cones, the nearest point of each cone kept), where the
kernel takes four points per thread, against the oracle bit for bit: every
cone's key, the point counts, the same step from a page-locked host cloud and
from a cloud at an address that is not 16-byte aligned (one point per thread),
and the every-point collision set (its item flags) through the grid lists.
Sizes are not multiples of four, so the last points take the tail path;
non-finite points, the start itself (range zero), duplicates (equal keys: the
lowest index wins) and points outside the range and the elevation span sit at
every position of a group of four."""
import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I
from gpu_util import run_gpu

pytestmark = pytest.mark.gpu

N_MIXED = 4_000_003
N_RAW = 4_000_001


@pytest.fixture(scope="module")
def aero():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero as A
    return A


def _workload(n: int, spread: float, seed: int, raw: int) -> I.Workload:
    w = I.make_workload("plain", seed=seed)
    rng = np.random.default_rng(seed)
    w.q0 = I.random_unit_quaternion(rng)
    p0 = w.p0.astype(np.float32)
    cloud = (p0 + rng.uniform(-spread, spread, size=(n, 3))).astype(np.float32)
    # corner cases at each position of a group of four, and in the tail
    where = np.concatenate([np.arange(0, 16), np.arange(n - 7, n),
                            rng.choice(n - 32, 64, replace=False) + 16])
    kinds = np.arange(len(where)) % 8
    for i, k in zip(where, kinds):
        if k == 0:
            cloud[i] = [np.nan, 0.0, 1.0]
        elif k == 1:
            cloud[i] = [1.0, np.inf, -2.0]
        elif k == 2:
            cloud[i] = p0                       # range zero: not kept
        elif k == 3:
            cloud[i] = cloud[(i + 1) % n]        # a duplicate: equal keys
        elif k == 4:
            cloud[i] = p0 + [0.0, 0.0, 9.0]      # steep: often outside the elevation span
        elif k == 5:
            cloud[i] = p0 + [40.0, 0.0, 0.0]     # beyond r_max
        elif k == 6:
            cloud[i] = p0 + [0.5, 0.25, 0.1]     # close: likely its cone's winner
        else:
            cloud[i] = p0 + [-0.5, -0.25, -0.05]
    w.cloud = cloud
    w.params.update(E=1, M_h=1, M_v=1, K=32, T=4, r_max=12.0, el_lo=-0.45, el_hi=0.6,
                    fine_az=256, fine_el=64, pool_az=4, pool_el=8, collision_set=raw)
    return w


@pytest.fixture(scope="module")
def mixed(aero, orc):
    w = _workload(N_MIXED, 9.0, 21, 0)
    pl = aero.Planner(E_max=1, K_max=32, T_max=4, fine_cells_max=256 * 64, n_points_max=N_MIXED,
                      debug_samples_max=1)
    u0 = w.hover_nominal()
    g = run_gpu(aero, pl, w, w.params, u0)
    keys, kept = orc.partition(w.cloud, w.p0, w.q0, w.params)
    yield w, pl, u0, g, keys, kept
    pl.close()


def test_keys_and_counts_bit_exact(mixed):
    w, pl, u0, g, keys, kept = mixed
    assert np.array_equal(g["keys"], keys)
    nonfinite = int((~np.isfinite(w.cloud).all(axis=1)).sum())
    assert list(g["point_counts"]) == [N_MIXED, nonfinite, kept]
    assert 0 < kept < N_MIXED - nonfinite


def test_pinned_host_cloud_same_step(aero, mixed):
    # the partition reads the page-locked cloud in place and leaves the device
    # copy the later stages read
    import torch
    w, pl, u0, g, keys, kept = mixed
    P = w.params
    cloud = torch.from_numpy(w.cloud.copy()).pin_memory()
    un = torch.from_numpy(u0.copy()).pin_memory()
    ub = torch.zeros((P["T"], 4)).pin_memory()
    cand = torch.zeros(P["E"]).pin_memory()
    best = torch.zeros(1, dtype=torch.int32).pin_memory()
    pl.plan_step_host(aero.state_struct(w.p0, w.q0, w.v0), cloud, w.goal, aero.params_struct(P),
                      un, ub, cand, best)
    assert np.array_equal(pl.debug("FINE_KEYS"), keys)
    assert np.array_equal(pl.debug("POINT_COUNTS"), g["point_counts"])
    assert np.array_equal(un.numpy().astype(np.float64), g["u_nom"])
    assert np.array_equal(cand.numpy(), g["cand"]) and int(best[0]) == g["best"]


def test_unaligned_cloud_same_keys(aero, mixed):
    import torch
    w, pl, u0, g, keys, kept = mixed
    n = len(w.cloud)
    buf = torch.zeros((n + 1) * 3, dtype=torch.float32, device="cuda")
    buf[3:] = torch.from_numpy(w.cloud.reshape(-1)).cuda()
    cloud = buf[3:].view(n, 3)
    assert cloud.data_ptr() % 16 != 0
    un = torch.from_numpy(np.ascontiguousarray(u0, np.float32)).cuda()
    u_best, cand, best = aero.plan_step(pl, w.p0, w.q0, w.v0, cloud, w.goal, w.params, un)
    torch.cuda.synchronize()
    assert pl.sync_status() == 0
    assert np.array_equal(pl.debug("FINE_KEYS"), keys)
    assert np.array_equal(pl.debug("POINT_COUNTS"), g["point_counts"])
    assert np.array_equal(un.cpu().numpy().astype(np.float64), g["u_nom"])
    assert np.array_equal(cand.cpu().numpy(), g["cand"]) and int(best.cpu()[0]) == g["best"]


def test_every_point_set_item_flags(aero, orc):
    """The every-point collision set: the grid lists hold exactly the kept
    points (each entry's item is its point's index)."""
    w = _workload(N_RAW, 60.0, 22, 1)
    P = w.params
    pl = aero.Planner(E_max=1, K_max=32, T_max=4, fine_cells_max=256 * 64, n_points_max=N_RAW,
                      debug_samples_max=1, raw_points_max=N_RAW)
    try:
        g = run_gpu(aero, pl, w, P, w.hover_nominal())
        keys, kept = orc.partition(w.cloud, w.p0, w.q0, P)
        assert np.array_equal(g["keys"], keys)
        assert g["point_counts"][2] == kept and kept > 1000
        pts = pl.debug("GRID_POINTS")
        items_all = pts[:, 3].view(np.int32)
        # every entry is its item's point (relative to the start, in binary32)
        assert np.array_equal(pts[:, :3], (w.cloud[items_all] - w.p0).astype(np.float32))
        items = np.unique(items_all)
        ref = orc.collision_set(w.cloud, w.p0, w.q0, keys, P).astype(np.float32)
        assert len(items) == len(ref) == kept

        def rows(a):
            return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]
        assert np.array_equal(rows(w.cloud[items]), rows(ref))
    finally:
        pl.close()
