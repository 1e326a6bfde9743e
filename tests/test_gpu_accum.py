"""Multi-sweep accumulation on the GPU (aero_accum_*, Sec. IV-A.1) against the
oracle's pose transforms: ring contents and NaN padding, eviction of the
oldest frame, the compacted gathers in world and body frames, LiDAR sweeps
from poses along a path, and planning on the ring equal to planning on the
compacted cloud."""
import ctypes as C
import glob
import os

import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_POS = 2e-5   # m: binary32 transform of points within ~40 m


@pytest.fixture(scope="module")
def aero():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero as A
    return A


def _q(rng):
    q = rng.normal(size=4)
    return (q / np.linalg.norm(q)).astype(np.float32)


def _rot(q):
    w, x, y, z = (float(v) for v in q / np.linalg.norm(q))
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _device_to_host(ptr: int, nbytes: int) -> np.ndarray:
    """Copy library-owned device memory to the host with the CUDA runtime."""
    import torch
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcudart.so")]
    cands += sorted(glob.glob("/usr/local/cuda*/lib64/libcudart.so*"))
    cands += sorted(glob.glob(os.path.join(os.path.dirname(torch.__file__), "..", "nvidia", "*",
                                           "lib", "libcudart.so*")))
    for c in cands:
        if os.path.exists(c):
            rt = C.CDLL(c)
            break
    else:
        pytest.skip("no CUDA runtime library to copy the ring with")
    out = np.empty(nbytes, np.uint8)
    torch.cuda.synchronize()
    rt.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
    assert rt.cudaMemcpy(out.ctypes.data, ptr, nbytes, 2) == 0   # cudaMemcpyDeviceToHost
    return out


def _frames(rng, count, N):
    frames = []
    for f in range(count):
        n = N if f % 4 == 0 else int(rng.integers(0, N + 1))
        frames.append((rng.normal(0, 10, (n, 3)).astype(np.float32),
                       rng.normal(0, 15, 3).astype(np.float32), _q(rng)))
    return frames


def test_push_gather_world_and_body(aero, orc):
    import torch
    rng = np.random.default_rng(0)
    F, N = 5, 3000
    acc = aero.Accumulator(F, N)
    frames = _frames(rng, F + 3, N)          # the first three are evicted
    for ps, p, q in frames:
        acc.push(torch.from_numpy(ps).cuda(), p, q)
    live = frames[-F:]
    ref = np.concatenate([orc.accumulate(ps.astype(np.float64), p, q) for ps, p, q in live])
    cloud, valid = acc.view()
    assert cloud.shape[0] == F * N and valid == len(ref)
    dst = torch.empty((F * N, 3), device="cuda")
    n = acc.gather(dst)
    torch.cuda.synchronize()
    assert n == len(ref)
    assert np.abs(dst[:n].cpu().numpy() - ref).max() < TOL_POS
    p0, q0 = rng.normal(0, 5, 3).astype(np.float32), _q(rng)
    n = acc.gather(dst, p0, q0)
    torch.cuda.synchronize()
    refb = orc.project(ref, p0.astype(np.float64), q0.astype(np.float64))
    assert np.abs(dst[:n].cpu().numpy() - refb).max() < TOL_POS
    acc.reset()
    assert acc.gather(dst) == 0 and acc.view()[1] == 0
    acc.close()


def test_ring_layout_and_nan_padding(aero, orc):
    """The ring as a cloud: slot s holds its frame's points, then NaN."""
    import torch
    rng = np.random.default_rng(1)
    F, N = 3, 1000
    acc = aero.Accumulator(F, N)
    frames = _frames(rng, F + 1, N)
    for ps, p, q in frames:
        acc.push(torch.from_numpy(ps).cuda(), p, q)
    cloud, _ = acc.view()
    host = _device_to_host(cloud.ptr, F * N * 12).view(np.float32).reshape(F * N, 3)
    # after F + 1 pushes slot 0 holds frame F, slot s (1 <= s < F) frame s
    for slot, f in [(0, F)] + [(s, s) for s in range(1, F)]:
        ps, p, q = frames[f]
        blk = host[slot * N:(slot + 1) * N]
        if len(ps):
            assert np.abs(blk[:len(ps)] - orc.accumulate(ps.astype(np.float64), p, q)).max() < TOL_POS
        assert np.all(np.isnan(blk[len(ps):]))
    acc.close()


def test_lidar_sweeps_along_a_path_round_trip(aero, orc):
    """Sweeps of the forest scene from three poses, each pushed in its sensor
    frame, come back in world coordinates as the ray-cast hit points."""
    import torch
    rng = np.random.default_rng(2)
    _, scene = I.scene_ensemble(0)
    acc = aero.Accumulator(10, 40000)
    hits = []
    for k, x in enumerate([0.0, 1.5, 3.0]):
        p = np.array([x, 0.2 * k, 1.5], np.float32)
        q = _q(rng) if k else np.array([1, 0, 0, 0], np.float32)
        pw = I.lidar_sweep(scene, p, 512, 16, -15, 15, 30.0, 0.0, rng)
        ps = orc.project(pw, p.astype(np.float64), q.astype(np.float64)).astype(np.float32)
        acc.push(torch.from_numpy(np.ascontiguousarray(ps)).cuda(), p, q)
        hits.append(pw)
    ref = np.concatenate(hits)
    dst = torch.empty((10 * 40000, 3), device="cuda")
    n = acc.gather(dst)
    torch.cuda.synchronize()
    assert n == len(ref) > 10000
    # binary32 sensor coordinates and transform: within TOL_POS of the hits
    assert np.abs(dst[:n].cpu().numpy() - ref).max() < TOL_POS
    acc.close()


def test_planning_on_the_ring_equals_planning_on_the_gathered_cloud(aero):
    import torch
    w = I.make_workload("ensemble")
    P = dict(w.params, K=256, T=20)
    rng = np.random.default_rng(3)
    acc = aero.Accumulator(4, 8000)
    for f in range(4):
        part = w.cloud[f::4][:8000].astype(np.float64)
        q, p = _q(rng), rng.normal(0, 1, 3).astype(np.float32)
        ps = ((part - p) @ _rot(q)).astype(np.float32)   # the part seen from pose (p, q)
        acc.push(torch.from_numpy(np.ascontiguousarray(ps)).cuda(), p, q)
    ring, valid = acc.view()
    gathered = torch.empty((valid, 3), device="cuda")
    assert acc.gather(gathered) == valid
    pl = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                      fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=ring.shape[0])
    u0 = np.ascontiguousarray(np.tile(w.hover_nominal()[:, :1], (1, P["T"], 1)))
    out = []
    for cloud in (ring, gathered):
        un = torch.from_numpy(u0.copy()).cuda()
        ub, cand = torch.empty((P["T"], 4), device="cuda"), torch.empty((P["E"],), device="cuda")
        best = torch.empty((1,), dtype=torch.int32, device="cuda")
        pl.plan_step(aero.state_struct(w.p0, w.q0, w.v0), cloud, w.goal, aero.params_struct(P),
                     un, ub, cand, best)
        torch.cuda.synchronize()
        out.append((un, cand, int(best.cpu()[0]), pl.debug("COARSE_WIN"), pl.debug("ANCHOR_CELLS")))
    # the same points (the ring adds NaN padding and other indices): the same
    # decisions, and costs and nominals equal to rounding of the summation order
    assert np.array_equal(out[0][3], out[1][3]) and np.array_equal(out[0][4], out[1][4])
    torch.testing.assert_close(out[0][1], out[1][1], rtol=1e-6, atol=0)
    torch.testing.assert_close(out[0][0], out[1][0], rtol=1e-5, atol=1e-5)
    assert out[0][2] == out[1][2]
    pl.close()
    acc.close()


def test_accumulator_rejects_bad_arguments(aero):
    import torch
    acc = aero.Accumulator(2, 100)
    with pytest.raises(aero.AeroError):
        acc.push(torch.zeros((101, 3), device="cuda"), [0, 0, 0], [1, 0, 0, 0])   # too many points
    with pytest.raises(aero.AeroError):
        acc.push(torch.zeros((10, 3), device="cuda"), [0, 0, 0], [0, 0, 0, 0])    # zero quaternion
    acc.push(torch.zeros((50, 3), device="cuda"), [0, 0, 0], [1, 0, 0, 0])
    with pytest.raises(aero.AeroError):
        acc.gather(torch.empty((10, 3), device="cuda"))                              # capacity
    with pytest.raises(aero.AeroError):
        aero.Accumulator(0, 100)
    acc.close()
