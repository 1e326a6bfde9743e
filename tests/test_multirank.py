"""The multi-rank logic of bench.py on CPU with gloo (world size 2): each rank
plans its own scene (weak scaling), the step time is the maximum over ranks,
the value counts the units of all ranks; and the reference arm runs on CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2509_17340_gb300 import inputs as I
    seed = bench.rank_seed(rank)
    w = I.make_workload("plain", seed=seed)
    t = bench.max_over_ranks(1.5 + rank, dist)
    v = bench.job_value(w.params, world, 10, t)
    q.put((rank, seed, float(w.cloud[0, 0]), t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, c0, t0, v0), (_, s1, c1, t1, v1) = out
    assert s0 != s1 and c0 != c1            # different scenes per rank
    assert t0 == t1 == 2.5                  # the slowest rank's time on every rank
    P = __import__("paper_2509_17340_gb300.inputs", fromlist=["x"]).workload_params("plain")
    steps_per_plan = P["E"] * P["K"] * P["T"] + P["E"] * P["T"]
    assert v0 == v1 == pytest.approx(2 * steps_per_plan * 10 / 2.5)


def test_reference_arm_runs_the_oracle_on_cpu():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--reference-budget", "3"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "rollout-steps/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
