"""Benchmark of one AERO-MPPI planning step on GB300 (prints ONE JSON line).

A "step" is one pass of the whole hot path over one synthetic scene: fine
partition and collision grid, coarse argmax, anchors, quintic guides, the E x K
x T sampled rollouts with their Stage I costs, the softmax-weighted update, the
Stage II re-rollout and the selection.  The workload is the anchor-guided
ensemble (E=8, K=1024, T=40, forest LiDAR sweep).

Metric: rollout-steps per second = (E K T iters + E T) / step time.  Each timed
step is bracketed by CUDA events on the planner's stream; L2 (129 MB) is
flushed by writing a 512 MB buffer between timed steps, outside the events.
Every step plans from the same state and hover warm start (a fresh Philox
step_id each time), so the timed work does not drift with the step index.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank plans its own scene (seed = rank): weak scaling, no
data-path collective; the step time is the maximum over ranks.  ``--impl
reference`` times the CPU oracle on the host cores instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_17340_gb300 import inputs as I  # noqa: E402

WORKLOAD = "ensemble"
METRIC = "rollout-steps/s (anchor-guided ensemble plan step)"
METRICS = {"ensemble": METRIC, "large": "rollout-steps/s (large-clutter ensemble plan step)",
           "plain": "rollout-steps/s (plain single-MPPI plan step)",
           "batched": "rollout-steps/s (64 independent planners in one batched call)",
           "refined": "rollout-steps/s (ensemble plan step with 5 gradient-refinement steps)",
           "accumulate": "points/s (LiDAR frame push + 10-frame gather)"}
UNIT = "rollout-steps/s"
CPU_SAMPLE_SECONDS = 15.0


def rollout_steps(P: dict) -> int:
    return P["E"] * P["K"] * P["T"] * P["iters"] + P["E"] * P["T"]


def rollout_flops_per_step() -> int:
    """Algorithmic FP32 flops of one sample-step of the fused rollout kernel
    (counted from the formulas; FMA = 2, nearest-point distance tests excluded):
      noise: Box-Muller 2 x (log, sqrt, sincos) + 4 scalings + 4 adds ... 16
      clamp and perturbation: 8 min/max + 4 add ..................... 12
      RK4: 4 evaluations of Eq. dynamics (q' 16, v' 13) = 116, three stage
           states 3 x 20 = 60, combination 10 x 5 = 50 ................ 226
      renormalisation: 8 + rsqrt + 4 ................................. 13
      costs: ctrl 16, track 9, vnorm 6, goal 9 + 9 + 16, J_col 4 ...... 69
      Kahan accumulation ............................................. 4
      second pass for the update: noise 16 + clamp 12 + 4 products ... 32
    """
    return 16 + 12 + 226 + 13 + 69 + 4 + 32


def set_workload(name: str) -> None:
    global WORKLOAD, METRIC
    WORKLOAD, METRIC = name, METRICS[name]


def rank_seed(rank: int) -> int:
    """Scene seed of a rank: every rank plans its own scene (weak scaling)."""
    return rank


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The slowest rank's time (an all-reduce of the timing only, no data path)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(P: dict, world: int, steps: int, seconds: float) -> float:
    """Whole-job rollout-steps/s: the units all ranks processed over the slowest time."""
    return world * rollout_steps(P) * steps / seconds


def env_int(name, default):
    v = os.environ.get(name)
    return int(v) if v is not None else default


def host_cores() -> dict:
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                info["model"] = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return info


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# E*K at or below which a planning step runs the split Stage I pass (four or
# more threads per sample, the update fused into its last CTAs)
SPLIT_MAX_SAMPLES = 32768


def step_percentiles(step_ms: list) -> dict:
    """p10 / p90 of the per-step device times (nearest rank)."""
    xs = sorted(step_ms)
    if not xs:
        return {}
    pick = lambda q: xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]
    return {"ms_per_step_p10": pick(0.10), "ms_per_step_p90": pick(0.90)}


def rollout_kernel_name(P: dict) -> str:
    lanes = P.get("lanes_per_sample", 0) or (4 if P["E"] * P["K"] <= SPLIT_MAX_SAMPLES else 1)
    if lanes == 4:
        return ("k_rollout_split (noise, RK4, S(1), per-CTA partials; the last CTA of each "
                "instance merges them, updates the nominal and runs Stage II)")
    return "k_rollout (fused noise + RK4 + S(1) + update partials)"


def rollout_traffic(workload: str):
    """DRAM bytes per k_rollout launch from the committed ncu summary, or None
    when the kernel's source changed since those counters were taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "k_rollout_traffic.json")
    try:
        d = json.load(open(p))
        h = hashlib.sha256()
        for f in d["source_files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != d["source_sha256"]:
            return None
        return d["workloads"][workload]["bytes_per_launch"]
    except Exception:
        return None


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            pass
    return {}


def fp32_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# --------------------------------------------------------------------------- reference arm

# wall time the reference arm aims at for its whole --steps/--warmup run
REFERENCE_BUDGET_S = 120.0


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    if WORKLOAD == "batched":
        run_reference_batched(args, O)
        return
    w = I.make_workload(WORKLOAD, seed=0)
    P = dict(w.params)
    # each step is a bounded sample of the workload: one full step calibrates
    # the oracle's time, then every step runs K' <= K samples per instance so
    # that the whole run takes about REFERENCE_BUDGET_S
    t0 = time.perf_counter()
    O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, dict(P, step_id=10**6), w.hover_nominal(), debug=False)
    t_full = time.perf_counter() - t0
    per_step = min(t_full, REFERENCE_BUDGET_S / max(1, args.warmup + args.steps))
    k_sample = max(8, min(P["K"], int(P["K"] * per_step / t_full)))
    Ps = dict(P, K=k_sample)
    u = w.hover_nominal()
    times = []
    for s in range(args.warmup + args.steps):
        Ps["step_id"] = s
        t0 = time.perf_counter()
        out = O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, Ps, u, debug=False)
        dt = time.perf_counter() - t0
        u = out["u_nom"].astype(np.float32)
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = rollout_steps(Ps) * len(times) / tot
    sample = (f"{len(times)} plan steps of the {WORKLOAD} workload with K = {k_sample} of {P['K']} "
              f"samples per instance (a full step takes {t_full:.2f} s), single-threaded FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(P, w),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_cores()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_batched(args, O):
    """The oracle over the batch's planners in turn; each step is a bounded
    sample (as many planners as fit in about 10 s, at least one)."""
    ws = I.batch_workloads(64, seed=1)
    done, tot, k = 0, 0.0, 0
    for s in range(args.warmup + args.steps):
        t_start, units, t_step = time.perf_counter(), 0, 0.0
        while units == 0 or time.perf_counter() - t_start < 10.0 / max(1, args.steps):
            w = ws[k % len(ws)]
            k += 1
            t0 = time.perf_counter()
            O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, dict(w.params, step_id=s),
                        w.hover_nominal(), debug=False)
            t_step += time.perf_counter() - t0
            units += rollout_steps(w.params)
        if s >= args.warmup:
            done, tot = done + units, tot + t_step
    val = done / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "batched: 64 planners (oracle over a bounded sample of them)",
                       "planners": len(ws)},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{k} planner steps of the batch in order, single-threaded "
                                       "FP64 oracle", "host": host_cores()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(P: dict, w) -> dict:
    return {"workload": f"{WORKLOAD}: E={P['E']} (M_h x M_v = {P['M_h']}x{P['M_v']}), K={P['K']}, "
                        f"T={P['T']}, dt={P['dt']}, iters={P['iters']}, fine {P['fine_az']}x{P['fine_el']} "
                        f"pooled {P['pool_az']}x{P['pool_el']}, refine {P.get('refine_steps', 0)} x {P.get('refine_step', 0)}, "
                        f"scene of {len(w.cloud)} points",
            "E": P["E"], "K": P["K"], "T": P["T"], "n_points": int(len(w.cloud)),
            "l2": "flushed between timed steps (512 MB write)"}


# --------------------------------------------------------------------------- CPU baseline

def cpu_baseline(w, P) -> dict:
    from oracle import oracle as O
    O.build()
    u = w.hover_nominal()
    times = []
    t_start = time.perf_counter()
    s = 0
    while time.perf_counter() - t_start < CPU_SAMPLE_SECONDS or s < 1:
        Q = dict(P, step_id=s)
        t0 = time.perf_counter()
        out = O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, Q, u, debug=False)
        times.append(time.perf_counter() - t0)
        u = out["u_nom"].astype(np.float32)
        s += 1
    tot = sum(times)
    return {"value": rollout_steps(P) * len(times) / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} full plan steps of the same workload (FP64 oracle, one thread, "
                      f"{tot:.1f} s)", "host": host_cores()}


# --------------------------------------------------------------------------- accumulation

def run_accumulate(args, rank: int, world: int, local: int):
    """Sec. IV-A.1 accumulation: per step one 20k-point sensor-frame sweep is
    pushed into a 10-frame ring (transform by its capture pose) and the 10 live
    frames (200k points) are gathered compacted in world coordinates."""
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero
    F, N = 10, 20000
    rng = np.random.default_rng(1 + rank_seed(rank))
    dev = torch.device("cuda", local)
    frames = []
    for f in range(16):
        pts = torch.from_numpy(rng.normal(0, 8, (N, 3)).astype(np.float32)).to(dev)
        q = rng.normal(size=4)
        frames.append((pts, rng.normal(0, 2, 3), q / np.linalg.norm(q)))
    acc = aero.Accumulator(F, N)
    dst = torch.empty((F * N, 3), device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for f in range(F):
        acc.push(frames[f][0], frames[f][1], frames[f][2])
    for s in range(args.warmup):
        acc.push(*frames[s % 16])
        acc.gather(dst)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            acc.push(*frames[i % 16])
            n = acc.gather(dst)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    units = N + F * N
    # end to end: the sweep copied from pinned host memory, the gathered cloud read back
    h_pts = [f[0].cpu().pin_memory() for f in frames]
    h_out = torch.empty((F * N, 3)).pin_memory()
    d_in = torch.empty((N, 3), device=dev)
    times = []
    for i in range(args.warmup + max(10, args.steps // 4)):
        stream.synchronize()
        t0 = time.perf_counter()
        d_in.copy_(h_pts[i % 16], non_blocking=True)
        acc.push(d_in, frames[i % 16][1], frames[i % 16][2])
        n = acc.gather(dst)
        h_out[:n].copy_(dst[:n], non_blocking=True)
        stream.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    e_tot = max_over_ranks(sum(times), dist, dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    avg_s = total_ms / args.steps / 1e3
    bytes_step = 24 * units      # push: 12 B read + 12 B written per slot point; gather: 12 + 12 per point
    peaks = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    line = {
        "metric": METRIC, "value": world * units * args.steps / (total_ms / 1e3), "unit": "points/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "ms_per_step_median": statistics.median(step_ms), **step_percentiles(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"accumulate: {F} frames x {N} points, push one frame + gather all",
                   "l2": "flushed between timed steps (512 MB write)"},
        "roofline": {"kernel": "k_accum_push + k_accum_gather", "bound": "hbm",
                     "achieved": bytes_step / avg_s / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": bytes_step / avg_s / 1e9 / peak, "traffic": None,
                     "bytes_per_step": bytes_step,
                     "peak_note": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback"},
        "clocks": clk.summary(),
        "e2e": {"value": world * units * len(times) / e_tot, "unit": "points/s",
                "h2d_bytes_per_step": 12 * N, "d2h_bytes_per_step": 12 * F * N,
                "ms_per_step": 1e3 * e_tot / len(times)},
        "gpu_launches": 2 * args.steps,
    }
    print(json.dumps(line), flush=True)
    acc.close()
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- batched planners

def run_batched(args, rank: int, world: int, local: int):
    """64 planners of uneven sizes (inputs.batch_workloads) per aero_batch_plan call."""
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero
    ws = I.batch_workloads(args.batch_planners, seed=1 + 1000 * rank_seed(rank))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    lim = dict(E_max=16, K_max=4096, T_max=60, fine_cells_max=128 * 64,
               n_points_max=max(len(w.cloud) for w in ws))
    batch = aero.Batch(len(ws), **lim)
    clouds = [torch.from_numpy(w.cloud).to(dev) for w in ws]
    u0 = [torch.from_numpy(w.hover_nominal()).to(dev) for w in ws]
    un = [u.clone() for u in u0]
    ub = [torch.empty((w.params["T"], 4), device=dev) for w in ws]
    cand = [torch.empty((w.params["E"],), device=dev) for w in ws]
    best = [torch.empty((1,), dtype=torch.int32, device=dev) for w in ws]
    states = [aero.state_struct(w.p0, w.q0, w.v0) for w in ws]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def items(step_id):
        out = []
        for i, w in enumerate(ws):
            w.params["step_id"] = step_id
            out.append(aero.Batch.item(states[i], clouds[i], w.goal, aero.params_struct(w.params),
                                       un[i], ub[i], cand[i], best[i]))
        return out

    plans = [items(s) for s in range(args.warmup + args.steps)]
    # one-off autotuning of the launch configuration (outside the timed region;
    # it writes only the batch's scratch buffers)
    if args.batch_config:
        q, c, d, g = (int(x) for x in args.batch_config.split(","))
        batch.set_config(q, c, d, g)
        tuned, tune_ms = batch.config(), None
    else:
        tuned, tune_ms = batch.tune(plans[0], repeats=3, stream=stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for s in range(args.warmup):
            flush.fill_(float(s))
            for a, b in zip(un, u0):
                a.copy_(b)
            batch.plan(plans[s], stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.fill_(float(i))
                for a, b in zip(un, u0):
                    a.copy_(b)
                ev[i][0].record(stream)
                batch.plan(plans[args.warmup + i], stream)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    units = sum(rollout_steps(w.params) for w in ws)

    # end to end through the batch API: pinned host inputs in, results out
    h_clouds = [torch.from_numpy(w.cloud.copy()).pin_memory() for w in ws]
    h_u0 = [torch.from_numpy(w.hover_nominal()).pin_memory() for w in ws]
    h_un = [torch.empty_like(u).pin_memory() for u in h_u0]
    h_ub = [torch.empty((w.params["T"], 4)).pin_memory() for w in ws]
    h_cand = [torch.empty((w.params["E"],)).pin_memory() for w in ws]
    h_best = [torch.empty((1,), dtype=torch.int32).pin_memory() for w in ws]
    e2e_steps = max(10, args.steps // 4)
    times = []
    for i in range(args.warmup + e2e_steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        stream.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(len(ws)):
                clouds[k].copy_(h_clouds[k], non_blocking=True)
                un[k].copy_(h_u0[k], non_blocking=True)
            batch.plan(plans[i % len(plans)], stream)
            for k in range(len(ws)):
                h_un[k].copy_(un[k], non_blocking=True)
                h_ub[k].copy_(ub[k], non_blocking=True)
                h_cand[k].copy_(cand[k], non_blocking=True)
                h_best[k].copy_(best[k], non_blocking=True)
        stream.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    e_tot = max_over_ranks(sum(times), dist, dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    flops = sum(w.params["E"] * w.params["K"] * w.params["T"] * w.params["iters"]
                for w in ws) * rollout_flops_per_step()
    achieved = flops / (total_ms / args.steps / 1e3) / 1e12
    peak = fp32_peak_tflops(measured_peaks().get("sm_max_mhz", 2070.0))
    line = {
        "metric": METRIC, "value": world * units * args.steps / (total_ms / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "ms_per_step_median": statistics.median(step_ms), **step_percentiles(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batched: {len(ws)} planners, E in {{4,8,16}}, K in {{256,1024,4096}}, "
                               "T in {20,40,60}, forest / walls with 1.5 m gaps / inclines, "
                               f"{min(len(w.cloud) for w in ws)}-{max(len(w.cloud) for w in ws)} points",
                   "planners": len(ws), "rollout_steps_per_batch": units,
                   "launch": dict(tuned, tune_ms=tune_ms),
                   "l2": "flushed between timed steps (512 MB write)"},
        "roofline": {"kernel": "the whole batched step (Stage I is the dominant launch)",
                     "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "flops_per_launch": flops, "avg_launch_ms": total_ms / args.steps,
                     "peak_note": "FP32 FMA pipes: 152 SMs x 128 lanes x 2 x 2070 MHz; whole batch step"},
        "clocks": clk.summary(),
        "e2e": {"value": world * units * len(times) / e_tot, "unit": UNIT,
                "h2d_bytes_per_step": sum(c.numel() * 4 + u.numel() * 4 for c, u in zip(h_clouds, h_u0)),
                "d2h_bytes_per_step": sum(u.numel() * 4 + b.numel() * 4 + c.numel() * 4 + 4
                                          for u, b, c in zip(h_un, h_ub, h_cand)),
                "ms_per_step": 1e3 * e_tot / len(times)},
        "gpu_launches": (4 + 2 * max(w.params["iters"] for w in ws)) * args.steps,
    }
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        done, t_cpu, t_start = 0, 0.0, time.perf_counter()
        for w in ws:
            if time.perf_counter() - t_start > CPU_SAMPLE_SECONDS and done > 0:
                break
            t0 = time.perf_counter()
            O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, w.params, w.hover_nominal(), debug=False)
            t_cpu += time.perf_counter() - t0
            done += rollout_steps(w.params)
        line["cpu_baseline"] = {"value": done / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"the batch's first planners in order, {t_cpu:.1f} s of "
                                          "FP64 oracle on one thread", "host": host_cores()}
    print(json.dumps(line), flush=True)
    batch.close()
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(METRICS))
    ap.add_argument("--batch-planners", type=int, default=64,
                    help="batched workload: number of planners (64 is the measured configuration)")
    ap.add_argument("--batch-config", default="",
                    help="batched workload: fixed launch configuration 'quad_max,ctas_per_sm,"
                         "dynamic,coarse' instead of autotuning")
    ap.add_argument("--no-stage-timing", action="store_true",
                    help="diagnostic: no per-stage events in the timed steps (no roofline)")
    args = ap.parse_args()
    set_workload(args.workload)

    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if WORKLOAD == "batched":
        run_batched(args, rank, world, local)
        return
    if WORKLOAD == "accumulate":
        run_accumulate(args, rank, world, local)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero

    w = I.make_workload(WORKLOAD, seed=rank_seed(rank))
    P = w.params
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    pl = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                      fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=len(w.cloud))
    cloud = torch.from_numpy(w.cloud).to(dev)
    u0 = torch.from_numpy(w.hover_nominal()).to(dev)
    u_nom = u0.clone()
    u_best = torch.empty((P["T"], 4), device=dev)
    cand = torch.empty((P["E"],), device=dev)
    best = torch.empty((1,), dtype=torch.int32, device=dev)
    state = aero.state_struct(w.p0, w.q0, w.v0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(s):
        P["step_id"] = s
        pl.plan_step(state, cloud, w.goal, aero.params_struct(P), u_nom, u_best, cand, best, stream)

    with torch.cuda.stream(stream):
        for s in range(args.warmup):
            flush.fill_(float(s))
            u_nom.copy_(u0)
            step(s)
        torch.cuda.synchronize()
        pl.profile_read()  # discard warm-up stage times
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        # only the dominant kernel is bracketed by events in the timed steps
        pl.profile(False if args.no_stage_timing else ["rollout"])
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.fill_(float(i))
                u_nom.copy_(u0)   # every step plans from the same warm start
                ev[i][0].record(stream)
                step(args.warmup + i)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
        pl.profile(False)
        if dist:
            dist.barrier()
        st = pl.sync_status(stream)
        if st != 0:
            raise RuntimeError(f"planner status {st}")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    stages = pl.profile_read()
    # per-stage breakdown from a separate, shorter pass (events around every stage)
    with torch.cuda.stream(stream):
        pl.profile(True)
        n_diag = min(args.steps, 50)
        for i in range(n_diag):
            flush.fill_(float(i))
            u_nom.copy_(u0)
            step(20_000 + i)
        torch.cuda.synchronize()
        pl.profile(False)
    breakdown = pl.profile_read()
    total_ms = max_over_ranks(sum(step_ms), dist, dev)

    # diagnostic: the same step captured once in a CUDA graph and replayed (no
    # host launch cost, no events between the kernels; L2 flushed before each)
    graph_ms = []
    with torch.cuda.stream(stream):
        P["step_id"] = 30_000
        ps = aero.params_struct(P)
        u_nom.copy_(u0)
        pl.plan_step(state, cloud, w.goal, ps, u_nom, u_best, cand, best, stream)
        graph = torch.cuda.CUDAGraph()
        stream.synchronize()
        graph.capture_begin()
        pl.plan_step(state, cloud, w.goal, ps, u_nom, u_best, cand, best, stream)
        graph.capture_end()
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(min(args.steps, 200))]
        for i in range(args.warmup + len(gev)):
            flush.fill_(float(i))
            u_nom.copy_(u0)
            if i >= args.warmup:
                gev[i - args.warmup][0].record(stream)
            graph.replay()
            if i >= args.warmup:
                gev[i - args.warmup][1].record(stream)
        torch.cuda.synchronize()
        graph_ms = [a.elapsed_time(b) for a, b in gev]
        del graph

    # end-to-end through the host-memory entry point (pinned buffers)
    e2e = None
    if True:
        hc = torch.from_numpy(w.cloud.copy()).pin_memory()
        hu = torch.from_numpy(w.hover_nominal()).pin_memory()
        hb = torch.empty((P["T"], 4)).pin_memory()
        hcand = torch.empty((P["E"],)).pin_memory()
        hbest = torch.empty((1,), dtype=torch.int32).pin_memory()
        e2e_steps = max(20, args.steps // 2)
        times = []
        ps = aero.params_struct(P)  # marshalled once; only the step counter changes
        h0 = torch.from_numpy(w.hover_nominal())
        for i in range(args.warmup + e2e_steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            stream.synchronize()
            hu.copy_(h0)
            ps.step_id = 10_000 + i
            t0 = time.perf_counter()
            pl.plan_step_host(state, hc, w.goal, ps, hu, hb, hcand, hbest, stream)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                times.append(dt)
        e_tot = max_over_ranks(sum(times), dist, dev)
        e2e = {"value": job_value(P, world, len(times), e_tot), "unit": UNIT,
               "h2d_bytes_per_step": hc.numel() * 4 + hu.numel() * 4,
               "d2h_bytes_per_step": hu.numel() * 4 + hb.numel() * 4 + hcand.numel() * 4 + 4,
               "ms_per_step": 1e3 * e_tot / len(times)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    value = job_value(P, world, args.steps, total_ms / 1e3)
    clocks = clk.summary()
    peaks = measured_peaks()
    r_ms, r_n = stages["rollout"]
    r_avg_ms = r_ms / max(r_n, 1)
    flops = P["E"] * P["K"] * P["T"] * rollout_flops_per_step()
    achieved = flops / (r_avg_ms / 1e3) / 1e12 if r_avg_ms > 0 else 0.0
    peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    launches = args.steps * sum(n for _, n in breakdown.values()) // max(n_diag, 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "ms_per_step_median": statistics.median(step_ms), **step_percentiles(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(P, w),
        "stage_ms_per_step": {k: v[0] / n_diag for k, v in breakdown.items()},
        "graph_replay": {"ms_per_step_median": statistics.median(graph_ms) if graph_ms else None,
                         "steps": len(graph_ms),
                         "note": "diagnostic: one step captured in a CUDA graph and replayed, "
                                 "L2 flushed before each replay; not the headline value"},
        "roofline": {"kernel": rollout_kernel_name(P),
                     "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": rollout_traffic(WORKLOAD),
                     "flops_per_launch": flops, "avg_launch_ms": r_avg_ms,
                     "flops_note": "Stage I only (noise, RK4, S(1)); the launch time also "
                                   "covers what the kernel fuses",
                     "peak_note": "FP32 FMA pipes: 152 SMs x 128 lanes x 2 x 2070 MHz (max SM clock)"},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, P)
    print(json.dumps(line), flush=True)
    pl.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
