"""Benchmark of the AERO-MPPI planning step on GB300 (prints ONE JSON line).

A "step" is one pass of the whole hot path over one synthetic scene: fine
partition and collision grid, coarse argmax, anchors, quintic guides, the E x K
x T sampled rollouts with their Stage I costs, the softmax-weighted update, the
Stage II re-rollout and the selection.

The headline workload is the large-clutter ensemble (E=32, K=8192, T=64,
dt=0.03, 200,000 points merged from three LiDAR sweeps), the largest planning
step that fits one GPU.  The same line carries, under "forms", the other
forms of the step measured on the same GPU in the same run: the anchor-guided
ensemble (E=8, K=1024, T=40), the plain single MPPI (E=1, K=256, T=20), the
ensemble with 5 gradient-refinement steps, the large clutter with every kept
point as collision set, and 64 independent planners in one batched call.

Metric: rollout-steps per second = (E K T iters + E T) / step time.  Each timed
step is bracketed by CUDA events on the planner's stream; L2 (129 MB) is
flushed by writing a 512 MB buffer between timed steps, outside the events.
Every step plans from the same state and hover warm start (a fresh Philox
step_id each time), so the timed work does not drift with the step index.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload large|ensemble|plain|refined|batched|accumulate|partition_sweep]

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

WORKLOAD = "large"
METRICS = {"large": "rollout-steps/s (large-clutter ensemble plan step)",
           "ensemble": "rollout-steps/s (anchor-guided ensemble plan step)",
           "plain": "rollout-steps/s (plain single-MPPI plan step)",
           "batched": "rollout-steps/s (64 independent planners in one batched call)",
           "refined": "rollout-steps/s (ensemble plan step with 5 gradient-refinement steps)",
           "accumulate": "points/s (LiDAR frame push + 10-frame gather)",
           "partition_sweep": "points/s (fine partition of the cloud: cone keys and per-cone minimum)"}
METRIC = METRICS[WORKLOAD]
UNIT = "rollout-steps/s"
CPU_SAMPLE_SECONDS = 10.0
# the forms measured beside the headline, in the same line
FORMS = ["ensemble", "plain", "refined", "large_raw", "batched"]
# parity bar each form is held to by the GPU test suite
FORM_PARITY = {
    "large": "S(2) of every instance within 1e-4 relative and the selected index equal to the "
             "FP64 oracle's; updated controls within 1e-4 absolute (tests/test_gpu_parity.py)",
    "ensemble": "per-sample S(1) and S(2) within 1e-4 relative, updated controls within 1e-4 "
                "absolute, partition/anchor/selection indices bit-exact (tests/test_gpu_parity.py)",
    "plain": "as ensemble (tests/test_gpu_parity.py)",
    "refined": "S(2) of the refined nominals within 1e-4 relative of the oracle's S(2) of the same "
               "nominals; the refinement within 1e-4 of the oracle's refinement of the GPU's "
               "pre-refinement nominal (tests/test_gpu_adjoint.py)",
    "large_raw": "as large, with every kept point as collision set (tests/test_gpu_parity.py)",
    "batched": "per planner: decisions equal to the single planner's, S(2) within 1e-4 relative "
               "of the oracle (tests/test_gpu_batch.py)",
}


def rollout_steps(P: dict) -> int:
    return P["E"] * P["K"] * P["T"] * P["iters"] + P["E"] * P["T"]


def rollout_flops_per_step() -> int:
    """Algorithmic FP32 flops of one sample-step of Stage I (counted from the
    formulas of the method, each computed once; FMA = 2, nearest-point
    distance tests excluded):
      noise: Box-Muller 2 x (log, sqrt, sincos) + 4 scalings + 4 adds ... 16
      clamp and perturbation: 8 min/max + 4 add ..................... 12
      RK4: 4 evaluations of Eq. dynamics (q' 16, v' 13) = 116, three stage
           states 3 x 20 = 60, combination 10 x 5 = 50 ................ 226
      renormalisation: 8 + rsqrt + 4 ................................. 13
      costs: ctrl 16, track 9, vnorm 6, goal 9 + 9 + 16, J_col 4 ...... 69
      accumulation of S^(1) .......................................... 1
      weighted sum of the update, w_k du_k over 4 components .......... 8
    Work an implementation adds (regenerating perturbations instead of
    storing them, exponentials of the weights) is not counted."""
    return 16 + 12 + 226 + 13 + 69 + 1 + 8


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
    """nvidia-smi clock / throttle / utilisation samples (read-only queries).

    Started before the first GPU work of the run and stopped after the last,
    so that it covers every GPU-busy pass (warm-up, timed steps, graph replay,
    the end-to-end pass and the other forms), which together last seconds."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.t = None

    def start(self, wait_s: float = 5.0):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < wait_s and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.proc = None

    def __enter__(self):
        return self.start()

    def __exit__(self, *a):
        self.stop()

    def summary(self) -> dict:
        return clock_summary(self.lines)


def clock_summary(lines) -> dict:
    """Median SM clock over the samples taken under load (utilisation >= 50%,
    all samples if none), the maximum clock, and every throttle reason seen."""
    all_sm, busy_sm, mx, reasons, power = [], [], None, set(), []
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 10:
            continue
        try:
            sm, mx_i = float(f[1]), float(f[2])
        except ValueError:
            continue
        mx = mx_i
        all_sm.append(sm)
        try:
            util = float(f[4])
        except ValueError:
            util = 0.0
        if util >= 50.0:
            busy_sm.append(sm)
        try:
            power.append(float(f[3]))
        except ValueError:
            pass
        for n, v in zip(ClockSampler.REASONS, f[6:10]):
            if v.lower() == "active":
                reasons.add(n)
    sm = busy_sm if busy_sm else all_sm
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
            "reasons": sorted(reasons), "samples": len(all_sm), "samples_under_load": len(busy_sm),
            "power_w_max": max(power) if power else None}


def step_percentiles(step_ms: list) -> dict:
    """p10 / p90 of the per-step device times (nearest rank)."""
    xs = sorted(step_ms)
    if not xs:
        return {}
    pick = lambda q: xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]
    return {"ms_per_step_p10": pick(0.10), "ms_per_step_p90": pick(0.90)}


# E*K at or below which a planning step runs the split Stage I pass (four or
# more threads per sample, the update fused into its last CTAs)
SPLIT_MAX_SAMPLES = 32768


def rollout_kernel_name(P: dict) -> str:
    lanes = P.get("lanes_per_sample", 0) or (4 if P["E"] * P["K"] <= SPLIT_MAX_SAMPLES else 1)
    if lanes == 4:
        return ("k_rollout_split (noise, RK4, S(1), per-CTA partials; the last CTA of each "
                "instance merges them, updates the nominal and runs Stage II)")
    return "k_rollout (fused noise + RK4 + S(1) + update partials)"


def rollout_traffic(workload: str):
    """DRAM bytes per Stage I launch from the committed ncu summary, or None
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


def fp32_peak_tflops(sm_mhz: float, sms: int) -> float:
    """SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def device_sms(dev) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def peak_info(dev) -> tuple[float, str]:
    peaks = measured_peaks()
    sms = device_sms(dev)
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    src = "MEASURED_PEAKS.json sm_max_mhz" if "sm_max_mhz" in peaks else "nominal maximum SM clock"
    return fp32_peak_tflops(mhz, sms), (f"FP32 FMA pipes: {sms} SMs (queried from the device) x 128 "
                                        f"lanes x 2 flops x {mhz:.0f} MHz ({src})")


# --------------------------------------------------------------------------- CPU oracle timing

def oracle_bounded(w, P: dict, budget_s: float, threads: int, O) -> dict:
    """The FP64 oracle on a bounded sample of the workload: every instance with
    K' <= K samples (all T steps, the whole step around them: partition,
    anchors, guides, update, Stage II), K' sized so the run takes about
    budget_s.  Returns throughput in rollout-steps/s of the sample."""
    used = O.set_threads(threads)
    u = w.hover_nominal()
    E, T = P["E"], P["T"]
    k_try = max(1, min(P["K"], 2 * used))
    t0 = time.perf_counter()
    O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, dict(P, K=k_try, step_id=10**6), u, debug=False)
    t_try = time.perf_counter() - t0
    k_s = max(1, min(P["K"], int(k_try * budget_s / max(t_try, 1e-6))))
    Ps = dict(P, K=k_s)
    times, s, t_start = [], 0, time.perf_counter()
    while s < 1 or time.perf_counter() - t_start < budget_s:
        Ps["step_id"] = s
        t0 = time.perf_counter()
        O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, Ps, u, debug=False)
        times.append(time.perf_counter() - t0)
        s += 1
    tot = sum(times)
    O.set_threads(1)
    return {"value": rollout_steps(Ps) * len(times) / tot, "threads": used, "steps": len(times),
            "K_sample": k_s, "seconds": tot}


def cpu_baseline(w, P) -> dict:
    """The oracle as it stands on the host cores, one thread and all threads
    (OpenMP over the samples of an instance), each on a bounded sample."""
    from oracle import oracle as O
    O.build()
    one = oracle_bounded(w, P, CPU_SAMPLE_SECONDS, 1, O)
    allc = oracle_bounded(w, P, CPU_SAMPLE_SECONDS, os.cpu_count() or 1, O)
    return {"value": allc["value"], "unit": UNIT, "cores": allc["threads"], "kind": "oracle",
            "value_1core": one["value"], "value_all_cores": allc["value"],
            "sample": (f"FP64 oracle plan steps of the same workload with every instance and K' of "
                       f"{P['K']} samples each: {one['steps']} steps of K'={one['K_sample']} on one "
                       f"thread ({one['seconds']:.1f} s), {allc['steps']} steps of K'={allc['K_sample']} "
                       f"on {allc['threads']} threads ({allc['seconds']:.1f} s)"),
            "host": host_cores()}


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
    if WORKLOAD in ("accumulate", "partition_sweep"):
        print(json.dumps({"impl": "reference", "unavailable": f"the {WORKLOAD} workload has no "
                          "oracle timing arm"}), flush=True)
        return
    w = I.make_workload(WORKLOAD, seed=0)
    P = dict(w.params)
    threads = O.set_threads(os.cpu_count() or 1)
    # each step is a bounded sample of the workload: a short calibration step,
    # then every step runs K' <= K samples per instance so that the whole run
    # takes about REFERENCE_BUDGET_S
    per_step = args.reference_budget / max(1, args.warmup + args.steps)
    k_try = max(1, min(P["K"], 2 * threads))
    t0 = time.perf_counter()
    O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, dict(P, K=k_try, step_id=10**6), w.hover_nominal(),
                debug=False)
    t_try = time.perf_counter() - t0
    k_sample = max(1, min(P["K"], int(k_try * per_step / max(t_try, 1e-6))))
    Ps = dict(P, K=k_sample)
    u = w.hover_nominal()
    times = []
    for s in range(args.warmup + args.steps):
        Ps["step_id"] = s
        t0 = time.perf_counter()
        O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, Ps, u, debug=False)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = rollout_steps(Ps) * len(times) / tot
    sample = (f"{len(times)} plan steps of the {WORKLOAD} workload with every instance and K = "
              f"{k_sample} of {P['K']} samples each, FP64 oracle, OpenMP over samples on {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(P, w),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample, "host": host_cores()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_batched(args, O):
    """The oracle over the batch's planners in turn; each step is a bounded
    sample (as many planners as fit in about 10 s, at least one)."""
    ws = I.batch_workloads(64, seed=1)
    threads = O.set_threads(os.cpu_count() or 1)
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
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{k} planner steps of the batch in order, FP64 oracle, "
                                       f"OpenMP over samples on {threads} threads",
                             "host": host_cores()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(P: dict, w, name: str = None) -> dict:
    name = name or WORKLOAD
    raw = " every kept point as collision set," if P.get("collision_set", 0) == 1 else ""
    return {"workload": f"{name}: E={P['E']} (M_h x M_v = {P['M_h']}x{P['M_v']}), K={P['K']}, "
                        f"T={P['T']}, dt={P['dt']}, iters={P['iters']}, fine {P['fine_az']}x{P['fine_el']} "
                        f"pooled {P['pool_az']}x{P['pool_el']}, r_max={P['r_max']},{raw} refine "
                        f"{P.get('refine_steps', 0)} x {P.get('refine_step', 0)}, scene of {len(w.cloud)} points",
            "E": P["E"], "K": P["K"], "T": P["T"], "n_points": int(len(w.cloud)),
            "l2": "flushed between timed steps (512 MB write)"}


# --------------------------------------------------------------------------- single-planner runs

class PlannerRun:
    """One planner on one workload: the timed steps, a per-stage breakdown, a
    CUDA-graph replay and the end-to-end pass through the host-buffer call."""

    def __init__(self, aero, name: str, seed: int, dev, stream, flush, raw: bool = False):
        import torch
        self.torch = torch
        self.aero = aero
        self.name = name
        base = "large" if name == "large_raw" else name
        self.w = I.make_workload(base, seed=seed)
        self.P = self.w.params
        if raw:
            self.P["collision_set"] = 1
        P, w = self.P, self.w
        self.dev, self.stream, self.flush = dev, stream, flush
        self.pl = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                               fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=len(w.cloud),
                               raw_points_max=0 if raw else -1)
        self.cloud = torch.from_numpy(w.cloud).to(dev)
        self.u0 = torch.from_numpy(w.hover_nominal()).to(dev)
        self.u_nom = self.u0.clone()
        self.u_best = torch.empty((P["T"], 4), device=dev)
        self.cand = torch.empty((P["E"],), device=dev)
        self.best = torch.empty((1,), dtype=torch.int32, device=dev)
        self.state = aero.state_struct(w.p0, w.q0, w.v0)

    def step(self, s):
        self.P["step_id"] = s
        self.pl.plan_step(self.state, self.cloud, self.w.goal, self.aero.params_struct(self.P),
                          self.u_nom, self.u_best, self.cand, self.best, self.stream)

    def timed(self, steps: int, warmup: int, dist=None, stage_events: bool = True) -> dict:
        """Per-step device times (events around each step) and the average
        Stage I launch time (events around the Stage I launch of every step)."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            for s in range(warmup):
                self.flush.fill_(float(s))
                self.u_nom.copy_(self.u0)
                self.step(s)
            torch.cuda.synchronize()
            self.pl.profile_read()  # discard warm-up stage times
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            # only the dominant kernel is bracketed by events in the timed steps
            self.pl.profile(["rollout"] if stage_events else False)
            for i in range(steps):
                self.flush.fill_(float(i))
                self.u_nom.copy_(self.u0)   # every step plans from the same warm start
                ev[i][0].record(self.stream)
                self.step(warmup + i)
                ev[i][1].record(self.stream)
            torch.cuda.synchronize()
            self.pl.profile(False)
            if dist:
                dist.barrier()
            st = self.pl.sync_status(self.stream)
            if st != 0:
                raise RuntimeError(f"planner status {st} ({self.name})")
        step_ms = [a.elapsed_time(b) for a, b in ev]
        stages = self.pl.profile_read()
        r_ms, r_n = stages["rollout"]
        return {"step_ms": step_ms, "rollout_avg_ms": r_ms / max(r_n, 1) if r_n else None}

    def breakdown(self, n: int) -> tuple[dict, int]:
        """Stage times per step (events around every stage) and launches per step."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            self.pl.profile(True)
            for i in range(n):
                self.flush.fill_(float(i))
                self.u_nom.copy_(self.u0)
                self.step(20_000 + i)
            torch.cuda.synchronize()
            self.pl.profile(False)
        b = self.pl.profile_read()
        launches = sum(v[1] for v in b.values()) // max(n, 1)
        return {k: v[0] / n for k, v in b.items()}, launches

    def graph_replay(self, n: int, warmup: int) -> list:
        """The step captured once in a CUDA graph and replayed (L2 flushed before each)."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            self.P["step_id"] = 30_000
            ps = self.aero.params_struct(self.P)
            self.u_nom.copy_(self.u0)
            self.pl.plan_step(self.state, self.cloud, self.w.goal, ps, self.u_nom, self.u_best,
                              self.cand, self.best, self.stream)
            graph = torch.cuda.CUDAGraph()
            self.stream.synchronize()
            graph.capture_begin()
            self.pl.plan_step(self.state, self.cloud, self.w.goal, ps, self.u_nom, self.u_best,
                              self.cand, self.best, self.stream)
            graph.capture_end()
            gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(n)]
            for i in range(warmup + n):
                self.flush.fill_(float(i))
                self.u_nom.copy_(self.u0)
                if i >= warmup:
                    gev[i - warmup][0].record(self.stream)
                graph.replay()
                if i >= warmup:
                    gev[i - warmup][1].record(self.stream)
            torch.cuda.synchronize()
            del graph
        return [a.elapsed_time(b) for a, b in gev]

    def e2e(self, n: int, warmup: int, dist=None) -> dict:
        """End to end through the C-ABI call aero_plan_step_host: pinned host
        cloud and warm start in, nominals, best sequence, costs and index out,
        every step.  The call's arguments are marshalled once (only the step
        counter in the parameter struct changes); the timed region is the
        call itself, which returns when the outputs are in the host buffers."""
        import ctypes as C
        torch = self.torch
        P, w = self.P, self.w
        hc = torch.from_numpy(w.cloud.copy()).pin_memory()
        hu = torch.from_numpy(w.hover_nominal()).pin_memory()
        hb = torch.empty((P["T"], 4)).pin_memory()
        hcand = torch.empty((P["E"],)).pin_memory()
        hbest = torch.empty((1,), dtype=torch.int32).pin_memory()
        times = []
        ps = self.aero.params_struct(P)
        h0 = torch.from_numpy(w.hover_nominal())
        goal = (C.c_float * 3)(*[float(x) for x in w.goal])
        call = self.aero.lib().aero_plan_step_host
        args = (self.pl.handle, C.byref(self.state), hc.data_ptr(), hc.shape[0], goal, C.byref(ps),
                hu.data_ptr(), hb.data_ptr(), hcand.data_ptr(), hbest.data_ptr(),
                self.stream.cuda_stream)
        for i in range(warmup + n):
            with torch.cuda.stream(self.stream):
                self.flush.fill_(float(i))
            self.stream.synchronize()
            hu.copy_(h0)
            ps.step_id = 10_000 + i
            t0 = time.perf_counter()
            rc = call(*args)
            dt = time.perf_counter() - t0
            if rc != 0:
                raise RuntimeError(f"aero_plan_step_host returned {rc}")
            if i >= warmup:
                times.append(dt)
        e_tot = max_over_ranks(sum(times), dist, self.dev)
        return {"seconds": e_tot, "steps": len(times),
                "h2d_bytes_per_step": hc.numel() * 4 + hu.numel() * 4,
                "d2h_bytes_per_step": hu.numel() * 4 + hb.numel() * 4 + hcand.numel() * 4 + 4}

    def close(self):
        self.pl.close()


def stage1_roofline(P: dict, r_avg_ms, peak: float) -> dict:
    flops = P["E"] * P["K"] * P["T"] * P["iters"] * rollout_flops_per_step()
    # the iterations' Stage I launches are averaged; flops are per launch
    flops_launch = P["E"] * P["K"] * P["T"] * rollout_flops_per_step()
    achieved = flops_launch / (r_avg_ms / 1e3) / 1e12 if r_avg_ms else 0.0
    return {"achieved": achieved, "frac": achieved / peak, "flops_per_launch": flops_launch,
            "flops_per_step": flops, "avg_launch_ms": r_avg_ms}


def form_summary(run: PlannerRun, steps: int, warmup: int, peak: float) -> dict:
    t = run.timed(steps, warmup)
    ms = t["step_ms"]
    P = run.P
    rl = stage1_roofline(P, t["rollout_avg_ms"], peak)
    return {"workload": config_of(P, run.w, run.name)["workload"], "steps": steps, "warmup": warmup,
            "ms_per_step": sum(ms) / len(ms), "ms_per_step_median": statistics.median(ms),
            "rollout_steps_per_s": rollout_steps(P) * len(ms) / (sum(ms) / 1e3),
            "stage1_kernel": rollout_kernel_name(P), "stage1_ms": t["rollout_avg_ms"],
            "stage1_fp32_frac": rl["frac"], "parity": FORM_PARITY.get(run.name, "")}


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
    clk = ClockSampler(local).start()
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
    clk.stop()
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
                     "peak_note": "of measured copy bandwidth" if "hbm_gbs" in peaks else "of fallback"},
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


# --------------------------------------------------------------------------- partition sweep

SWEEP_SIZES = [10**5, 10**6, 10**7, 10**8]


def partition_sweep_cloud(n: int, seed: int, dev):
    """n points uniform in a 40 m cube around the start (2, 0, 2) (seeded,
    generated on the device): nearly every point lies within r_max = 35 m, so
    the partition keeps it and takes its cone's minimum."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(1000 + seed)
    c = torch.rand((n, 3), generator=g, device=dev, dtype=torch.float32) * 40.0 - 20.0
    c += torch.tensor([2.0, 0.0, 2.0], device=dev)
    return c


def partition_sweep(aero, dev, stream, flush, sizes, steps: int, warmup: int, seed: int = 0) -> list:
    """k_partition and the three grid launches timed with CUDA events (the
    planner's stage events) on clouds of the given sizes; the rest of the step
    is a one-sample, one-step planner (E=1, K=32, T=1)."""
    import torch
    w = I.make_workload("large", seed=seed)
    P = dict(w.params, E=1, M_h=1, M_v=1, K=32, T=1, r_max=35.0, collision_set=0)
    p0 = np.array([2.0, 0.0, 2.0], np.float32)
    out = []
    for n in sizes:
        cloud = partition_sweep_cloud(n, seed, dev)
        pl = aero.Planner(E_max=1, K_max=32, T_max=1, fine_cells_max=P["fine_az"] * P["fine_el"],
                          n_points_max=n, raw_points_max=-1)
        u0 = torch.from_numpy(np.tile(np.array([P["mass"] * P["g"], 0, 0, 0], np.float32), (1, 1, 1))).to(dev)
        un, ub = u0.clone(), torch.empty((1, 4), device=dev)
        cand, best = torch.empty((1,), device=dev), torch.empty((1,), dtype=torch.int32, device=dev)
        state = aero.state_struct(p0, w.q0, np.zeros(3, np.float32))
        with torch.cuda.stream(stream):
            def step(s):
                P["step_id"] = s
                pl.plan_step(state, cloud, w.goal, aero.params_struct(P), un, ub, cand, best, stream)
            for s in range(warmup):
                flush.fill_(float(s))
                step(s)
            torch.cuda.synchronize()
            pl.profile_read()
            pl.profile(["partition", "grid"])
            for i in range(steps):
                flush.fill_(float(i))
                step(warmup + i)
            torch.cuda.synchronize()
            pl.profile(False)
            st = pl.sync_status(stream)
            if st != 0:
                raise RuntimeError(f"planner status {st} (partition sweep, {n} points)")
        b = pl.profile_read()
        part_ms = b["partition"][0] / steps
        grid_ms = b["grid"][0] / steps
        cells = P["fine_az"] * P["fine_el"]
        # algorithmic bytes: the cloud read once (12 B/pt), the fine keys
        # filled (8 B/cone) and merged (8 B/cone written)
        alg = 12 * n + 16 * cells
        out.append({"n_points": n, "partition_ms": part_ms, "grid_ms": grid_ms,
                    "partition_points_per_s": n / (part_ms / 1e3),
                    "partition_bytes": alg, "partition_gbs": alg / (part_ms / 1e3) / 1e9})
        pl.close()
        del cloud
        torch.cuda.empty_cache()
    return out


def run_partition_sweep(args, rank: int, world: int, local: int):
    import torch
    torch.cuda.set_device(local)
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sizes = ([int(x) for x in args.sweep_sizes.split(",")] if args.sweep_sizes else
             [n for n in SWEEP_SIZES if n <= args.sweep_max])
    clk = ClockSampler(local).start()
    rows = partition_sweep(aero, dev, stream, flush, sizes, args.steps, args.warmup, rank_seed(rank))
    clk.stop()
    if rank != 0:
        return
    peaks = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    top = rows[-1]
    line = {
        "metric": METRIC, "value": world * top["partition_points_per_s"], "unit": "points/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": top["partition_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"partition_sweep: fine 256x64 cones, r_max 35 m, uniform clouds in a "
                               f"40 m cube; value at {top['n_points']} points",
                   "l2": "flushed between timed steps (512 MB write)"},
        "roofline": {"kernel": "k_partition (with the fine-key fill)", "bound": "hbm",
                     "achieved": top["partition_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": top["partition_gbs"] / peak, "traffic": None,
                     "bytes_per_launch": top["partition_bytes"],
                     "peak_note": "of measured copy bandwidth" if "hbm_gbs" in peaks else "of fallback"},
        "sweep": rows,
        "clocks": clk.summary(),
        "gpu_launches": 5 * args.steps * len(rows),
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- batched planners

def bench_batched(aero, args, dev, stream, flush, rank: int, dist=None) -> dict:
    """64 planners of uneven sizes (inputs.batch_workloads) per aero_batch_plan
    call: autotuned launch configuration, timed calls, the end-to-end pass."""
    import torch
    ws = I.batch_workloads(args.batch_planners, seed=1 + 1000 * rank_seed(rank))
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
        batch.set_config(*(int(x) for x in args.batch_config.split(",")))
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
        for i in range(args.steps):
            flush.fill_(float(i))
            for a, b in zip(un, u0):
                a.copy_(b)
            ev[i][0].record(stream)
            batch.plan(plans[args.warmup + i], stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if batch.sync_status() != 0:
        raise RuntimeError("batched planner status")
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
    batch.close()
    flops = sum(w.params["E"] * w.params["K"] * w.params["T"] * w.params["iters"]
                for w in ws) * rollout_flops_per_step()
    return {"ws": ws, "step_ms": step_ms, "total_ms": total_ms, "units": units, "tuned": tuned,
            "tune_ms": tune_ms, "flops": flops, "e2e_s": e_tot, "e2e_steps": len(times),
            "h2d": sum(c.numel() * 4 + u.numel() * 4 for c, u in zip(h_clouds, h_u0)),
            "d2h": sum(u.numel() * 4 + b.numel() * 4 + c.numel() * 4 + 4
                       for u, b, c in zip(h_un, h_ub, h_cand)),
            "launches": 4 + 2 * max(w.params["iters"] for w in ws)}


def batched_description(r: dict) -> str:
    ws = r["ws"]
    return (f"batched: {len(ws)} planners, E in {{4,8,16}}, K in {{256,1024,4096}}, T in {{20,40,60}}, "
            f"forest / walls with 1.5 m gaps / inclines, {min(len(w.cloud) for w in ws)}-"
            f"{max(len(w.cloud) for w in ws)} points")


def run_batched(args, rank: int, world: int, local: int):
    """The batched call as the headline of its own line."""
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clk = ClockSampler(local).start()
    r = bench_batched(aero, args, dev, stream, flush, rank, dist)
    clk.stop()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    ws = r["ws"]
    peak, peak_note = peak_info(dev)
    achieved = r["flops"] / (r["total_ms"] / args.steps / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": world * r["units"] * args.steps / (r["total_ms"] / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["total_ms"] / args.steps, "ms_per_step_median": statistics.median(r["step_ms"]),
        **step_percentiles(r["step_ms"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": batched_description(r), "planners": len(ws),
                   "rollout_steps_per_batch": r["units"],
                   "launch": dict(r["tuned"], tune_ms=r["tune_ms"]),
                   "l2": "flushed between timed steps (512 MB write)"},
        "roofline": {"kernel": "the whole batched step (Stage I is the dominant launch)",
                     "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "flops_per_launch": r["flops"], "avg_launch_ms": r["total_ms"] / args.steps,
                     "peak_note": peak_note + "; whole batch step"},
        "clocks": clk.summary(),
        "e2e": {"value": world * r["units"] * r["e2e_steps"] / r["e2e_s"], "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                "ms_per_step": 1e3 * r["e2e_s"] / r["e2e_steps"]},
        "gpu_launches": r["launches"] * args.steps,
    }
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        threads = O.set_threads(os.cpu_count() or 1)
        done, t_cpu, t_start = 0, 0.0, time.perf_counter()
        for w in ws:
            if time.perf_counter() - t_start > CPU_SAMPLE_SECONDS and done > 0:
                break
            t0 = time.perf_counter()
            O.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, w.params, w.hover_nominal(), debug=False)
            t_cpu += time.perf_counter() - t0
            done += rollout_steps(w.params)
        O.set_threads(1)
        line["cpu_baseline"] = {"value": done / t_cpu, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"the batch's first planners in order, {t_cpu:.1f} s of "
                                          f"FP64 oracle, OpenMP over samples on {threads} threads",
                                "host": host_cores()}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(METRICS))
    ap.add_argument("--forms", default=",".join(FORMS),
                    help="forms measured beside the headline workload (comma list; '' for none)")
    ap.add_argument("--form-steps", type=int, default=0,
                    help="timed steps of each form (default: max(--steps, 50))")
    ap.add_argument("--batch-planners", type=int, default=64,
                    help="batched workload: number of planners (64 is the measured configuration)")
    ap.add_argument("--batch-config", default="",
                    help="batched workload: fixed launch configuration 'quad_max,ctas_per_sm,"
                         "dynamic,coarse[,samples_per_cta]' instead of autotuning")
    ap.add_argument("--reference-budget", type=float, default=REFERENCE_BUDGET_S,
                    help="reference arm: wall seconds its whole run aims at")
    ap.add_argument("--sweep-max", type=int, default=10**8,
                    help="partition_sweep: largest cloud size")
    ap.add_argument("--sweep-sizes", default="",
                    help="partition_sweep: cloud sizes (comma list) instead of 1e5 .. --sweep-max")
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
    if WORKLOAD == "partition_sweep":
        run_partition_sweep(args, rank, world, local)
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

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peak, peak_note = peak_info(dev)
    # the clock record covers every GPU-busy pass of the run
    clk = ClockSampler(local).start()
    run = PlannerRun(aero, WORKLOAD, rank_seed(rank), dev, stream, flush)
    P, w = run.P, run.w
    t = run.timed(args.steps, args.warmup, dist, stage_events=not args.no_stage_timing)
    step_ms = t["step_ms"]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    n_diag = min(args.steps, 50)
    breakdown, launches_per_step = run.breakdown(n_diag)
    graph_ms = run.graph_replay(min(args.steps, 200), args.warmup)
    e2e_steps = max(20, args.steps // 2)
    e = run.e2e(e2e_steps, args.warmup, dist)
    run.close()

    forms = {}
    form_steps = args.form_steps or max(args.steps, 50)
    names = [f for f in args.forms.split(",") if f and f != WORKLOAD]
    for name in names:
        if name == "batched":
            fa = argparse.Namespace(**vars(args))
            fa.steps, fa.warmup = form_steps, max(args.warmup, 3)
            r = bench_batched(aero, fa, dev, stream, flush, rank, dist)
            forms[name] = {"workload": batched_description(r), "steps": fa.steps, "warmup": fa.warmup,
                           "ms_per_step": r["total_ms"] / fa.steps,
                           "ms_per_step_median": statistics.median(r["step_ms"]),
                           "rollout_steps_per_s": r["units"] * fa.steps / (r["total_ms"] / 1e3),
                           "whole_step_fp32_frac": r["flops"] / (r["total_ms"] / fa.steps / 1e3) / 1e12 / peak,
                           "launch": dict(r["tuned"], tune_ms=r["tune_ms"]),
                           "parity": FORM_PARITY["batched"]}
            continue
        fr = PlannerRun(aero, name, rank_seed(rank), dev, stream, flush, raw=name == "large_raw")
        forms[name] = form_summary(fr, form_steps, max(args.warmup, 3), peak)
        fr.close()
    clk.stop()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    value = job_value(P, world, args.steps, total_ms / 1e3)
    rl = stage1_roofline(P, t["rollout_avg_ms"], peak)
    forms = {WORKLOAD: {"workload": config_of(P, w)["workload"], "steps": args.steps,
                        "ms_per_step": total_ms / args.steps,
                        "ms_per_step_median": statistics.median(step_ms),
                        "rollout_steps_per_s": value / world, "stage1_kernel": rollout_kernel_name(P),
                        "stage1_ms": t["rollout_avg_ms"], "stage1_fp32_frac": rl["frac"],
                        "parity": FORM_PARITY.get(WORKLOAD, "")}, **forms}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "ms_per_step_median": statistics.median(step_ms), **step_percentiles(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": config_of(P, w),
        "stage_ms_per_step": breakdown,
        "graph_replay": {"ms_per_step_median": statistics.median(graph_ms) if graph_ms else None,
                         "steps": len(graph_ms),
                         "note": "diagnostic: one step captured in a CUDA graph and replayed, "
                                 "L2 flushed before each replay; not the headline value"},
        "roofline": {"kernel": rollout_kernel_name(P),
                     "bound": "alu", "achieved": rl["achieved"], "peak": peak, "unit": "TFLOP/s",
                     "frac": rl["frac"], "traffic": rollout_traffic(WORKLOAD),
                     "flops_per_launch": rl["flops_per_launch"], "avg_launch_ms": rl["avg_launch_ms"],
                     "flops_note": "Stage I only (noise, RK4, S(1)); the launch time also "
                                   "covers what the kernel fuses",
                     "peak_note": peak_note},
        "clocks": clk.summary(),
        "e2e": {"value": job_value(P, world, e["steps"], e["seconds"]), "unit": UNIT,
                "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                "d2h_bytes_per_step": e["d2h_bytes_per_step"],
                "ms_per_step": 1e3 * e["seconds"] / e["steps"]},
        "gpu_launches": launches_per_step * args.steps,
        "forms": forms,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, P)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
