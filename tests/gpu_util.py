"""Shared helpers of the GPU parity tests: run one planning step through the
C-ABI (CUDA path) and read back its debug buffers."""
from __future__ import annotations

import numpy as np
import torch

# Tolerances, FP32 GPU against the FP64 oracle.
TOL_POS = 1e-4        # m
TOL_QUAT = 1e-5
TOL_VEL = 1e-4        # m/s
TOL_COST_REL = 1e-4   # relative
TOL_U = 1e-4          # absolute, updated controls
TOL_DELTA = 1e-5      # absolute, perturbations (normals scaled by sigma)
JUMP_BAND = 1e-5      # m: samples with an oracle distance this close to d_min or d_max
                      # sit on a jump of J_col and are compared by membership only


def make_planner(aero, E=64, K=8192, T=64, cells=512 * 64, n=1 << 18, D=8):
    return aero.Planner(E_max=E, K_max=K, T_max=T, fine_cells_max=cells, n_points_max=n,
                        debug_samples_max=D)


def run_gpu(aero, planner, w, P: dict, u0: np.ndarray, cloud=None, debug=True) -> dict:
    """One step on the GPU; returns outputs and (optionally) debug buffers."""
    cloud = w.cloud if cloud is None else cloud
    dev = torch.device("cuda")
    c = torch.from_numpy(np.ascontiguousarray(cloud, np.float32)).to(dev)
    un = torch.from_numpy(np.ascontiguousarray(u0, np.float32)).to(dev)
    u_best, cand, best = aero.plan_step(planner, w.p0, w.q0, w.v0, c, w.goal, P, un)
    torch.cuda.synchronize()
    assert planner.sync_status() == 0
    out = dict(u_nom=un.cpu().numpy().astype(np.float64), u_best=u_best.cpu().numpy(),
               cand=cand.cpu().numpy(), best=int(best.cpu().numpy()[0]))
    if debug:
        E, K, T = P["E"], P["K"], P["T"]
        D = min(P.get("debug_samples", 0), K)
        out["keys"] = planner.debug("FINE_KEYS")
        out["point_counts"] = planner.debug("POINT_COUNTS")
        out["coarse"] = planner.debug("COARSE_WIN")
        out["goal_cell"] = int(planner.debug("GOAL_CELL")[0])
        out["anchor_cells"] = planner.debug("ANCHOR_CELLS")
        p0 = w.p0.astype(np.float64)
        out["anchors"] = planner.debug("ANCHORS").reshape(E, 3) + p0
        out["guides"] = planner.debug("GUIDES").reshape(E, T, 3) + p0
        out["S1"] = planner.debug("SAMPLE_COSTS").reshape(E, K).astype(np.float64)
        X2 = planner.debug("STAGE2_STATES").reshape(E, T + 1, 10).astype(np.float64)
        X2[..., :3] += p0
        out["X2"] = X2
        if D > 0:
            out["sU"] = planner.debug("SAMPLE_U").reshape(E, D, T, 4).astype(np.float64)
            sX = planner.debug("SAMPLE_X").reshape(E, D, T + 1, 10).astype(np.float64)
            sX[..., :3] += p0
            out["sX"] = sX
            out["sD"] = planner.debug("SAMPLE_DIST").reshape(E, D, T).astype(np.float64)
    return out


def x0_of(w) -> np.ndarray:
    return np.concatenate([w.p0, w.q0, w.v0]).astype(np.float64)
