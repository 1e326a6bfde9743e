"""The GPU's Gaussian draws against the oracle's: Box-Muller on the same
Philox words, the GPU with CUDA's hardware logarithm, sine and cosine (and the
series of ln(1 - v) near u = 1), the oracle in binary64.  With sigma = 1 and
bounds too wide to clamp, every recorded perturbation is a normal; the stated
bound is 5e-6 (absolute)."""
import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I
from gpu_util import make_planner, run_gpu

pytestmark = pytest.mark.gpu

BOUND = 5e-6


@pytest.fixture(scope="module")
def aero():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero as A
    return A


@pytest.mark.parametrize("lanes", [1, 4])
def test_normals_within_stated_bound(aero, orc, lanes):
    w = I.make_workload("plain")
    P = dict(w.params, K=1024, T=48, sigma=[1.0, 1.0, 1.0, 1.0], u_min=[-1e6] * 4, u_max=[1e6] * 4,
             debug_samples=1024, lanes_per_sample=lanes, seed=12345, step_id=7)
    pl = make_planner(aero, E=1, K=1024, T=48, cells=P["fine_az"] * P["fine_el"], n=len(w.cloud), D=1024)
    u0 = np.zeros((1, 48, 4), np.float32)
    g = run_gpu(aero, pl, w, P, u0)
    n_gpu = g["sU"][0].reshape(-1, 4)          # u = 0 + delta, delta = normal
    n_orc = orc.noise_range(P, 0, 0, 1024).reshape(-1, 4)
    err = np.abs(n_gpu - n_orc)
    assert err.max() <= BOUND, err.max()
    assert len(err) * 4 >= 196608
    pl.close()
