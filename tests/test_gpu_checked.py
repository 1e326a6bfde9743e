"""The checked build (libaero_mppi_checked.so, AERO_CHECKED): every index the
kernels rely on is checked on the device and a failed check is reported by
aero_sync_status.  The edge cases of the parity suite, a batched call and the
accumulator run through it without a failed check, with the integer decisions
of the product library and its floating-point results to rounding.  Each
library runs in its own interpreter (the binding loads one of them)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import paper_2509_17340_gb300 as pkg
if sys.argv[2] == "checked":
    pkg.use_checked_build()
from paper_2509_17340_gb300 import aero, inputs as I
from gpu_util import make_planner, run_gpu
import test_gpu_parity as TP
out = {}
pl = make_planner(aero, T=128, cells=512 * 256)
for name in ["plain", "ensemble_small", "ensemble_small_l1", "ragged", "raw", "empty",
             "single_point", "k1_t1", "degenerate", "el_span"]:
    w = TP._case(name)
    g = run_gpu(aero, pl, w, w.params, w.hover_nominal())
    out[name] = dict(status=pl.sync_status(), keys=g["keys"].tolist(), coarse=g["coarse"].tolist(),
                     counts=g["point_counts"].tolist(), S1=g["S1"].ravel().tolist(),
                     u=g["u_nom"].ravel().tolist(), best=g["best"])
pl.close()
# a batched call over a few planners of both Stage I passes
ws = I.batch_workloads(6, seed=2)
for i, w in enumerate(ws):
    w.params["lanes_per_sample"] = 1 if i % 2 else 4
dev = torch.device("cuda")
lim = dict(E_max=16, K_max=4096, T_max=60, fine_cells_max=128 * 64,
           n_points_max=max(len(w.cloud) for w in ws))
b = aero.Batch(len(ws), **lim)
bufs = [(torch.from_numpy(w.cloud).to(dev), torch.from_numpy(w.hover_nominal()).to(dev),
         torch.empty((w.params["T"], 4), device=dev), torch.empty((w.params["E"],), device=dev),
         torch.empty((1,), dtype=torch.int32, device=dev)) for w in ws]
items = [aero.Batch.item(aero.state_struct(w.p0, w.q0, w.v0), c[0], w.goal, aero.params_struct(w.params),
                         c[1], c[2], c[3], c[4]) for w, c in zip(ws, bufs)]
b.plan(items)
torch.cuda.synchronize()
out["batch"] = dict(status=b.sync_status(), cand=[c[3].cpu().numpy().tolist() for c in bufs],
                    best=[int(c[4].cpu()[0]) for c in bufs])
b.close()
# accumulator: pushes with eviction and a gather
acc = aero.Accumulator(3, 500)
rng = np.random.default_rng(0)
for f in range(5):
    acc.push(torch.from_numpy(rng.normal(0, 5, (400 + 20 * f, 3)).astype(np.float32)).to(dev),
             [0.0, 0.0, float(f)], [1.0, 0.0, 0.0, 0.0])
dst = torch.empty((1500, 3), device=dev)
n = acc.gather(dst)
torch.cuda.synchronize()
out["accum"] = dict(n=int(n), sum=float(dst[:n].double().sum().cpu()))
acc.close()
pl2 = make_planner(aero, E=2, K=64, T=8, cells=64 * 32, n=16)
out["final_status"] = pl2.sync_status()
# the reporting path: a recorded check bit is reported once, then cleared
out["raise"] = aero.raise_check(1 << 8)
out["raised_status"] = pl2.sync_status()
out["after_raise"] = pl2.sync_status()
pl2.close()
print(json.dumps(out))
'''


def _run(which: str) -> dict:
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, which], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def runs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_17340_gb300 import build
    build.build()
    build.build(checked=True)
    return _run("product"), _run("checked")


def test_checked_build_reports_no_failed_check(runs):
    _, chk = runs
    for name, v in chk.items():
        if isinstance(v, dict) and "status" in v:
            assert v["status"] == 0, name
    assert chk["final_status"] == 0


def test_a_recorded_check_is_reported_once(runs):
    prod, chk = runs
    assert prod["raise"] == -1                       # no checks in the product build
    assert chk["raise"] == 0 and chk["raised_status"] == -5 and chk["after_raise"] == 0


def test_checked_build_matches_the_product_library(runs):
    prod, chk = runs
    for name, p in prod.items():
        c = chk[name]
        if name == "batch":
            assert c["best"] == p["best"]
            np.testing.assert_allclose(np.concatenate([np.asarray(x) for x in c["cand"]]),
                                       np.concatenate([np.asarray(x) for x in p["cand"]]), rtol=1e-5)
        elif name == "accum":
            assert c["n"] == p["n"] and c["sum"] == p["sum"]
        elif isinstance(p, dict):
            for k in ("keys", "coarse", "counts", "best"):
                assert c[k] == p[k], (name, k)
            np.testing.assert_allclose(c["S1"], p["S1"], rtol=1e-5, err_msg=name)
            np.testing.assert_allclose(c["u"], p["u"], rtol=1e-5, atol=1e-5, err_msg=name)
