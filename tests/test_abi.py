"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; host-only behaviour of the boundary (no GPU needed)."""
import ctypes as C
import glob
import json
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def so():
    from paper_2509_17340_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(aero_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["aero_create", "aero_destroy", "aero_plan_step", "aero_plan_step_host",
                 "aero_get_debug", "aero_debug_size", "aero_sync_status", "aero_status_str",
                 "aero_params_default", "aero_philox"]:
        assert must in names


def test_library_exports_every_declared_symbol(so):
    for name in declared_functions():
        assert hasattr(so, name), name


def test_status_strings(so):
    so.aero_status_str.restype = C.c_char_p
    assert so.aero_status_str(0) == b"ok"
    for code in range(-6, 0):
        assert so.aero_status_str(code) != b"unknown status"
    assert so.aero_status_str(-99) == b"unknown status"


def test_null_arguments_are_rejected_without_cuda(so):
    # argument checks come before any CUDA call
    assert so.aero_create(None, None) == -1
    assert so.aero_plan_step(None, None, None, C.c_int64(0), None, None, None, None, None, None, None) == -1
    assert so.aero_plan_step_host(None, None, None, C.c_int64(0), None, None, None, None, None, None, None) == -1
    assert so.aero_get_debug(None, 0, None, C.c_size_t(0), None) == -1
    assert so.aero_destroy(None) == 0


def test_params_default_is_table_I(so):
    import sys
    sys.path.insert(0, ROOT)
    # the binding's struct mirrors the header; it imports torch but needs no GPU
    from paper_2509_17340_gb300 import aero
    p = aero.default_params_struct()
    t = json.load(open(os.path.join(ROOT, "tests", "golden", "table1.json")))
    f32 = lambda v: C.c_float(v).value
    assert p.mass == f32(t["m_kg"]) and p.dt == f32(t["dt_s"]) and p.lam == f32(t["lambda"])
    assert p.K == t["K"] and p.T == t["N"] and p.E == t["M_h"] * t["M_v"]
    assert p.u_min[0] == f32(t["F_t_min_N"]) and p.u_max[0] == f32(t["F_t_max_N"])
    assert p.u_max[1] == f32(t["omega_xy_max"]) and p.u_max[3] == f32(t["omega_z_max"])
    assert abs(p.sigma[3] ** 2 - t["Sigma_omega_z"]) < 1e-6 and p.sigma[0] ** 2 == t["Sigma_Ft"]
    for a, b in [("Q_p", "Q_p"), ("Q_v", "Q_v"), ("Q_q", "Q_q"), ("Q_vnorm", "Q_vnorm"),
                 ("Q_track", "Q_track"), ("Q_c", "Q_c"), ("Q_cd", "Q_cdelta"), ("ell", "ell_m"),
                 ("C_col", "C"), ("a_col", "a"), ("d_min", "d_obs_min_m"), ("d_max", "d_obs_max_m"),
                 ("r_max", "r_max_m")]:
        assert getattr(p, a) == f32(t[b]), a
    assert [p.fine_az, p.fine_el] == t["fine_grid"] and [p.pool_az, p.pool_el] == t["pooling"]
    assert abs(p.el_hi - math.pi / 2) < 1e-6 and p.q_goal[0] == 1.0


def test_binding_struct_sizes_match_header(tmp_path):
    """The ctypes structures have the sizes the C compiler gives the header's."""
    import subprocess
    from paper_2509_17340_gb300 import aero
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "aero_mppi.h"\nint main(void) {\n'
                   '  printf("%zu %zu %zu %zu %zu\\n", sizeof(aero_state_t), sizeof(aero_limits_t),\n'
                   '         sizeof(aero_params_t), sizeof(aero_batch_item_t), sizeof(aero_batch_config_t));\n'
                   '  return 0;\n}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sizes = [int(x) for x in subprocess.check_output([str(exe)], text=True).split()]
    assert sizes == [C.sizeof(aero.State), C.sizeof(aero.Limits), C.sizeof(aero.Params),
                     C.sizeof(aero.BatchItem), C.sizeof(aero.BatchConfig)]


def test_allocation_test_hooks_without_cuda(so):
    # the counters and the injection countdown are host state: readable and
    # settable without a device
    so.aero_test_alloc_stats.restype = C.c_int64
    live = C.c_int64(-1)
    total = so.aero_test_alloc_stats(C.byref(live))
    assert total >= 0 and 0 <= live.value <= total
    assert so.aero_test_alloc_stats(None) == total
    assert so.aero_test_fail_alloc(C.c_int64(3)) == 0
    assert so.aero_test_fail_alloc(C.c_int64(-1)) == 0


def test_checked_build_exports_every_declared_symbol():
    # the checked build compiles the same sources with AERO_CHECKED
    from paper_2509_17340_gb300 import build
    lib = C.CDLL(build.build(checked=True))
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_non_finite_inputs_are_rejected_before_any_device_call():
    # the no-allocation entry point checks its arguments before any CUDA call:
    # a non-finite state, goal, sigma or scalar parameter is INVALID_ARG
    from paper_2509_17340_gb300 import aero
    lib = aero._lib
    bufs = [(C.c_float * 4096)() for _ in range(4)]
    ptrs = [C.cast(b, C.c_void_p) for b in bufs]
    cloud = (C.c_float * 3)(0.0, 0.0, 0.0)

    def call(state, goal, params):
        g = (C.c_float * 3)(*goal)
        return lib.aero_plan_step_noalloc(C.byref(state), C.cast(cloud, C.c_void_p), C.c_int64(1), g,
                                          C.byref(params), ptrs[0], ptrs[1], ptrs[2], ptrs[3], None)

    def state(p=(0.0, 0.0, 1.0), q=(1.0, 0.0, 0.0, 0.0), v=(0.0, 0.0, 0.0)):
        s = aero.State()
        s.p[:] = list(p)
        s.q[:] = list(q)
        s.v[:] = list(v)
        return s

    nan, inf = float("nan"), float("inf")
    P = aero.default_params_struct()
    assert call(state(p=(nan, 0.0, 1.0)), (5.0, 0.0, 1.0), P) == -1
    assert call(state(q=(1.0, 0.0, inf, 0.0)), (5.0, 0.0, 1.0), P) == -1
    assert call(state(v=(0.0, -inf, 0.0)), (5.0, 0.0, 1.0), P) == -1
    assert call(state(), (5.0, nan, 1.0), P) == -1
    for field, value in [("dt", inf), ("lam", inf), ("d_max", inf), ("mass", inf), ("r_max", inf)]:
        Q = aero.default_params_struct()
        assert field in [f for f, _ in aero.Params._fields_]
        setattr(Q, field, value)
        assert call(state(), (5.0, 0.0, 1.0), Q) == -1, field
    Q = aero.default_params_struct()
    Q.sigma[1] = inf
    assert call(state(), (5.0, 0.0, 1.0), Q) == -1


def test_missing_library_fails_loudly():
    """The binding has no CPU fallback: without the CUDA library the import
    raises (run in a child process so this one keeps its loaded library)."""
    import subprocess
    import sys
    code = ("import paper_2509_17340_gb300 as p\n"
            "p._library = 'libaero_mppi_absent.so'\n"
            "try:\n"
            "    import paper_2509_17340_gb300.aero\n"
            "except ImportError as e:\n"
            "    print('ImportError', e)\n"
            "else:\n"
            "    print('imported')\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("ImportError") and "no CPU fallback" in out.stdout
