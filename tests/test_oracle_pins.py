"""Pins of the CPU oracle against things other than itself.

Each test checks one oracle function against a closed form, an invariant, an
independent library routine (cuRAND's host Philox generator, scipy's rotations
and k-d tree), a value printed in the paper, or brute force on tiny inputs.
None of these tests touch the GPU or the CUDA library.
"""
import ctypes
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation
from scipy import stats

from paper_2509_17340_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Table I

def test_table1_values_match_paper():
    """Table I (Sec. V-A) values as printed, against the parameter defaults."""
    t = json.load(open(os.path.join(GOLD, "table1.json")))
    p = I.default_params()
    assert p["mass"] == t["m_kg"]
    assert p["u_min"][0] == t["F_t_min_N"] and p["u_max"][0] == t["F_t_max_N"]
    assert p["u_max"][1] == p["u_max"][2] == t["omega_xy_max"] and p["u_max"][3] == t["omega_z_max"]
    assert p["u_min"][1] == -t["omega_xy_max"] and p["u_min"][3] == -t["omega_z_max"]
    # Table I gives the covariance diagonal; the planner takes standard deviations.
    assert np.allclose(np.square(p["sigma"]), [t["Sigma_Ft"], t["Sigma_omega_xy"],
                                               t["Sigma_omega_xy"], t["Sigma_omega_z"]])
    assert p["dt"] == t["dt_s"] and p["K"] == t["K"] and p["T"] == t["N"] and p["lam"] == t["lambda"]
    for k, kk in [("Q_p", "Q_p"), ("Q_v", "Q_v"), ("Q_q", "Q_q"), ("Q_vnorm", "Q_vnorm"),
                  ("Q_track", "Q_track"), ("Q_c", "Q_c"), ("Q_cd", "Q_cdelta"), ("ell", "ell_m"),
                  ("C_col", "C"), ("a_col", "a"), ("d_min", "d_obs_min_m"), ("d_max", "d_obs_max_m"),
                  ("r_max", "r_max_m")]:
        assert p[k] == t[kk], k
    assert [p["fine_az"], p["fine_el"]] == t["fine_grid"]
    assert [p["pool_az"], p["pool_el"]] == t["pooling"]
    assert [p["fine_az"] // p["pool_az"], p["fine_el"] // p["pool_el"]] == t["coarse_grid"]
    assert p["M_h"] == t["M_h"] and p["M_v"] == t["M_v"] and p["E"] == t["M_h"] * t["M_v"]


# ----------------------------------------------------------------- Philox

def _curand_host_stream(seed: int, n_words: int, offset: int = 0):
    try:
        lib = ctypes.CDLL("libcurand.so")
    except OSError:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:   # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
    out = np.zeros(n_words, np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
    lib.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 0x123456789ABCDEF, 0xFEDCBA9876543210])
def test_philox_matches_curand_host_generator(orc, seed):
    """cuRAND's CPU Philox4x32-10 emits block b from counter
    (lo32(b >> 16), hi32(b >> 16), b & 0xffff, 0) under key (lo32(seed), hi32(seed))."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    blocks = _curand_host_stream(seed, 4 * 2048)
    for b in list(range(0, 2048, 7)) + [2047]:
        assert np.array_equal(orc.philox([0, 0, b, 0], key), blocks[b]), b
    # far into the stream: counter words 0 and 1 non-zero
    base = (1 << 32) * 65536 + 65536 * 3
    blocks = _curand_host_stream(seed, 4 * 64, offset=4 * base)
    for i in range(64):
        b = base + i
        c = b >> 16
        ctr = [c & 0xFFFFFFFF, c >> 32, b & 0xFFFF, 0]
        assert np.array_equal(orc.philox(ctr, key), blocks[i]), i


def test_noise_statistics(orc):
    """delta ~ N(0, diag(sigma^2)) (Sec. III-B): moments and Kolmogorov-Smirnov."""
    P = I.workload_params("plain")
    P["T"] = 50
    d = orc.noise_block(P, e=3, ks=range(400), it=0).reshape(-1, 4)
    sig = np.array(P["sigma"])
    z = d / sig
    n = len(z)
    assert np.all(np.abs(z.mean(0)) < 5 / math.sqrt(n))
    assert np.all(np.abs(z.var(0) - 1) < 6 * math.sqrt(2 / n))
    for c in range(4):
        assert stats.kstest(z[:, c], "norm").pvalue > 1e-4
    # the four components of one draw are uncorrelated
    cc = np.corrcoef(z.T)
    assert np.all(np.abs(cc - np.eye(4)) < 5 / math.sqrt(n))


def test_noise_counter_layout(orc):
    """Different (k, j, e, iter, step) give different draws; the same ones repeat."""
    P = I.workload_params("plain")
    a = orc.noise(P, 1, 2, 3, 0)
    assert np.array_equal(a, orc.noise(P, 1, 2, 3, 0))
    for args in [(0, 2, 3, 0), (1, 1, 3, 0), (1, 2, 4, 0), (1, 2, 3, 1)]:
        assert not np.allclose(a, orc.noise(P, *args))
    P2 = dict(P, step_id=5)
    assert not np.allclose(a, orc.noise(P2, 1, 2, 3, 0))


# ----------------------------------------------------------------- rotations and dynamics

def _rand_q(rng):
    q = I.random_unit_quaternion(rng).astype(np.float64)
    return q / np.linalg.norm(q)


def _scipy_R(q):
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def test_rotation_matches_scipy(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = _rand_q(rng)
        assert np.allclose(orc.rotation(q), _scipy_R(q), atol=1e-14)


def test_quaternion_product_composes_rotations(orc):
    rng = np.random.default_rng(2)
    for _ in range(50):
        a, b = _rand_q(rng), _rand_q(rng)
        assert np.allclose(_scipy_R(orc.quat_mul(a, b)), _scipy_R(a) @ _scipy_R(b), atol=1e-13)


def _skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def test_attitude_kinematics_body_rates(orc):
    """Eq. dynamics: q' = 1/2 q (x) [0, w] with w in the body frame, i.e.
    dR/dt = R [w]_x.  Checked by differencing scipy's R along q'."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = _rand_q(rng)
        w = rng.normal(size=3)
        x = np.concatenate([[0, 0, 0], q, [0, 0, 0]])
        qd = orc.dynamics(x, [0.0, *w])[3:7]
        h = 1e-6
        Rp, Rm = _scipy_R(q + h * qd), _scipy_R(q - h * qd)
        assert np.allclose((Rp - Rm) / (2 * h), _scipy_R(q) @ _skew(w), atol=1e-6)


def test_translational_dynamics(orc):
    """v' = (F/m) R(q) e3 - g e3, p' = v."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        q = _rand_q(rng)
        v = rng.normal(size=3)
        F, m = rng.uniform(0, 20), rng.uniform(0.5, 2)
        x = np.concatenate([rng.normal(size=3), q, v])
        xd = orc.dynamics(x, [F, 0.1, 0.2, 0.3], m=m, g=9.81)
        assert np.allclose(xd[:3], v, atol=0)
        assert np.allclose(xd[7:], F / m * _scipy_R(q)[:, 2] - [0, 0, 9.81], atol=1e-12)


def test_rk4_hover_is_fixed_point(orc):
    x = np.array([1.0, -2.0, 3.0, 1, 0, 0, 0, 0, 0, 0])
    X = orc.rollout(x, np.tile([9.81, 0, 0, 0], (40, 1)), 0.05)
    assert np.array_equal(X[-1], x)


def test_rk4_constant_thrust_closed_form(orc):
    """q = I, w = 0: p(t) = p0 + v0 t + 1/2 (F/m - g) t^2 e3; RK4 is exact here."""
    x = np.array([0.5, 0.25, 1.0, 1, 0, 0, 0, 1.0, -2.0, 0.5])
    F, T, dt = 12.0, 30, 0.05
    X = orc.rollout(x, np.tile([F, 0, 0, 0], (T, 1)), dt)
    t = T * dt
    a = F - 9.81
    assert np.allclose(X[-1, :3], x[:3] + x[7:] * t + 0.5 * np.array([0, 0, a]) * t * t, atol=1e-12)
    assert np.allclose(X[-1, 7:], x[7:] + np.array([0, 0, a]) * t, atol=1e-12)


def test_rk4_yaw_rate_closed_form(orc):
    """Constant yaw rate from q = I: with c = w + i z, c' = (i wz/2) c, so one RK4
    step multiplies c by P(i phi) = 1 + i phi - phi^2/2 - i phi^3/6 + phi^4/24,
    phi = wz dt / 2, and renormalising divides by |P|.  Thrust g keeps p fixed."""
    wz, dt, T = 1.7, 0.05, 40
    x = np.array([0, 0, 2.0, 1, 0, 0, 0, 0, 0, 0])
    X = orc.rollout(x, np.tile([9.81, 0, 0, wz], (T, 1)), dt)
    phi = wz * dt / 2
    Pz = 1 + 1j * phi - phi ** 2 / 2 - 1j * phi ** 3 / 6 + phi ** 4 / 24
    c = (Pz / abs(Pz)) ** T
    assert abs(X[-1, 3] - c.real) < 1e-13 and abs(X[-1, 6] - c.imag) < 1e-13
    assert np.allclose(X[-1, 4:6], 0) and np.allclose(X[-1, :3], x[:3], atol=1e-13)
    # and within RK4's O(dt^4) global error of the exact rotation
    ex = np.exp(1j * wz * T * dt / 2)
    assert abs(c - ex) < T * phi ** 5 / 120 * 1.01


def test_rk4_fourth_order_convergence(orc):
    """Global error of the RK4 rollout shrinks by ~16 when dt halves."""
    rng = np.random.default_rng(5)
    x0 = np.concatenate([[0, 0, 0], _rand_q(rng), rng.normal(size=3)])
    u = np.array([11.0, 0.7, -0.4, 0.9])
    Tend = 1.0

    def run(n):
        return orc.rollout(x0, np.tile(u, (n, 1)), Tend / n)[-1]

    ref = run(2048)
    e1 = np.abs(run(16) - ref).max()
    e2 = np.abs(run(32) - ref).max()
    assert 12 < e1 / e2 < 20


# ----------------------------------------------------------------- partition

def _exact_cell(b, P):
    """Cone of a body-frame direction from binary64 angles (independent of the
    oracle's binary32 edge predicates)."""
    A, El = P["fine_az"], P["fine_el"]
    al = math.atan2(b[1], b[0])
    if al >= math.pi:
        al -= 2 * math.pi
    be = math.atan2(b[2], math.hypot(b[0], b[1]))
    lo, hi = P["el_lo"], P["el_hi"]
    i = int(math.floor((al + math.pi) / (2 * math.pi / A)))
    j = int(math.floor((be - lo) / ((hi - lo) / El)))
    # angular distance to the nearest edge, to skip ambiguous points
    da = abs(((al + math.pi) / (2 * math.pi / A)) - round((al + math.pi) / (2 * math.pi / A)))
    de = abs(((be - lo) / ((hi - lo) / El)) - round((be - lo) / ((hi - lo) / El)))
    return min(i, A - 1), min(j, El - 1), min(da, de)


@pytest.mark.parametrize("A,El", [(120, 60), (16, 8), (128, 64)])
def test_partition_brute_force(orc, A, El):
    """Sec. IV-A.1 on a tiny cloud: per-cone nearest point by enumeration."""
    P = I.default_params()
    P.update(fine_az=A, fine_el=El, r_max=6.0)
    rng = np.random.default_rng(A)
    q0 = I.random_unit_quaternion(rng)
    p0 = np.array([0.5, -1.0, 1.5], np.float32)
    cloud = (p0 + rng.uniform(-7, 7, size=(300, 3))).astype(np.float32)
    keys, kept = orc.partition(cloud, p0, q0, P)
    R = _scipy_R(q0.astype(np.float64))
    best = {}
    n_in = 0
    for idx, p in enumerate(cloud.astype(np.float64)):
        b = R.T @ (p - p0)
        r = np.linalg.norm(b)
        if r > 6.0:
            continue
        n_in += 1
        i, j, dedge = _exact_cell(b, P)
        c = j * A + i
        if dedge < 1e-4:
            continue
        if c not in best or r < best[c][0]:
            best[c] = (r, idx)
    assert abs(kept - n_in) <= 2   # points within rounding of r_max may differ
    for c, (r, idx) in best.items():
        k = keys[c]
        assert k != orc.EMPTY
        # the winning point may only differ if ranges tie within binary32 rounding
        widx = int(k & np.uint64(0xFFFFFFFF))
        if widx != idx:
            rw = np.linalg.norm(R.T @ (cloud[widx].astype(np.float64) - p0))
            assert abs(rw - r) < 1e-5
        r2 = np.array([int(k >> np.uint64(32))], np.uint32).view(np.float32)[0]
        assert abs(math.sqrt(r2) - r) < 1e-5
    # cones with no point stay empty
    occupied = set(best)
    for c in range(A * El):
        if keys[c] != orc.EMPTY and c not in occupied:
            # only allowed for points we skipped as ambiguous near an edge
            widx = int(keys[c] & np.uint64(0xFFFFFFFF))
            _, _, dedge = _exact_cell(R.T @ (cloud[widx].astype(np.float64) - p0), P)
            assert dedge < 1e-4


def test_partition_hand_cases(orc):
    P = I.default_params()   # 120 x 60 over the full sphere
    p0 = np.array([1.0, 2.0, 3.0], np.float32)
    q_id = np.array([1, 0, 0, 0], np.float32)
    keys, kept = orc.partition(np.zeros((0, 3), np.float32), p0, q_id, P)
    assert kept == 0 and np.all(keys == orc.EMPTY)
    # a point straight ahead (+x body): azimuth 0 -> column 60, elevation 0 -> row 30
    keys, kept = orc.partition(p0[None] + np.array([[2.0, 0, 0]], np.float32), p0, q_id, P)
    assert kept == 1 and keys[30 * 120 + 60] == (np.uint64(np.float32(4.0).view(np.uint32)) << np.uint64(32))
    # yawed by +90 deg: a world point on +y is straight ahead in the body frame
    qy = np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)], np.float32)
    keys, _ = orc.partition(p0[None] + np.array([[0, 3.0, 0]], np.float32), p0, qy, P)
    assert keys[30 * 120 + 60] != orc.EMPTY
    # behind (-x): azimuth -pi -> column 0; straight up -> top row
    keys, _ = orc.partition(p0[None] + np.array([[-2.0, 0, 0], [0, 0, 4.0]], np.float32), p0, q_id, P)
    assert keys[30 * 120 + 0] != orc.EMPTY
    assert np.any(keys[59 * 120:60 * 120] != orc.EMPTY)
    # beyond r_max, at the origin, and non-finite points are not in P_t
    bad = np.array([[11.0, 0, 0], [0, 0, 0], [np.nan, 0, 0], [np.inf, 1, 1]], np.float32) + p0
    keys, kept = orc.partition(bad, p0, q_id, P)
    assert kept == 0
    # two points in one cone: the nearer wins, equal ranges -> lower index
    two = p0 + np.array([[3.0, 0.01, 0], [2.0, 0.01, 0], [2.0, 0.01, 0]], np.float32)
    keys, _ = orc.partition(two, p0, q_id, P)
    assert int(keys[30 * 120 + 60] & np.uint64(0xFFFFFFFF)) == 1


def test_coarse_argmax_invariants(orc):
    """Eq. safe-vector: the winner is in Omega_IJ and has the largest r there."""
    P = I.default_params()
    P.update(r_max=6.0)
    rng = np.random.default_rng(7)
    cloud = rng.uniform(-6, 6, size=(3000, 3)).astype(np.float32)
    p0 = np.zeros(3, np.float32)
    q0 = np.array([1, 0, 0, 0], np.float32)
    keys, _ = orc.partition(cloud, p0, q0, P)
    win, rwin = orc.coarse(keys, P)
    A, Pa, Pe = P["fine_az"], P["pool_az"], P["pool_el"]
    Ac = A // Pa
    rmax2 = np.float32(6.0) * np.float32(6.0)
    r = np.where(keys == orc.EMPTY, math.sqrt(rmax2),
                 np.sqrt((keys >> np.uint64(32)).astype(np.uint32).view(np.float32).astype(np.float64)))
    for cc, w in enumerate(win):
        I_, J_ = cc % Ac, cc // Ac
        i, j = w % A, w // A
        assert I_ * Pa <= i < (I_ + 1) * Pa and J_ * Pe <= j < (J_ + 1) * Pe
        members = [(jj * A + ii) for jj in range(J_ * Pe, (J_ + 1) * Pe) for ii in range(I_ * Pa, (I_ + 1) * Pa)]
        assert r[w] == max(r[m] for m in members)
        assert abs(rwin[cc] - r[w]) < 1e-12


def test_coarse_empty_cloud_picks_centre_cone(orc):
    """Empty cloud: every cone is at r_max, so the winner is the centre-most cone
    (for even pooling the four central cones tie; the lowest index wins)."""
    P = I.default_params()
    keys = np.full(P["fine_az"] * P["fine_el"], orc.EMPTY, np.uint64)
    win, rwin = orc.coarse(keys, P)
    A, Pa, Pe = P["fine_az"], P["pool_az"], P["pool_el"]
    Ac = A // Pa
    for cc, w in enumerate(win):
        I_, J_ = cc % Ac, cc // Ac
        assert w == (J_ * Pe + Pe // 2 - 1) * A + I_ * Pa + Pa // 2 - 1
        assert abs(rwin[cc] - 10.0) < 1e-6


def test_goal_cell_and_anchor_cells(orc):
    """Goal straight ahead: fine cell (60, 30) of 120x60, coarse (10, 5) of 20x10.
    5x3 anchors: azimuth offsets -2..2 (wrapping), elevation -1..1 (clamped)."""
    P = I.default_params()
    p0 = np.array([0, 0, 2], np.float32)
    q0 = np.array([1, 0, 0, 0], np.float32)
    g = orc.goal_fine_cell(np.array([45, 0, 2], np.float32), p0, q0, P)
    assert g == 30 * 120 + 60
    cells = orc.anchor_cells(g, P)
    exp = [J * 20 + I_ for J in (4, 5, 6) for I_ in (8, 9, 10, 11, 12)]
    assert list(cells) == exp
    # goal behind the drone: coarse column 0 -> azimuth wraps to 18, 19, 0, 1, 2
    g = orc.goal_fine_cell(np.array([-45, 0.0, 2], np.float32), p0, q0, P)
    cells = orc.anchor_cells(g, P)
    assert [c % 20 for c in cells[:5]] == [18, 19, 0, 1, 2]
    # goal straight up: elevation clamps to the top row
    g = orc.goal_fine_cell(np.array([0, 0, 50], np.float32), p0, q0, P)
    cells = orc.anchor_cells(g, P)
    assert [c // 20 for c in cells] == [8] * 5 + [9] * 5 + [9] * 5


def test_cell_direction_and_anchor(orc):
    """Eq. unit direction and Eq. anchor-point on hand-computable cases."""
    P = I.default_params()
    # cell (60, 30): alpha = 1.5 deg, beta = 1.5 deg
    d = orc.cell_direction(P, 30 * 120 + 60)
    a = b = math.radians(1.5)
    assert np.allclose(d, [math.cos(b) * math.cos(a), math.cos(b) * math.sin(a), math.sin(b)], atol=1e-7)
    assert abs(np.linalg.norm(d) - 1) < 1e-15
    # anchor for a yawed drone: body +x becomes world +y
    qy = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]
    pr = orc.anchor([1, 2, 3], qy, [1, 0, 0], 5.0)
    assert np.allclose(pr, [1, 7, 3], atol=1e-12)


# ----------------------------------------------------------------- quintic guides

def test_quintic_boundary_conditions_and_closed_form(orc):
    rng = np.random.default_rng(8)
    for _ in range(10):
        ps, vs, pe, ve = (rng.normal(size=3) * 3 for _ in range(4))
        As, Ae = rng.normal(size=3), rng.normal(size=3)
        Tg = rng.uniform(0.5, 3)
        coef = orc.quintic(ps, vs, As, pe, ve, Ae, Tg)
        for mu in range(3):
            c = coef[mu]
            f = np.polynomial.Polynomial(c)
            df, ddf = f.deriv(), f.deriv(2)
            assert abs(f(0) - ps[mu]) < 1e-12 and abs(df(0) - vs[mu]) < 1e-12 and abs(ddf(0) - As[mu]) < 1e-12
            assert abs(f(Tg) - pe[mu]) < 1e-9 and abs(df(Tg) - ve[mu]) < 1e-9 and abs(ddf(Tg) - Ae[mu]) < 1e-9
            # textbook closed form of the minimum-jerk quintic
            h = pe[mu] - ps[mu]
            a3 = (20 * h - (8 * ve[mu] + 12 * vs[mu]) * Tg - (3 * As[mu] - Ae[mu]) * Tg ** 2) / (2 * Tg ** 3)
            a4 = (-30 * h + (14 * ve[mu] + 16 * vs[mu]) * Tg + (3 * As[mu] - 2 * Ae[mu]) * Tg ** 2) / (2 * Tg ** 4)
            a5 = (12 * h - 6 * (ve[mu] + vs[mu]) * Tg - (As[mu] - Ae[mu]) * Tg ** 2) / (2 * Tg ** 5)
            assert np.allclose(c, [ps[mu], vs[mu], As[mu] / 2, a3, a4, a5], rtol=1e-9, atol=1e-9)


def test_guide_endpoints(orc):
    P = I.workload_params("ensemble")
    p0, v0, pref = np.array([0, 0, 1.5]), np.array([1.0, 0.5, 0]), np.array([4.0, 3.0, 1.5])
    coef, g = orc.guide(p0, v0, pref, P)
    assert np.allclose(g[-1], pref, atol=1e-9)
    Tg = P["T"] * P["dt"]
    vT = np.array([np.polynomial.Polynomial(coef[m]).deriv()(Tg) for m in range(3)])
    assert np.allclose(vT, (P["ell"] / Tg) * (pref - p0) / np.linalg.norm(pref - p0), atol=1e-9)


# ----------------------------------------------------------------- costs

def test_nn_distance_matches_kdtree(orc):
    rng = np.random.default_rng(9)
    pts = rng.uniform(-5, 5, size=(500, 3))
    tree = cKDTree(pts)
    for _ in range(50):
        q = rng.uniform(-6, 6, size=3)
        assert abs(orc.nn_dist(q, pts) - tree.query(q)[0]) < 1e-12
    assert orc.nn_dist(np.zeros(3), np.zeros((0, 3))) == math.inf


def test_collision_penalty_pieces(orc):
    P = I.default_params()
    C, a, dmin, dmax = P["C_col"], P["a_col"], P["d_min"], P["d_max"]
    assert orc.jcol(0.0, P) == C and orc.jcol(dmin - 1e-9, P) == C
    assert orc.jcol(dmin, P) == C
    assert abs(orc.jcol(dmax - 1e-12, P) - C * math.exp(-a * (dmax - dmin))) < 1e-3
    assert orc.jcol(dmax, P) == 0.0 and orc.jcol(math.inf, P) == 0.0
    assert abs(orc.jcol(0.7, P) - C * math.exp(-a * 0.3)) < 1e-6


def test_attitude_error_frobenius(orc):
    """||R(q) R(q_g)^T - I||_F = sqrt(8 (1 - w^2)) = 2 sqrt(2) |sin(theta/2)|,
    theta the angle of the relative rotation (scipy)."""
    rng = np.random.default_rng(10)
    for _ in range(30):
        q, qg = _rand_q(rng), _rand_q(rng)
        th = (Rotation.from_quat([q[1], q[2], q[3], q[0]]) *
              Rotation.from_quat([qg[1], qg[2], qg[3], qg[0]]).inv()).magnitude()
        assert abs(orc.attitude_err(q, qg) - 2 * math.sqrt(2) * abs(math.sin(th / 2))) < 1e-12
        assert abs(orc.attitude_err(q, [1, 0, 0, 0]) - math.sqrt(max(0, 8 * (1 - q[0] ** 2)))) < 1e-7


def test_cost_terms_hand_built(orc):
    """Each cost term of Sec. IV-C on a hovering trajectory with known values."""
    P = I.default_params()
    T = P["T"]
    p = np.array([1.0, 2.0, 3.0])
    X = np.tile(np.concatenate([p, [1, 0, 0, 0], [0, 0, 0]]), (T + 1, 1))
    X[:, 9] = 0.0
    U = np.zeros((T, 4))
    U[:, 0] = np.arange(T)          # u_t = (t, 0, 0, 0): |u_t|^2 = t^2, |du_t|^2 = 1
    guide = np.tile(p + [0, 0, 2.0], (T, 1))
    goal = p + [3.0, 4.0, 0]
    pts = np.array([p + [0.7, 0, 0]])
    out = orc.cost_terms(X, U, guide, goal, pts, P, stage=1, want_dist=True)
    assert abs(out["J_track"] - T * P["Q_track"] * 2.0) < 1e-9
    assert out["J_vnorm"] == 0.0
    ctrl = P["Q_c"] * sum(t * t for t in range(0, T - 1)) + P["Q_cd"] * (T - 2)
    assert abs(out["J_ctrl"] - ctrl) < 1e-9
    assert abs(out["J_goal"] - T * P["Q_p"] * 5.0) < 1e-9
    assert np.allclose(out["dist"], 0.7)
    assert abs(out["J_col"] - T * P["C_col"] * math.exp(-P["a_col"] * 0.3)) < 1e-3
    assert abs(out["S"] - (out["J_track"] + out["J_vnorm"] + out["J_ctrl"] + out["J_goal"] + out["J_col"])) < 1e-6
    o2 = orc.cost_terms(X, U, guide, goal, pts, P, stage=2)
    assert abs(o2["S"] - (out["J_goal"] + out["J_col"])) < 1e-6
    # velocity terms: |v|^2 and |v - v_goal|
    X[1:, 7:10] = [0.0, 3.0, 4.0]
    out = orc.cost_terms(X, U, None, goal, np.zeros((0, 3)), P, stage=1)
    assert abs(out["J_vnorm"] - T * P["Q_vnorm"] * 25.0) < 1e-9
    assert abs(out["J_goal"] - T * (P["Q_p"] * 5.0 + P["Q_v"] * 5.0)) < 1e-9
    assert out["J_col"] == 0.0 and out["J_track"] == 0.0


def test_ctrl_cost_short_horizons(orc):
    """Sum limits t = 0..N-2 and t = 1..N-2: empty for N = 1, one term for N = 2."""
    for T, expect in [(1, 0.0), (2, 0.5 * 4.0), (3, 0.5 * (4.0 + 9.0) + 0.5 * 1.0)]:
        P = I.default_params()
        P["T"] = T
        X = np.tile(np.array([0, 0, 0, 1, 0, 0, 0, 0, 0, 0.0]), (T + 1, 1))
        U = np.array([[2.0, 0, 0, 0], [3.0, 0, 0, 0], [5.0, 0, 0, 0]])[:T]
        out = orc.cost_terms(X, U, None, [0, 0, 0], np.zeros((0, 3)), P)
        assert abs(out["J_ctrl"] - expect) < 1e-12


# ----------------------------------------------------------------- MPPI weights and update

def test_mppi_weights_invariants(orc):
    rng = np.random.default_rng(11)
    K, T = 64, 5
    S = rng.uniform(10, 20, K)
    dU = rng.normal(size=(K, T * 4))
    u0 = rng.normal(size=(T, 4))
    u, eps = orc.mppi_update(S, dU, 1.0, u0)
    assert abs(eps.sum() - 1) < 1e-14 and np.all(eps > 0)
    assert np.argmax(eps) == np.argmin(S)
    # zero noise returns the nominal
    u, _ = orc.mppi_update(S, np.zeros_like(dU), 1.0, u0)
    assert np.array_equal(u, u0)
    # lambda -> infinity: the sample mean; equal costs: the mean as well
    u, _ = orc.mppi_update(S, dU, 1e12, u0)
    assert np.allclose(u, u0 + dU.mean(0).reshape(T, 4), atol=1e-9)
    u, _ = orc.mppi_update(np.full(K, 3.0), dU, 0.1, u0)
    assert np.allclose(u, u0 + dU.mean(0).reshape(T, 4), atol=1e-12)
    # lambda -> 0: the argmin sample (Sec. III-B)
    u, _ = orc.mppi_update(S, dU, 1e-9, u0)
    assert np.allclose(u, u0 + dU[np.argmin(S)].reshape(T, 4), atol=1e-12)
    # shift invariance of the weights
    _, e1 = orc.mppi_update(S, dU, 0.7, u0)
    _, e2 = orc.mppi_update(S + 1234.5, dU, 0.7, u0)
    assert np.allclose(e1, e2, rtol=1e-9)


# ----------------------------------------------------------------- whole step

def _small_step_inputs(seed=0, E=4, K=32, T=8):
    P = I.workload_params("ensemble")
    P.update(E=E, K=K, T=T, M_h=E // 2 if E > 1 else 1, M_v=2 if E > 1 else 1, seed=seed)
    w = I.make_workload("plain", seed)
    return P, w


def test_plan_step_invariants(orc):
    P, w = _small_step_inputs()
    E, T = P["E"], P["T"]
    u0 = np.zeros((E, T, 4), np.float32)
    u0[..., 0] = 9.81
    out = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, u0)
    lo, hi = np.array(P["u_min"]), np.array(P["u_max"])
    assert np.all(out["u_nom"] >= lo - 1e-12) and np.all(out["u_nom"] <= hi + 1e-12)
    assert out["best"] == int(np.argmin(out["cand"]))
    assert np.array_equal(out["u_best"], out["u_nom"][out["best"]])
    assert np.all(np.isfinite(out["S1"]))
    # Stage II costs are recomputed from the Stage II states
    assert np.allclose(out["X2"][:, 0, :3], w.p0)


def test_plan_step_zero_noise_keeps_nominal(orc):
    P, w = _small_step_inputs()
    P["sigma"] = [0.0, 0.0, 0.0, 0.0]
    u0 = np.zeros((P["E"], P["T"], 4), np.float32)
    u0[..., 0] = 9.0
    out = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, u0)
    assert np.array_equal(out["u_nom"], u0.astype(np.float64))


def test_plan_step_large_lambda_is_sample_mean(orc):
    """lambda -> infinity: u_nom + mean_k (clamp(u_nom + delta) - u_nom)."""
    P, w = _small_step_inputs(E=2, K=16, T=4)
    P["lam"] = 1e15
    u0 = np.zeros((P["E"], P["T"], 4), np.float32)
    u0[..., 0] = 19.0      # near the thrust bound 2g and the rate bounds: clamping is active
    u0[..., 1:] = 5.5
    out = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, u0)
    lo, hi = np.array(P["u_min"]), np.array(P["u_max"])
    for e in range(P["E"]):
        d = orc.noise_block(P, e, range(P["K"]))
        u = np.clip(u0[e].astype(np.float64) + d, lo, hi)
        assert np.any(u != u0[e].astype(np.float64) + d)
        assert np.allclose(out["u_nom"][e], u.mean(0), atol=1e-9)
        assert np.all(out["u_nom"][e] <= hi + 1e-12)


def test_plan_step_empty_cloud(orc):
    P, w = _small_step_inputs()
    u0 = np.zeros((P["E"], P["T"], 4), np.float32)
    u0[..., 0] = 9.81
    out = orc.plan_step(np.zeros((0, 3), np.float32), w.p0, w.q0, w.v0, w.goal, P, u0)
    assert np.all(out["keys"] == orc.EMPTY)
    assert np.all(np.isfinite(out["cand"]))


@pytest.mark.parametrize("iters", [1, 2])
def test_plan_step_is_the_stated_composition(orc, iters):
    """The whole step (Sec. IV) equals its stages composed by hand from the
    separately pinned functions: partition, coarse argmax, goal and anchor
    cells, anchors and quintic guides, then per iteration the clamped
    perturbations of that iteration's counter, the rollouts, S(1) with the
    instance's guide and the update of the iteration's nominal; then Stage II
    (S(2) of the updated nominals) and the argmin.  A step that wired a stage
    to the wrong instance, iteration, guide or cost stage fails here."""
    w = I.make_workload("plain", seed=4)
    P = I.workload_params("ensemble")
    P.update(E=4, M_h=2, M_v=2, K=24, T=6, iters=iters, Q_track=15.0, step_id=9, seed=77)
    rng = np.random.default_rng(4)
    q0 = I.random_unit_quaternion(rng)
    v0 = np.array([1.0, -0.4, 0.2], np.float32)
    u0 = np.zeros((P["E"], P["T"], 4), np.float32)
    u0[..., 0] = 9.81
    u0[..., 1:] = rng.uniform(-0.5, 0.5, (P["E"], P["T"], 3))
    out = orc.plan_step(w.cloud, w.p0, q0, v0, w.goal, P, u0)
    x0 = np.concatenate([w.p0, q0, v0]).astype(np.float64)
    goal = w.goal.astype(np.float64)
    keys, _ = orc.partition(w.cloud, w.p0, q0, P)
    assert np.array_equal(out["keys"], keys)
    win, _ = orc.coarse(keys, P)
    cells = orc.anchor_cells(orc.goal_fine_cell(w.goal, w.p0, q0, P), P)
    pts = orc.collision_set(w.cloud, w.p0, q0, keys, P)
    assert len(pts) > 0
    lo, hi = np.array(P["u_min"]), np.array(P["u_max"])
    K, T = P["K"], P["T"]
    cand = np.zeros(P["E"])
    for e in range(P["E"]):
        pref = orc.anchor(x0[:3], x0[3:7], orc.cell_direction(P, int(win[cells[e]])), P["ell"])
        assert np.abs(out["anchors"][e] - pref).max() < 1e-12
        _, guide = orc.guide(x0[:3], x0[7:], pref, P)
        assert np.abs(out["guides"][e] - guide).max() < 1e-12
        un = u0[e].astype(np.float64)
        for it in range(iters):
            d = orc.noise_range(P, e, 0, K, it=it)
            U = np.clip(un + d, lo, hi)
            S = np.array([orc.cost_terms(orc.rollout(x0, U[k], P["dt"], P["mass"], P["g"]), U[k],
                                         guide, goal, pts, P, stage=1)["S"] for k in range(K)])
            un, _ = orc.mppi_update(S, (U - un).reshape(K, -1), P["lam"], un)
        assert np.allclose(out["S1"][e], S, rtol=1e-12, atol=0)
        assert np.abs(out["u_nom"][e] - un).max() < 1e-12
        X2 = orc.rollout(x0, un, P["dt"], P["mass"], P["g"])
        assert np.abs(out["X2"][e] - X2).max() < 1e-12
        cand[e] = orc.cost_terms(X2, un, None, goal, pts, P, stage=2)["S"]
    assert np.allclose(out["cand"], cand, rtol=1e-12, atol=0)
    assert out["best"] == int(np.argmin(cand))
    assert np.array_equal(out["u_best"], out["u_nom"][out["best"]])


# ----------------------------------------------------------------- collision sets

def _clean_cloud(rng, p0, R, P, n):
    """n points around p0 none of which is within 1e-3 rad of a cone edge or of
    the elevation span's ends, nor within 1e-3 m of r_max (so that binary32
    and binary64 decisions agree), plus the degenerate points the partition
    drops: p0 itself, non-finite coordinates, a point beyond r_max."""
    out = []
    while len(out) < n:
        p = p0 + rng.uniform(-1.3, 1.3, 3) * P["r_max"]
        b = R.T @ (p.astype(np.float32).astype(np.float64) - p0)
        r = np.linalg.norm(b)
        _, _, dedge = _exact_cell(b, P)
        be = math.atan2(b[2], math.hypot(b[0], b[1]))
        if dedge < 1e-3 or abs(r - P["r_max"]) < 1e-3:
            continue
        if min(abs(be - P["el_lo"]), abs(be - P["el_hi"])) < 1e-3:
            continue
        out.append(p)
    out += [p0, [np.nan, 1, 1], [1, np.inf, 1], p0 + [0, 0, 3 * P["r_max"]]]
    return np.array(out, np.float32)


@pytest.mark.parametrize("span", [(-math.pi / 2, math.pi / 2), (-0.4, 0.9)])
def test_collision_sets_by_enumeration(orc, span):
    """Sec. IV-C's filtered cloud P_f: the nearest point of every non-empty
    cone, in world coordinates, in cone order; and the every-point set: the
    points the partition keeps (finite, 0 < r <= r_max, inside the elevation
    span), in point order.  Both by enumeration with binary64 angles on a
    rotated start, so a wrong frame, a wrong half of the packed key or a
    filter that keeps points outside the span or range fails."""
    P = I.default_params()
    P.update(fine_az=24, fine_el=12, r_max=5.0, el_lo=span[0], el_hi=span[1])
    rng = np.random.default_rng(17)
    q0 = I.random_unit_quaternion(rng)
    p0 = np.array([1.5, -2.0, 0.7], np.float32)
    R = _scipy_R(q0.astype(np.float64))
    p0d = p0.astype(np.float64)
    cloud = _clean_cloud(rng, p0d, R, P, 400)
    best, kept = {}, []
    for idx, p in enumerate(cloud.astype(np.float64)):
        if not np.all(np.isfinite(p)):
            continue
        b = R.T @ (p - p0d)
        r = np.linalg.norm(b)
        if r == 0.0 or r > P["r_max"]:
            continue
        be = math.atan2(b[2], math.hypot(b[0], b[1]))
        if not (P["el_lo"] <= be <= P["el_hi"]):
            continue
        kept.append(idx)
        i, j, _ = _exact_cell(b, P)
        c = j * P["fine_az"] + i
        if c not in best or r < best[c][0]:
            best[c] = (r, idx)
    keys, n_kept = orc.partition(cloud, p0, q0, P)
    assert n_kept == len(kept)
    pf = orc.collision_set(cloud, p0, q0, keys, dict(P, collision_set=0))
    want = np.array([cloud[best[c][1]] for c in sorted(best)], np.float64).reshape(-1, 3)
    assert pf.shape == want.shape and np.array_equal(pf, want)
    raw = orc.collision_set(cloud, p0, q0, keys, dict(P, collision_set=1))
    assert np.array_equal(raw, cloud[kept].astype(np.float64))
    if span[1] - span[0] < math.pi:
        # the narrow span drops points that the full sphere keeps
        full = orc.collision_set(cloud, p0, q0, keys, dict(P, collision_set=1, el_lo=-math.pi / 2,
                                                           el_hi=math.pi / 2))
        assert len(full) > len(raw)


def test_collision_set_of_empty_and_single_point_clouds(orc):
    P = I.default_params()
    p0 = np.array([0.0, 0.0, 1.0], np.float32)
    q0 = np.array([1, 0, 0, 0], np.float32)
    empty = np.zeros((0, 3), np.float32)
    keys, _ = orc.partition(empty, p0, q0, P)
    assert len(orc.collision_set(empty, p0, q0, keys, dict(P, collision_set=0))) == 0
    one = np.array([[3.0, 0.5, 1.25]], np.float32)
    keys, _ = orc.partition(one, p0, q0, P)
    for mode in (0, 1):
        s = orc.collision_set(one, p0, q0, keys, dict(P, collision_set=mode))
        assert np.array_equal(s, one.astype(np.float64))
