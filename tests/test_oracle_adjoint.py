"""Pins of the oracle's gradient of S^(1) with respect to the controls
(orc_cost_grad) and of the gradient refinement (orc_refine), against things
the adjoint code does not share: central finite differences (h = 1e-6) of the
oracle's forward cost (orc_rollout + orc_cost_terms), closed forms, exact zeros
and descent.  The finite-difference scenes exercise every term of S^(1): guide
tracking, velocity norm, both control terms, goal position, goal velocity,
attitude against a non-identity goal attitude from a tilted start, and the
collision term inside (d_min, d_max); trajectories stay clear of the
non-differentiable points (d_min, d_max, zero norms, nearest-point ties)."""
import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I


def _unit(q):
    q = np.asarray(q, np.float64)
    return q / np.linalg.norm(q)


def _scene(seed=0, T=12):
    rng = np.random.default_rng(seed)
    P = dict(I.default_params(), T=T, E=1, K=1, M_h=1, M_v=1)
    P["q_goal"] = list(_unit([0.97, 0.05, -0.1, 0.2]))
    P["v_goal"] = [1.0, 0.2, 0.0]
    q0 = _unit([0.99, 0.03, 0.08, -0.05])
    x0 = np.array([0.0, 0.0, 1.5, *q0, 2.0, 0.1, 0.0])
    U = np.tile([P["g"], 0.0, 0.0, 0.0], (T, 1)) + rng.normal(0, [0.8, 0.6, 0.6, 0.6], (T, 4))
    guide = np.stack([np.linspace(0.1, 1.2, T), 0.05 * np.ones(T), 1.5 + 0.02 * np.arange(T)], 1)
    goal = np.array([6.0, 0.5, 1.8])
    return P, x0, U, guide, goal


def _forward(orc, P, x0, U, guide, goal, pts):
    X = orc.rollout(x0, U, P["dt"], P["mass"], P["g"])
    return orc.cost_terms(X, U, guide, goal, pts, P, stage=1, want_dist=True)


def _clear_of_kinks(orc, P, x0, U, guide, goal, pts, margin=2e-3):
    t = _forward(orc, P, x0, U, guide, goal, pts)
    d = t["dist"]
    X = orc.rollout(x0, U, P["dt"], P["mass"], P["g"])
    p = X[1:, :3]
    ok = np.all(np.abs(d - P["d_min"]) > margin) and np.all(np.abs(d - P["d_max"]) > margin)
    ok &= np.all(np.linalg.norm(p - guide, axis=1) > margin)
    ok &= np.all(np.linalg.norm(p - goal, axis=1) > margin)
    if len(pts) > 1:
        dd = np.sort(np.linalg.norm(p[:, None, :] - pts[None], axis=2), axis=1)
        ok &= np.all(dd[:, 1] - dd[:, 0] > margin)
    return bool(ok), t


def _fd(orc, P, x0, U, guide, goal, pts, h=1e-6):
    G = np.zeros_like(U)
    for j in range(U.shape[0]):
        for c in range(4):
            Up, Um = U.copy(), U.copy()
            Up[j, c] += h
            Um[j, c] -= h
            G[j, c] = (_forward(orc, P, x0, Up, guide, goal, pts)["S"] -
                       _forward(orc, P, x0, Um, guide, goal, pts)["S"]) / (2 * h)
    return G


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(orc, seed):
    P, x0, U, guide, goal = _scene(seed)
    # obstacle points beside the path: some steps fall inside (d_min, d_max)
    X = orc.rollout(x0, U, P["dt"], P["mass"], P["g"])
    mid = X[len(X) // 2, :3]
    pts = np.array([mid + [0.1, 0.7, 0.0], mid + [2.0, -3.0, 0.5], [9.0, 9.0, 9.0]])
    ok, t = _clear_of_kinks(orc, P, x0, U, guide, goal, pts)
    assert ok, "scene too close to a non-differentiable point"
    band = (t["dist"] > P["d_min"]) & (t["dist"] < P["d_max"])
    assert band.sum() >= 2 and t["J_col"] > 0            # the collision term is exercised
    S, G = orc.cost_grad(x0, U, guide, goal, pts, P)
    assert abs(S - t["S"]) <= 1e-9 * abs(t["S"])
    G_fd = _fd(orc, P, x0, U, guide, goal, pts)
    err = np.abs(G - G_fd).max()
    assert err <= 1e-6 * np.abs(G).max() + 1e-3, err


def test_gradient_without_obstacles_matches_central_differences(orc):
    P, x0, U, guide, goal = _scene(3, T=20)
    pts = np.zeros((0, 3))
    ok, _ = _clear_of_kinks(orc, P, x0, U, guide, goal, pts)
    assert ok
    S, G = orc.cost_grad(x0, U, guide, goal, pts, P)
    G_fd = _fd(orc, P, x0, U, guide, goal, pts)
    assert np.abs(G - G_fd).max() <= 1e-6 * np.abs(G).max() + 1e-6


def test_gradient_with_long_steps_and_fast_rates(orc):
    """dt = 0.25 s with body rates of several rad/s: RK4 then changes |q| by
    far more than rounding, so the renormalisation's share of the gradient
    is visible to the finite differences."""
    P, x0, U, guide, goal = _scene(6, T=10)
    P["dt"] = 0.25
    rng = np.random.default_rng(7)
    U[:, 1:] = rng.normal(0, 4.0, (P["T"], 3))
    pts = np.zeros((0, 3))
    X = orc.rollout(x0, U, P["dt"], P["mass"], P["g"])
    guide = X[1:, :3] + [0.3, -0.2, 0.1]          # clear of the path, nonzero tracking error
    ok, _ = _clear_of_kinks(orc, P, x0, U, guide, goal, pts)
    assert ok
    S, G = orc.cost_grad(x0, U, guide, goal, pts, P)
    G_fd = _fd(orc, P, x0, U, guide, goal, pts)
    assert np.abs(G - G_fd).max() <= 1e-7 * np.abs(G).max() + 1e-6


def test_control_cost_gradient_closed_form(orc):
    """With every state weight and C_col zero, S = J_ctrl and dS/du_t is
    2 Q_c u_t (t <= T-2) + 2 Q_cd (u_t - u_{t-1}) - 2 Q_cd (u_{t+1} - u_t) over
    the stated index ranges; u_{T-1} has zero gradient."""
    P, x0, U, guide, goal = _scene(4)
    for k in ("Q_track", "Q_vnorm", "Q_p", "Q_v", "Q_q", "C_col"):
        P[k] = 0.0
    T = P["T"]
    S, G = orc.cost_grad(x0, U, guide, goal, np.zeros((0, 3)), P)
    ref = np.zeros_like(U)
    for t in range(T - 1):
        ref[t] += 2 * P["Q_c"] * U[t]
    for t in range(1, T - 1):
        ref[t] += 2 * P["Q_cd"] * (U[t] - U[t - 1])
        ref[t - 1] -= 2 * P["Q_cd"] * (U[t] - U[t - 1])
    assert np.abs(G - ref).max() < 1e-12
    assert np.all(G[T - 1] == 0.0)
    jc = sum(P["Q_c"] * U[t] @ U[t] for t in range(T - 1)) + \
        sum(P["Q_cd"] * (U[t] - U[t - 1]) @ (U[t] - U[t - 1]) for t in range(1, T - 1))
    assert abs(S - jc) < 1e-9 * jc


def test_hover_velocity_cost_has_zero_gradient(orc):
    """At hover (q = I, F = m g, w = 0) v stays exactly zero, so with only the
    velocity-norm term the cost and its gradient are exactly zero."""
    P, x0, U, guide, goal = _scene(5)
    for k in ("Q_track", "Q_c", "Q_cd", "Q_p", "Q_v", "Q_q", "C_col"):
        P[k] = 0.0
    x0 = np.array([0.0, 0.0, 1.5, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    U = np.tile([P["g"] * P["mass"], 0.0, 0.0, 0.0], (P["T"], 1))
    S, G = orc.cost_grad(x0, U, None, goal, np.zeros((0, 3)), P)
    assert S == 0.0 and np.all(G == 0.0)


def test_refinement_step_descends_and_stays_in_bounds(orc):
    P, x0, U, guide, goal = _scene(0)
    X = orc.rollout(x0, U, P["dt"], P["mass"], P["g"])
    mid = X[len(X) // 2, :3]
    pts = np.array([mid + [0.1, 0.7, 0.0]])
    S0, G = orc.cost_grad(x0, U, guide, goal, pts, P)
    step = 1e-3 / np.abs(G).max()
    U1 = orc.refine(x0, U, guide, goal, pts, dict(P, refine_steps=1, refine_step=step))
    ref = np.clip(U - step * G, P["u_min"], P["u_max"])
    assert np.abs(U1 - ref).max() < 1e-12
    S1 = _forward(orc, P, x0, U1, guide, goal, pts)["S"]
    assert S1 < S0
    U5 = orc.refine(x0, U, guide, goal, pts, dict(P, refine_steps=5, refine_step=50.0))
    assert np.all(U5 >= np.array(P["u_min"]) - 1e-12) and np.all(U5 <= np.array(P["u_max"]) + 1e-12)


def test_plan_step_refinement_is_the_stated_composition(orc):
    """plan_step with refine_steps = R equals the unrefined step's update,
    refined R times per instance with orc_refine, then Stage II."""
    w = I.make_workload("plain")
    P = dict(w.params, K=64, T=12)
    u0 = np.tile(w.hover_nominal()[:, :1, :], (1, P["T"], 1))
    a = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, P, u0)
    R = dict(P, refine_steps=3, refine_step=0.01)
    b = orc.plan_step(w.cloud, w.p0, w.q0, w.v0, w.goal, R, u0)
    x0 = np.concatenate([w.p0, w.q0, w.v0]).astype(np.float64)
    pts = orc.collision_set(w.cloud, w.p0, w.q0, a["keys"], P)
    for e in range(P["E"]):
        u = orc.refine(x0, a["u_nom"][e], a["guides"][e], w.goal.astype(np.float64), pts, R)
        assert np.abs(u - b["u_nom"][e]).max() < 1e-12
        X = orc.rollout(x0, u, P["dt"], P["mass"], P["g"])
        c = orc.cost_terms(X, u, None, w.goal.astype(np.float64), pts, P, stage=2)["S"]
        assert abs(c - b["cand"][e]) <= 1e-12 * max(1.0, abs(c))
