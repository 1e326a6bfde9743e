"""The adjoint on the GPU (aero_cost_grad, the gradient refinement inside the
update, RolloutCost) against the FP64 oracle (orc_cost_grad, orc_refine) on the
same inputs: the GPU's own guides, nominals and control sequences, the
oracle's collision set.  Sequences whose oracle trajectory comes within
KINK_BAND of d_min or d_max (where J_col has a kink or a jump) are excluded
from the gradient comparison, as are samples on the jump in the cost
comparisons elsewhere."""
import numpy as np
import pytest

from paper_2509_17340_gb300 import inputs as I
from gpu_util import JUMP_BAND, TOL_COST_REL, x0_of

pytestmark = pytest.mark.gpu

KINK_BAND = 2e-3     # m: FP32 states differ from the FP64 ones by ~1e-5 m
TOL_GRAD = 2e-3      # relative to the largest gradient entry of the sequence


@pytest.fixture(scope="module")
def aero():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_17340_gb300 import build
    build.build()
    from paper_2509_17340_gb300 import aero as A
    return A


def _case(name, **upd):
    if name == "column":
        # the plain scene plus a thin column of points 0.75 m from the start,
        # inside (d_min, d_max): every rollout pays J_col from its first steps
        w = I.make_workload("refined")
        rng = np.random.default_rng(11)
        th, z = rng.uniform(0, 2 * np.pi, 300), rng.uniform(0.5, 2.5, 300)
        col = np.stack([0.75 + 0.08 * np.cos(th), 0.08 * np.sin(th), z], 1).astype(np.float32)
        w.cloud = np.ascontiguousarray(np.concatenate([w.cloud, col]), np.float32)
    else:
        w = I.make_workload(name)
    w.params.update(upd)
    return w


def _step(aero, w, u0=None, debug=0):
    import torch
    P = w.params
    dev = torch.device("cuda")
    pl = aero.Planner(E_max=P["E"], K_max=P["K"], T_max=P["T"],
                      fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=max(1, len(w.cloud)),
                      debug_samples_max=debug)
    cloud = torch.from_numpy(w.cloud).to(dev)
    un = torch.from_numpy(w.hover_nominal() if u0 is None else u0).to(dev)
    ub = torch.empty((P["T"], 4), device=dev)
    cand = torch.empty((P["E"],), device=dev)
    best = torch.empty((1,), dtype=torch.int32, device=dev)
    pl.plan_step(aero.state_struct(w.p0, w.q0, w.v0), cloud, w.goal, aero.params_struct(P),
                 un, ub, cand, best)
    torch.cuda.synchronize()
    return pl, un, cand, best


def _oracle_pts(orc, w):
    keys = orc.partition(w.cloud, w.p0, w.q0, w.params)[0]
    return orc.collision_set(w.cloud, w.p0, w.q0, keys, w.params)


def _clear(orc, w, U, guide, pts):
    P = w.params
    X = orc.rollout(x0_of(w), U, P["dt"], P["mass"], P["g"])
    t = orc.cost_terms(X, U, guide, w.goal.astype(np.float64), pts, P, stage=1, want_dist=True)
    d = t["dist"]
    return bool(np.all(np.abs(d - P["d_min"]) > KINK_BAND) and np.all(np.abs(d - P["d_max"]) > KINK_BAND)), t


@pytest.mark.parametrize("name", ["refined", "column"])
def test_cost_grad_matches_oracle_adjoint(aero, orc, name):
    import torch
    w = _case(name, K=256, T=20, refine_steps=0)
    P = w.params
    pl, un, _, _ = _step(aero, w)
    guides = pl.debug("GUIDES").reshape(P["E"], P["T"], 3).astype(np.float64) + w.p0
    pts = _oracle_pts(orc, w)
    rng = np.random.default_rng(0)
    checked = with_col = 0
    for e in range(P["E"]):
        base = un[e].cpu().numpy()
        seqs = [base] + [np.clip(base + rng.normal(0, [1.0, 0.8, 0.8, 0.8], base.shape),
                                 P["u_min"], P["u_max"]).astype(np.float32) for _ in range(3)]
        U = torch.from_numpy(np.stack(seqs)).cuda()
        S = torch.empty(len(seqs), device="cuda")
        G = torch.empty_like(U)
        pl.cost_grad(e, U, S, G)
        torch.cuda.synchronize()
        for i, u in enumerate(seqs):
            ok, t = _clear(orc, w, u.astype(np.float64), guides[e], pts)
            if not ok:
                continue
            S_o, G_o = orc.cost_grad(x0_of(w), u.astype(np.float64), guides[e],
                                     w.goal.astype(np.float64), pts, P)
            assert abs(float(S[i]) - S_o) <= TOL_COST_REL * abs(S_o), (e, i)
            g = G[i].cpu().numpy().astype(np.float64)
            err = np.abs(g - G_o).max()
            assert err <= TOL_GRAD * np.abs(G_o).max() + 1e-3, (e, i, err, np.abs(G_o).max())
            checked += 1
            with_col += t["J_col"] > 0
    assert checked >= P["E"]
    if name == "column":
        assert with_col >= P["E"]      # the collision gradient is exercised
    # costs only (no gradient buffer) agree with the costs of the full call
    U = un[:2].contiguous() if P["E"] >= 2 else un.contiguous()
    S1 = torch.empty(U.shape[0], device="cuda")
    S2 = torch.empty(U.shape[0], device="cuda")
    pl.cost_grad(0, U, S1, None)
    pl.cost_grad(0, U, S2, torch.empty_like(U))
    torch.cuda.synchronize()
    torch.testing.assert_close(S1, S2, rtol=1e-6, atol=0)
    pl.close()


def test_autograd_function_uses_the_adjoint(aero):
    import torch
    w = _case("refined", K=256, T=20, refine_steps=0)
    pl, un, _, _ = _step(aero, w)
    U = un[:3].clone().requires_grad_(True)
    wts = torch.tensor([1.0, -2.0, 0.5], device="cuda")
    S = aero.RolloutCost.apply(U, pl, 1)
    (wts * S).sum().backward()
    S_ref = torch.empty(3, device="cuda")
    G_ref = torch.empty_like(un[:3])
    pl.cost_grad(1, un[:3].contiguous(), S_ref, G_ref)
    torch.cuda.synchronize()
    assert torch.equal(S.detach(), S_ref)
    assert torch.equal(U.grad, wts[:, None, None] * G_ref)
    pl.close()


@pytest.mark.parametrize("alpha,steps,full", [(1e-6, 2, False), (0.05, 5, False), (0.05, 5, True)])
def test_refinement_matches_oracle_from_the_pre_refinement_nominal(aero, orc, alpha, steps, full):
    """The update writes its nominal to PRE_REFINE, refines it in place and
    runs Stage II on the result.  The oracle refines the same (GPU) nominal:
    with a tiny step the refined nominals agree to the gradient tolerance;
    with the configured 5 x 0.05 (gradients reach 1e6 near obstacles, so most
    components end on a bound) the bounds hold and Stage II agrees with the
    oracle's Stage II of the GPU's refined nominal.  `full`: the refined
    workload at its own sizes (K=1024, T=40), as the benchmark runs it; every
    instance clear of the jump band is compared."""
    sizes = {} if full else dict(K=256, T=20)
    w = _case("refined", refine_steps=steps, refine_step=alpha, **sizes)
    P = w.params
    pl, un, cand, best = _step(aero, w)
    pre = pl.debug("PRE_REFINE").reshape(P["E"], P["T"], 4).astype(np.float64)
    guides = pl.debug("GUIDES").reshape(P["E"], P["T"], 3).astype(np.float64) + w.p0
    pts = _oracle_pts(orc, w)
    u_gpu = un.cpu().numpy().astype(np.float64)
    lo, hi = np.array(P["u_min"]), np.array(P["u_max"])
    assert np.all(u_gpu >= lo - 1e-6) and np.all(u_gpu <= hi + 1e-6)
    compared = compared_s2 = 0
    for e in range(P["E"]):
        if alpha < 1e-3:
            ok, _ = _clear(orc, w, pre[e], guides[e], pts)
            if not ok:
                continue
            ref = orc.refine(x0_of(w), pre[e], guides[e], w.goal.astype(np.float64), pts, P)
            _, G0 = orc.cost_grad(x0_of(w), pre[e], guides[e], w.goal.astype(np.float64), pts, P)
            step_tol = steps * alpha * (TOL_GRAD * np.abs(G0).max() + 1e-3) + 1e-6
            assert np.abs(u_gpu[e] - ref).max() <= step_tol, e
            assert np.abs(u_gpu[e] - pre[e]).max() > 0 or np.abs(G0).max() * alpha < 1e-7
            compared += 1
        X = orc.rollout(x0_of(w), u_gpu[e], P["dt"], P["mass"], P["g"])
        t = orc.cost_terms(X, u_gpu[e], None, w.goal.astype(np.float64), pts, P, stage=2,
                           want_dist=True)
        if np.min(np.abs(t["dist"] - P["d_max"])) > JUMP_BAND:
            assert abs(float(cand[e]) - t["S"]) <= TOL_COST_REL * abs(t["S"]), e
            compared_s2 += 1
    if alpha < 1e-3:
        assert compared >= P["E"] // 2
    assert compared_s2 >= 1
    c = cand.cpu().numpy()
    assert int(best.cpu()[0]) == int(np.argmin(c))
    pl.close()


def test_batched_refinement_matches_oracle(aero, orc):
    import torch
    ws = I.batch_workloads(4, seed=7)
    for w in ws:
        w.params.update(K=256, T=20, refine_steps=2, refine_step=1e-6, lanes_per_sample=1)
    dev = torch.device("cuda")
    lim = dict(E_max=16, K_max=256, T_max=20, fine_cells_max=128 * 64,
               n_points_max=max(len(w.cloud) for w in ws))
    batch = aero.Batch(len(ws), **lim)
    bufs = [(torch.from_numpy(w.cloud).to(dev), torch.from_numpy(w.hover_nominal()).to(dev),
             torch.empty((20, 4), device=dev), torch.empty((w.params["E"],), device=dev),
             torch.empty((1,), dtype=torch.int32, device=dev)) for w in ws]
    items = [aero.Batch.item(aero.state_struct(w.p0, w.q0, w.v0), b[0], w.goal,
                             aero.params_struct(w.params), b[1], b[2], b[3], b[4])
             for w, b in zip(ws, bufs)]
    batch.plan(items)
    torch.cuda.synchronize()
    compared = 0
    for i, (w, b) in enumerate(zip(ws, bufs)):
        P = w.params
        pre = batch.debug(i, "PRE_REFINE").reshape(P["E"], P["T"], 4).astype(np.float64)
        guides = batch.debug(i, "GUIDES").reshape(P["E"], P["T"], 3).astype(np.float64) + w.p0
        pts = _oracle_pts(orc, w)
        u_gpu = b[1].cpu().numpy().astype(np.float64)
        for e in range(P["E"]):
            ok, _ = _clear(orc, w, pre[e], guides[e], pts)
            if not ok:
                continue
            ref = orc.refine(x0_of(w), pre[e], guides[e], w.goal.astype(np.float64), pts, P)
            _, G0 = orc.cost_grad(x0_of(w), pre[e], guides[e], w.goal.astype(np.float64), pts, P)
            tol = 2 * 1e-6 * (TOL_GRAD * np.abs(G0).max() + 1e-3) + 1e-6
            assert np.abs(u_gpu[e] - ref).max() <= tol, (i, e)
            compared += 1
    assert compared >= 4
    batch.close()


def test_invalid_refinement_and_cost_grad_arguments(aero):
    import torch
    w = _case("refined", K=64, T=10, refine_steps=0)
    pl, un, _, _ = _step(aero, w)
    S = torch.empty(1, device="cuda")
    with pytest.raises(aero.AeroError) as ei:
        pl.cost_grad(w.params["E"], un[:1].contiguous(), S)     # instance out of range
    assert ei.value.code == aero.ERR_INVALID_ARG
    for upd in (dict(refine_steps=-1), dict(refine_steps=65), dict(refine_step=-0.1),
                dict(refine_step=float("nan"))):
        P = dict(w.params, **upd)
        ub = torch.empty((P["T"], 4), device="cuda")
        c = torch.empty((P["E"],), device="cuda")
        bi = torch.empty((1,), dtype=torch.int32, device="cuda")
        with pytest.raises(aero.AeroError) as ei:
            pl.plan_step(aero.state_struct(w.p0, w.q0, w.v0), torch.from_numpy(w.cloud).cuda(),
                         w.goal, aero.params_struct(P), un, ub, c, bi)
        assert ei.value.code == aero.ERR_INVALID_ARG, upd
    pl.close()


# ----------------------------------------------------------------- equidistant points

def _tie_case(**upd):
    """Two points mirrored across the plane y = 0 (at y = +-0.6 m, 1.07 m ahead)
    and a start moving along +x with zero body rates and no rate noise: every
    state of every rollout stays exactly on y = 0, so both points are at
    exactly the same binary32 distance from it.  They fall in different fine
    cones; the oracle takes the one of lower index in the collision set (the
    lower cone, y = -0.6), and so must the GPU, whatever the order of the
    entries in the cell's list.  The choice flips the sign of the collision
    gradient's lateral part."""
    w = I.make_workload("refined")
    far = I.random_cloud(200, seed=5, centre=(0.0, 0.0, 1.5), spread=9.0)
    far = far[np.linalg.norm(far - w.p0, axis=1) > 4.0]
    pair = np.array([[1.07, 0.6, 1.5], [1.07, -0.6, 1.5]], np.float32)
    w.cloud = np.ascontiguousarray(np.concatenate([pair, far]), np.float32)
    w.v0 = np.array([3.0, 0.0, 0.0], np.float32)
    w.params.update(K=64, T=20, sigma=[2.0, 0.0, 0.0, 0.0], refine_steps=0)
    w.params.update(upd)
    return w


def test_tied_nearest_points_follow_the_collision_set_order(aero, orc):
    """aero_cost_grad (one warp per sequence) at exact ties: the gradient is
    the oracle's, which takes the lower-index point, and differs from the one
    the other point would give."""
    import torch
    w = _tie_case()
    P = w.params
    pl, un, _, _ = _step(aero, w)
    guides = pl.debug("GUIDES").reshape(P["E"], P["T"], 3).astype(np.float64) + w.p0
    pts = _oracle_pts(orc, w)
    lower = int(np.argmin([np.linalg.norm(p - [1.07, -0.6, 1.5]) for p in pts]))
    upper = int(np.argmin([np.linalg.norm(p - [1.07, 0.6, 1.5]) for p in pts]))
    assert lower < upper      # the y = -0.6 point comes first in the collision set
    hover = np.zeros((P["T"], 4), np.float32)
    hover[:, 0] = P["mass"] * P["g"]
    U = torch.from_numpy(np.stack([hover])).cuda()
    S = torch.empty(1, device="cuda")
    G = torch.empty_like(U)
    for e in range(P["E"]):
        pl.cost_grad(e, U, S, G)
        torch.cuda.synchronize()
        ok, t = _clear(orc, w, hover.astype(np.float64), guides[e], pts)
        assert ok and t["J_col"] > 0
        S_o, G_o = orc.cost_grad(x0_of(w), hover.astype(np.float64), guides[e],
                                 w.goal.astype(np.float64), pts, P)
        swapped = pts.copy()
        swapped[[lower, upper]] = swapped[[upper, lower]]
        _, G_alt = orc.cost_grad(x0_of(w), hover.astype(np.float64), guides[e],
                                 w.goal.astype(np.float64), swapped, P)
        tol = TOL_GRAD * np.abs(G_o).max() + 1e-3
        assert np.abs(G_alt - G_o).max() > 10 * tol      # the tie decides the gradient
        g = G[0].cpu().numpy().astype(np.float64)
        assert abs(float(S[0]) - S_o) <= TOL_COST_REL * abs(S_o)
        assert np.abs(g - G_o).max() <= tol, e
    pl.close()


@pytest.mark.parametrize("batched", [False, True])
def test_tied_nearest_points_in_the_refinement(aero, orc, batched):
    """The refinement inside the update (the whole CTA; candidate entries as
    item indices in a single planner's step, as the points themselves in a
    batched step, where the winner's point is found by a second pass) at the
    same exact ties: one tiny step equals the oracle's step from the GPU's
    pre-refinement nominal."""
    import torch
    alpha = 1e-6
    w = _tie_case(refine_steps=1, refine_step=alpha)
    P = w.params
    if batched:
        dev = torch.device("cuda")
        batch = aero.Batch(1, E_max=P["E"], K_max=P["K"], T_max=P["T"],
                           fine_cells_max=P["fine_az"] * P["fine_el"], n_points_max=len(w.cloud))
        un = torch.from_numpy(w.hover_nominal()).to(dev)
        bufs = (torch.from_numpy(w.cloud).to(dev), torch.empty((P["T"], 4), device=dev),
                torch.empty((P["E"],), device=dev), torch.empty((1,), dtype=torch.int32, device=dev))
        batch.plan([aero.Batch.item(aero.state_struct(w.p0, w.q0, w.v0), bufs[0], w.goal,
                                    aero.params_struct(P), un, bufs[1], bufs[2], bufs[3])])
        torch.cuda.synchronize()
        pre = batch.debug(0, "PRE_REFINE").reshape(P["E"], P["T"], 4).astype(np.float64)
        guides = batch.debug(0, "GUIDES").reshape(P["E"], P["T"], 3).astype(np.float64) + w.p0
    else:
        pl, un, _, _ = _step(aero, w)
        pre = pl.debug("PRE_REFINE").reshape(P["E"], P["T"], 4).astype(np.float64)
        guides = pl.debug("GUIDES").reshape(P["E"], P["T"], 3).astype(np.float64) + w.p0
    pts = _oracle_pts(orc, w)
    u_gpu = un.cpu().numpy().astype(np.float64)
    compared = 0
    for e in range(P["E"]):
        assert np.all(pre[e][:, 1:] == 0.0)      # no rate noise: the nominal stays in the plane
        ok, t = _clear(orc, w, pre[e], guides[e], pts)
        if not ok or t["J_col"] == 0:
            continue
        ref = orc.refine(x0_of(w), pre[e], guides[e], w.goal.astype(np.float64), pts, P)
        _, G0 = orc.cost_grad(x0_of(w), pre[e], guides[e], w.goal.astype(np.float64), pts, P)
        tol = alpha * (TOL_GRAD * np.abs(G0).max() + 1e-3) + 1e-6
        assert np.abs(u_gpu[e] - ref).max() <= tol, e
        compared += 1
    assert compared >= P["E"] // 2
    if batched:
        batch.close()
    else:
        pl.close()
