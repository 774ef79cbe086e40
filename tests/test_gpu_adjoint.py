"""GPU discrete adjoint (dmx_rollout_grad through the C ABI) against the CPU
oracle's discrete adjoint along the SAME accepted step sequence (the GPU's,
read back from the tape): 1e-6 relative, the gradient tolerance of the
workload spec, per environment (scale max(|g_i|, ||g||_inf)); with and
without the straight-through CFD treatment; interval-boundary cotangents;
checkpoint intervals; central differences of the frozen-step map (eps 1e-6)
for the arm's controls; the torch.autograd.Function."""

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W
from tests.conftest import rel_err
from tests.test_gpu_rollout import BILLIARD_TRANS

pytestmark = pytest.mark.gpu
TOL = 1e-6
CFD_OPT = dict(W.CFD_OPTIONS)
# CFD continuation only (the forward right-hand side keeps d(0) = 0, so contact
# forces stay continuous and the box pushes integrate with ordinary step sizes)
CFD_ONLY = dict(solimp_cfd=W.CFD_SOLIMP_CFD)


@pytest.fixture(scope="module")
def dmx():
    import torch
    from paper_2506_14186_gb300 import _build
    _build.build()
    import paper_2506_14186_gb300 as d
    assert torch.cuda.is_available()
    return d


@pytest.fixture(scope="module")
def orc_mod():
    import oracle
    oracle.build()
    return oracle


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_grad(dmx, model, inp, xT_bar, xb_bar=None, cfd=False, K=32, mode="reverse", method="dopri5"):
    """Taped GPU rollout + adjoint (reverse-mode or tangent kernel).  Arrays
    env-major in and out."""
    model.set_adjoint(mode)
    ctrl = None if inp["ctrl"] is None else _dev(np.transpose(inp["ctrl"], (1, 2, 0)))
    out = dmx.rollout(model, _dev(inp["x0"].T), _dev(inp["T"]), ctrl=ctrl, NI=inp["NI"], rtol=inp["rtol"],
                      atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"], K=K, tape=True, method=method)
    xbb = None if xb_bar is None else _dev(np.transpose(xb_bar, (1, 2, 0)))
    gx, gu = dmx.rollout_grad(out["tape"], _dev(xT_bar.T), xbb, cfd=cfd)
    hlog, n = out["tape"].read()
    res = {"x0_bar": gx.cpu().numpy().T, "hlog": hlog.cpu().numpy().T, "n": n.cpu().numpy(),
           "xT": out["xT"].cpu().numpy().T, "status": out["status"].cpu().numpy()}
    if gu is not None:
        res["ctrl_bar"] = np.transpose(gu.cpu().numpy(), (2, 0, 1))
    return res


def oracle_grad(orc_mod, scene, inp, g, xT_bar, xb_bar=None, cfd=False, method="dopri5"):
    m = orc_mod.OracleModel(scene)
    return m.batch_replay_grad(inp["x0"], inp["T"], g["hlog"], g["n"], xT_bar, ctrl=inp["ctrl"], NI=inp["NI"],
                               cfd=cfd, xb_bar=xb_bar, method=method)


def assert_grad(g, o, key="x0_bar"):
    B = len(o[key])
    err = max(rel_err(np.ravel(g[key][e]), np.ravel(o[key][e])) for e in range(B))
    assert err < TOL, f"{key}: relative error {err:.3e}"
    return err


MODES = ["reverse", "recompute", "tangent"]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("cfd", [False, True])
def test_ball_gradient(dmx, orc_mod, cfd, mode):
    """Bouncing balls (full batch, T = 1 s): gradient of the final height and
    velocity w.r.t. the whole initial state; with CFD parameters of App. E.3."""
    sc = W.ball_scene(**CFD_OPT) if cfd else W.ball_scene()
    inp = W.ball_inputs(16)
    rng = np.random.default_rng(0)
    xT_bar = rng.normal(size=(16, 13))
    m = dmx.Model(sc)
    g = gpu_grad(dmx, m, inp, xT_bar, cfd=cfd, mode=mode)
    o = oracle_grad(orc_mod, sc, inp, g, xT_bar, cfd=cfd)
    assert_grad(g, o)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("cfd", [False, True])
@pytest.mark.parametrize("K", [1, 7, 32])
def test_box_gradient(dmx, orc_mod, cfd, K, mode):
    """Box pushes over 0.1 s (about 240 accepted steps of sliding contact).
    The frozen-step gradient of these pushes is ill-conditioned beyond that:
    a 1e-16 relative change of x0 moves it by 3e-8 (0.15 s), 2e-7 (0.2 s)
    and 8e-7 (0.3 s) relative (tests/test_oracle_adjoint.py pins this), so
    the 1e-6 bar is checked where rounding cannot reach it."""
    sc = W.box_scene(**CFD_ONLY) if cfd else W.box_scene()
    inp = W.box_push_inputs(24, seed=5, T=0.1)
    rng = np.random.default_rng(1)
    xT_bar = rng.normal(size=(24, 13))
    m = dmx.Model(sc)
    g = gpu_grad(dmx, m, inp, xT_bar, cfd=cfd, K=K, mode=mode)
    assert np.all(g["status"] == 0)
    assert_grad(g, oracle_grad(orc_mod, sc, inp, g, xT_bar, cfd=cfd))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("cfd", [False, True])
def test_chain_control_gradient_with_boundary_cotangents(dmx, orc_mod, cfd, mode):
    """Arm + cube: loss on the cube's final position and on every
    interval-boundary state; gradient w.r.t. x0 and every control."""
    sc = W.chain_cube_scene(**CFD_OPT) if cfd else W.chain_cube_scene()
    inp = W.chain_inputs(8, T=0.24, NI=6)
    rng = np.random.default_rng(2)
    nx = 27
    xT_bar = rng.normal(size=(8, nx))
    xb_bar = rng.normal(size=(8, 7, nx))
    m = dmx.Model(sc)
    g = gpu_grad(dmx, m, inp, xT_bar, xb_bar=xb_bar, cfd=cfd, K=5, mode=mode)
    o = oracle_grad(orc_mod, sc, inp, g, xT_bar, xb_bar=xb_bar, cfd=cfd)
    assert_grad(g, o)
    assert_grad(g, o, "ctrl_bar")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("cfd", [False, True])
def test_arm_tilt_gradient(dmx, orc_mod, cfd, mode):
    """Tilted arm (capsule ends pressed into the plane, sliding with
    friction): gradient w.r.t. x0 and every control, loss on the final state
    and the interval-boundary states."""
    sc = W.arm_tilt_scene(**CFD_OPT) if cfd else W.arm_tilt_scene()
    inp = W.arm_tilt_inputs(8, T=0.24, NI=6)
    rng = np.random.default_rng(6)
    xT_bar = rng.normal(size=(8, 27))
    xb_bar = rng.normal(size=(8, 7, 27))
    m = dmx.Model(sc)
    g = gpu_grad(dmx, m, inp, xT_bar, xb_bar=xb_bar, cfd=cfd, K=5, mode=mode)
    o = oracle_grad(orc_mod, sc, inp, g, xT_bar, xb_bar=xb_bar, cfd=cfd)
    assert_grad(g, o)
    assert_grad(g, o, "ctrl_bar")


@pytest.mark.parametrize("mode", MODES)
def test_quadruped_gradient(dmx, orc_mod, mode):
    """19 + 18 coordinates and 12 servo targets: 49 input directions (two
    32-lane passes per step for the tangent kernel)."""
    sc = W.quadruped_scene()
    inp = W.quadruped_inputs(6)
    inp["T"] = np.minimum(inp["T"], 0.2)
    rng = np.random.default_rng(3)
    xT_bar = np.zeros((6, 37)); xT_bar[:, 0:3] = rng.normal(size=(6, 3))
    m = dmx.Model(sc)
    g = gpu_grad(dmx, m, inp, xT_bar, K=16, mode=mode)
    o = oracle_grad(orc_mod, sc, inp, g, xT_bar)
    assert_grad(g, o)
    assert_grad(g, o, "ctrl_bar")


def test_chain_gradient_matches_central_differences(dmx, orc_mod):
    """The workload's check: loss = squared cube-to-goal distance, gradient
    w.r.t. 16 controls of each of 8 environments against central differences
    (eps = 1e-6) of the frozen-step map (the GPU's step sizes replayed)."""
    sc = W.chain_cube_scene()
    inp = W.chain_inputs(8, T=0.4, NI=10)
    goal = W.chain_goal()
    m = dmx.Model(sc)
    om = orc_mod.OracleModel(sc)
    # first pass for the final cube position, then the loss cotangent
    g0 = gpu_grad(dmx, m, inp, np.zeros((8, 27)))
    xT_bar = np.zeros((8, 27)); xT_bar[:, 7:10] = 2 * (g0["xT"][:, 7:10] - goal)
    g = gpu_grad(dmx, m, inp, xT_bar)
    rng = np.random.default_rng(4)
    worst = 0.0
    for e in range(8):
        n = int(g["n"][e])
        idx = rng.choice(10 * 7, 16, replace=False)

        def loss(ctrl):
            xT, _ = om.replay(inp["x0"][e], g["hlog"][e, :n], ctrl=ctrl, T=float(inp["T"][e]), NI=10)
            return float(((xT[7:10] - goal) ** 2).sum())
        fd = []
        for j in idx:
            c = inp["ctrl"][e].copy().ravel(); c[j] += 1e-6
            lp = loss(c.reshape(10, 7))
            c[j] -= 2e-6
            lm = loss(c.reshape(10, 7))
            fd.append((lp - lm) / 2e-6)
        fd = np.array(fd)
        got = g["ctrl_bar"][e].ravel()[idx]
        scale = max(np.abs(g["ctrl_bar"][e]).max(), 1e-12)
        worst = max(worst, np.abs(got - fd).max() / scale)
    assert worst < 1e-5, worst


def test_autograd_function(dmx):
    import torch
    sc = W.chain_cube_scene()
    inp = W.chain_inputs(4, T=0.2, NI=5)
    m = dmx.Model(sc)
    x0 = _dev(inp["x0"].T).requires_grad_(True)
    ctrl = _dev(np.transpose(inp["ctrl"], (1, 2, 0))).requires_grad_(True)
    xT, xb, status = dmx.rollout_fn(m, x0, _dev(inp["T"]), ctrl=ctrl, NI=5, K=8)
    goal = torch.tensor(W.chain_goal(), device="cuda")[:, None]
    loss = ((xT[7:10] - goal) ** 2).sum() + 0.1 * (xb[:, 7:10] ** 2).sum() + (xT[0:7] ** 2).sum()
    loss.backward()
    assert x0.grad is not None and ctrl.grad is not None
    assert torch.isfinite(ctrl.grad).all() and ctrl.grad.abs().max() > 0
    # same as calling the adjoint directly with the loss cotangents
    out = dmx.rollout(m, x0.detach(), _dev(inp["T"]), ctrl=ctrl.detach(), NI=5, K=8, tape=True, want_xb=True)
    xT_bar = torch.zeros_like(out["xT"]); xT_bar[7:10] = 2 * (out["xT"][7:10] - goal)
    xT_bar[0:7] = 2 * out["xT"][0:7]
    xb_bar = torch.zeros_like(out["xb"]); xb_bar[:, 7:10] = 0.2 * out["xb"][:, 7:10]
    gx, gu = dmx.rollout_grad(out["tape"], xT_bar, xb_bar)
    assert torch.allclose(gx, x0.grad, rtol=1e-12, atol=0) and torch.allclose(gu, ctrl.grad, rtol=1e-12, atol=0)


TOL_VJP = 1e-10


@pytest.mark.parametrize("cfd", [False, True])
@pytest.mark.parametrize("name", ["ball", "box", "chain_cube", "quadruped", "billiard", "capsules", "arm_tilt"])
def test_rhs_vjp_matches_oracle_jacobian(dmx, orc_mod, name, cfd):
    """Right-hand-side VJP (dmx_eval_rhs_vjp) against the transposed Jacobian
    of the oracle's right-hand side (its derivative scalars) at states near
    contact (angular velocities included), for several lane counts."""
    from tests.test_gpu_rollout import SEEDS, _random_states, arm_tilt_states, pair_states
    sc = W.SCENES[name](**CFD_OPT) if cfd else W.SCENES[name]()
    B = 48
    om = orc_mod.OracleModel(sc)
    if name in ("billiard", "capsules"):          # states near the ball-ball / capsule contacts
        _, q, v = pair_states(orc_mod, name, B, 31)
        u = np.zeros((B, 1))
    elif name == "arm_tilt":                      # capsule ends pressed into the plane
        _, q, v, u = arm_tilt_states(orc_mod, B, 37)
    else:
        q, v, u = _random_states(sc, B, SEEDS[name] + 100, om)
    rng = np.random.default_rng(SEEDS.get(name, 40))   # (pair and tilted-arm scenes: 40)
    gm = dmx.Model(sc)
    abar = rng.normal(size=(B, gm.nv))
    ref_q, ref_v, ref_u = [], [], []
    for e in range(B):
        Jq, Jv, Ju = om.rhs_jacobian(q[e], v[e], u[e], cfd=cfd)
        ref_q.append(Jq.T @ abar[e]); ref_v.append(Jv.T @ abar[e]); ref_u.append(Ju.T @ abar[e])
    ref = [np.concatenate([ref_q[e], ref_v[e], ref_u[e]]) for e in range(B)]
    for lanes in ((8, 16, 32) if name in ("chain_cube", "quadruped", "capsules", "arm_tilt") else (2, 8, 32)):   # large workspaces need >= 8 lanes
        qb, vb, ub, st = dmx.eval_rhs_vjp(gm, _dev(q.T), _dev(v.T), _dev(abar.T),
                                          u=_dev(u[:, :gm.nu].T) if gm.nu else None, cfd=cfd, lanes=lanes)
        assert np.all(st.cpu().numpy() == 0)
        qb = qb.cpu().numpy().T; vb = vb.cpu().numpy().T
        ub = ub.cpu().numpy().T if gm.nu else np.zeros((B, 0))
        # one scale per state: the largest cotangent component, at least |abar|_inf (a state
        # out of contact has a Jacobian that vanishes up to rounding on both sides)
        err = 0.0
        for e in range(B):
            got = np.concatenate([qb[e], vb[e], ub[e]])
            scale = max(np.abs(ref[e]).max(), np.abs(abar[e]).max())
            err = max(err, np.abs(got - ref[e]).max() / scale)
        assert err < TOL_VJP, f"lanes {lanes}: {err:.3e}"


@pytest.mark.parametrize("name", ["box", "chain_cube"])
def test_reverse_kernel_equals_tangent_kernel(dmx, name):
    """The two adjoint kernels compute the same derivative on the same tape:
    they differ only in rounding, which the product of a few hundred step
    Jacobians of a stiff contact map amplifies (a 1e-12 difference per
    right-hand-side VJP grows to a few 1e-7 here), so they are compared at
    the gradient tolerance, the bar each of them meets against the oracle."""
    import torch
    sc = W.SCENES[name]()
    inp = W.box_push_inputs(64, seed=9, T=0.1) if name == "box" else W.chain_inputs(16, T=0.2, NI=4)
    m = dmx.Model(sc)
    ctrl = None if inp["ctrl"] is None else _dev(np.transpose(inp["ctrl"], (1, 2, 0)))
    out = dmx.rollout(m, _dev(inp["x0"].T), _dev(inp["T"]), ctrl=ctrl, NI=inp["NI"], rtol=inp["rtol"],
                      atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"], K=16, tape=True)
    xT_bar = torch.randn((m.nx, len(inp["T"])), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    res = {}
    for mode in MODES:
        m.set_adjoint(mode)
        res[mode] = dmx.rollout_grad(out["tape"], xT_bar)
    for k in range(2 if m.nu else 1):
        a = res["reverse"][k].cpu().numpy().reshape(-1, len(inp["T"])).T
        b = res["tangent"][k].cpu().numpy().reshape(-1, len(inp["T"])).T
        err = max(rel_err(a[e], b[e]) for e in range(len(a)))
        assert err < TOL, err
        # stage snapshots restore exactly what a second evaluation computes
        # (the final active set, hence the Newton system, is the same)
        c = res["recompute"][k].cpu().numpy().reshape(-1, len(inp["T"])).T
        np.testing.assert_array_equal(a, c)


def _oracle_along(orc_mod, scene, inp, idx, hlog, n, xT_bar, NI):
    m = orc_mod.OracleModel(scene)
    ctrl = None if inp["ctrl"] is None else inp["ctrl"][idx]
    return m.batch_replay_grad(inp["x0"][idx], inp["T"][idx], hlog, n, xT_bar, ctrl=ctrl, NI=NI)


def test_arm_gradient_at_the_benchmark_configuration(dmx, orc_mod):
    """The fwd+adjoint benchmark as it is timed: arm + cube, all 16384
    environments, T = 2 s, 50 torque intervals, K = 32, persistent forward and
    reverse adjoint with autotuned lanes; cotangent = gradient of the squared
    cube-to-goal distance plus a random cotangent on every final coordinate.
    Six sampled environments (four where the arm reaches the cube) against
    the oracle's discrete adjoint along the GPU's step sizes: 1e-6 on x0_bar
    and on all 350 control gradients.  (The oracle's own conditioning floor at
    this horizon is below 1e-7: tests/test_oracle_adjoint.py.)"""
    import torch
    from paper_2506_14186_gb300 import autotune
    sc, inp = W.chain_cube_scene(), W.chain_inputs(16384)
    B = 16384
    m = dmx.Model(sc)
    x0, T = _dev(inp["x0"].T), _dev(inp["T"])
    ctrl = _dev(np.transpose(inp["ctrl"], (1, 2, 0)))
    fl, _ = autotune.tune_forward(m, x0, torch.clamp(T, max=0.2), ctrl=ctrl, NI=50, candidates=(8, 16, 32))
    autotune.tune_adjoint(m, x0, T, ctrl=ctrl, NI=50, K=32)
    m.set_lanes(B, fl)
    m.set_adjoint("reverse")
    out = dmx.rollout(m, x0, T, ctrl=ctrl, NI=50, K=32, tape=True)
    assert int((out["status"] != 0).sum().item()) == 0
    rnd = torch.tensor(np.random.default_rng(21).normal(size=(27, B)) * 0.1, device="cuda")
    xT_bar = rnd.clone()
    xT_bar[7:10] += 2 * (out["xT"][7:10] - torch.tensor(W.chain_goal(), device="cuda")[:, None])
    gx, gu = dmx.rollout_grad(out["tape"], xT_bar)
    idx = np.array([0, 5, 7, 11, 8195, 16383])
    hlog, n = out["tape"].read()
    n = n.cpu().numpy()[idx]
    hl = hlog[: int(n.max()), torch.tensor(idx, device="cuda")].cpu().numpy().T
    o = _oracle_along(orc_mod, sc, inp, idx, hl, n, xT_bar.cpu().numpy().T[idx], NI=50)
    g = {"x0_bar": gx.cpu().numpy().T[idx], "ctrl_bar": np.transpose(gu.cpu().numpy(), (2, 0, 1))[idx]}
    assert np.count_nonzero(np.abs(o["ctrl_bar"]).reshape(len(idx), -1).max(axis=1) > 1e-3) >= 4
    assert_grad(g, o)
    assert_grad(g, o, "ctrl_bar")


def test_quadruped_gradient_at_full_horizons(dmx, orc_mod):
    """Quadruped at its workload's batch (8192 robots, horizons U[0.5, 3] s,
    autotuned lanes and checkpoint interval): the three robots with the
    longest horizons (~3 s, ~4000 steps each) against the oracle's discrete
    adjoint along the GPU's step sizes, 1e-6 (the oracle's conditioning floor
    there is ~1e-8)."""
    import torch
    from paper_2506_14186_gb300 import autotune
    sc, inp = W.quadruped_scene(), W.quadruped_inputs(8192)
    B = 8192
    m = dmx.Model(sc)
    x0, T = _dev(inp["x0"].T), _dev(inp["T"])
    ctrl = _dev(np.transpose(inp["ctrl"], (1, 2, 0)))
    kw = dict(ctrl=ctrl, NI=1)
    fl, _ = autotune.tune_forward(m, x0, torch.clamp(T, max=0.25), **kw)
    autotune.tune_adjoint(m, x0, T, K=32, **kw)
    K, _ = autotune.tune_checkpoint(m, x0, T, **kw)
    m.set_lanes(B, fl)
    m.set_adjoint("reverse")
    out = dmx.rollout(m, x0, T, K=K, tape=True, **kw)
    assert int((out["status"] != 0).sum().item()) == 0
    xT_bar = torch.zeros_like(out["xT"])
    xT_bar[0:3] = 1.0
    gx, gu = dmx.rollout_grad(out["tape"], xT_bar)
    idx = np.sort(np.argsort(-inp["T"])[:3])
    hlog, n = out["tape"].read()
    n = n.cpu().numpy()[idx]
    hl = hlog[: int(n.max()), torch.tensor(idx, device="cuda")].cpu().numpy().T
    o = _oracle_along(orc_mod, sc, inp, idx, hl, n, xT_bar.cpu().numpy().T[idx], NI=1)
    g = {"x0_bar": gx.cpu().numpy().T[idx], "ctrl_bar": np.transpose(gu.cpu().numpy(), (2, 0, 1))[idx]}
    assert_grad(g, o)
    assert_grad(g, o, "ctrl_bar")


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("method", ["tsit5", "euler"])
def test_other_schemes_gradient(dmx, orc_mod, method, mode):
    """Discrete adjoint of the Tsitouras and semi-implicit Euler rollouts in
    every adjoint kernel against the oracle along the GPU's steps: balls
    (1 s, with CFD), box pushes (0.1 s) and the arm (controls, boundary
    cotangents; 0.2 s), K = 3 so segments span several checkpoints."""
    rng = np.random.default_rng(11)
    for name, inp, cfd in (("ball", W.ball_inputs(8), True), ("box", W.box_push_inputs(12, seed=5, T=0.1), False),
                           ("chain_cube", W.chain_inputs(6, T=0.2, NI=4), False)):
        sc = W.SCENES[name](**CFD_OPT) if cfd else W.SCENES[name]()
        m = dmx.Model(sc)
        B = len(inp["x0"])
        xT_bar = rng.normal(size=(B, m.nx))
        xb_bar = rng.normal(size=(B, inp["NI"] + 1, m.nx)) if name == "chain_cube" else None
        g = gpu_grad(dmx, m, inp, xT_bar, xb_bar=xb_bar, cfd=cfd, K=3, mode=mode, method=method)
        assert np.all(g["status"] == 0)
        o = oracle_grad(orc_mod, sc, inp, g, xT_bar, xb_bar=xb_bar, cfd=cfd, method=method)
        assert_grad(g, o)
        if m.nu:
            assert_grad(g, o, "ctrl_bar")


# ---------------------------------------------------------------- model-parameter gradients
def gpu_grad_params(dmx, model, inp, xT_bar, xb_bar=None, cfd=False, K=8):
    ctrl = None if inp["ctrl"] is None else _dev(np.transpose(inp["ctrl"], (1, 2, 0)))
    out = dmx.rollout(model, _dev(inp["x0"].T), _dev(inp["T"]), ctrl=ctrl, NI=inp["NI"], rtol=inp["rtol"],
                      atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"], K=K, tape=True)
    xbb = None if xb_bar is None else _dev(np.transpose(xb_bar, (1, 2, 0)))
    gx, gu, pb, ps = dmx.rollout_grad_params(out["tape"], _dev(xT_bar.T), xbb, cfd=cfd)
    hlog, n = out["tape"].read()
    res = {"x0_bar": gx.cpu().numpy().T, "p_bar": pb.cpu().numpy().T, "p_sum": ps.cpu().numpy(),
           "hlog": hlog.cpu().numpy().T, "n": n.cpu().numpy(), "status": out["status"].cpu().numpy()}
    if gu is not None:
        res["ctrl_bar"] = np.transpose(gu.cpu().numpy(), (2, 0, 1))
    return res


def param_inputs(name):
    """Inputs where the parameter gradient is defined to rounding (the oracle's
    conditioning floor is pinned in tests/test_oracle_adjoint.py): balls,
    pushed boxes dropped 2 cm with a spin (tumbling onto edges and corners),
    the arm with the cube dropped 5 cm onto the plane, the quadruped over
    0.3 s.  A cube resting or sliding flat on its face (four coplanar vertex
    contacts) puts friction rows at the edge of the active set, where the
    parameter gradient is not defined to 1e-6."""
    if name == "ball":
        return W.ball_inputs(8)
    if name == "box":
        inp = W.box_push_inputs(12, seed=5, T=0.1)
        x0 = inp["x0"].copy()
        x0[:, 2] += 0.02
        x0[:, 10:13] = 3.0 * np.random.default_rng(1).normal(size=(12, 3))
        return dict(inp, x0=x0)
    if name == "chain_cube":
        inp = W.chain_inputs(6, T=0.2, NI=4)
        x0 = inp["x0"].copy()
        x0[:, 9] += 0.05
        return dict(inp, x0=x0)
    inp = W.quadruped_inputs(6)
    return dict(inp, T=np.minimum(inp["T"], 0.3))


@pytest.mark.parametrize("name,cfd", [("ball", False), ("ball", True), ("box", False), ("chain_cube", False),
                                      ("quadruped", False)])
def test_parameter_gradient_matches_oracle(dmx, orc_mod, name, cfd):
    """p_bar (solref, solimp, friction of every pair, body masses) of dmx_rollout_grad_params
    against the oracle's discrete adjoint along the GPU's steps (1e-6, per
    environment); the state and control gradients of the same call too; the
    in-library sum over environments equals the sum of the per-environment
    gradients."""
    sc = W.SCENES[name](**CFD_OPT) if cfd else W.SCENES[name]()
    inp = param_inputs(name)
    m = dmx.Model(sc)
    B = len(inp["x0"])
    rng = np.random.default_rng(17)
    xT_bar = rng.normal(size=(B, m.nx))
    g = gpu_grad_params(dmx, m, inp, xT_bar, cfd=cfd)
    assert np.all(g["status"] == 0)
    om = orc_mod.OracleModel(sc)
    assert m.params().shape == (om.nparams(),)
    o_ = sc["options"]
    expect = (list(o_["solref"]) + list(o_["solimp"][:4]) + [p["mu"] for p in sc["pairs"]]
              + [b["mass"] for b in sc["bodies"]] + [2 * g["size"][0] for g in sc["geoms"] if g["type"] == "box"])
    np.testing.assert_array_equal(m.params(), expect)
    o = om.batch_replay_grad(inp["x0"], inp["T"], g["hlog"], g["n"], xT_bar, ctrl=inp["ctrl"], NI=inp["NI"], cfd=cfd,
                             params=True)
    assert_grad(g, o, "p_bar")
    assert_grad(g, o)
    if m.nu:
        assert_grad(g, o, "ctrl_bar")
    np.testing.assert_allclose(g["p_sum"], g["p_bar"].sum(axis=0), rtol=1e-12, atol=1e-12 * np.abs(g["p_bar"]).max())
    if name == "ball":
        assert np.all(g["p_bar"][:, 6] == 0.0)         # frictionless: mu enters no row


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name,cfd", [("billiard", False), ("billiard", True), ("capsules", False)])
def test_pair_gradient(dmx, orc_mod, name, cfd, mode):
    """Discrete adjoint through ball-ball and capsule contacts (closest-point
    derivatives by the implicit-function theorem in the reverse kernel) in
    every adjoint kernel, against the oracle along the GPU's steps; the
    billiard also with the straight-through CFD gradient (contacts from
    distance between the balls)."""
    sc = W.SCENES[name](**CFD_OPT) if cfd else W.SCENES[name]()
    inp = W.INPUTS[name](12)
    m = dmx.Model(sc)
    xT_bar = np.random.default_rng(23).normal(size=(12, m.nx))
    if name == "billiard":
        # a loss on the balls' positions and linear velocities; their
        # orientations and spins are inert rounding residue (see the billiard
        # trajectory test), and so are the cotangents of the initial ones
        keep = np.zeros(m.nx, dtype=bool); keep[BILLIARD_TRANS] = True
        xT_bar[:, ~keep] = 0.0
    g = gpu_grad(dmx, m, inp, xT_bar, cfd=cfd, K=4, mode=mode)
    assert np.all(g["status"] == 0)
    o = oracle_grad(orc_mod, sc, inp, g, xT_bar, cfd=cfd)
    if name == "billiard":
        g["x0_bar"], o["x0_bar"] = g["x0_bar"][:, BILLIARD_TRANS], o["x0_bar"][:, BILLIARD_TRANS]
    assert_grad(g, o)
