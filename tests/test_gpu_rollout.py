"""GPU forward path (CUDA kernels through the C ABI) against the CPU oracle on
the same seeded inputs.

Levels of parity:
  * right-hand side v' = F(q, v, u) (and F~) on random states: 1e-11 relative;
  * every accepted step of every trajectory: the oracle takes one step of the
    GPU's accepted size from the GPU's own state (tape with a checkpoint after
    every step) and must land on the GPU's next state: 1e-11 relative;
  * whole trajectories in replay mode (the oracle integrates with the GPU's
    accepted step sizes): 1e-9 relative (the trajectory tolerance of the
    workload spec) for the non-chaotic ball over its full horizon and for the
    first 50 ms of the contact-rich workloads.  Beyond that, tumbling boxes,
    flailing arms and walking feet amplify any rounding difference: the
    oracle's own replay moves by 1e-9 .. 3e-8 when x0 is perturbed by 1e-15
    (see tests/test_oracle_integrator.py::test_chaos_floor), so no two implementations with
    different rounding agree to 1e-9 at T = 1 s;
  * free-running trajectories (each side takes its own step decisions): the
    GPU's step sequence is valid (the oracle's error norm accepts every GPU
    step); states within 1e-4 relative for the ball, arm and quadruped batches;
    for the tumbling boxes, whose free-running states depend on the step
    sequence through that chaos, statuses and step-count statistics.
Relative errors use the per-environment scale max(|x_i|, ||x||_inf).
Also: bitwise equality of launch forms, alone vs. in a batch, host vs. device
buffers; status codes; empty batches.
"""

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W
from tests.conftest import rel_err

pytestmark = pytest.mark.gpu
TOL_RHS = 1e-11
TOL_REPLAY = 1e-9
TOL_FREE = 1e-4
TOL_STEP = 1e-11
CFD_OPT = dict(W.CFD_OPTIONS)


@pytest.fixture(scope="module")
def dmx():
    import torch
    from paper_2506_14186_gb300 import _build
    _build.build()
    import paper_2506_14186_gb300 as d
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return d


@pytest.fixture(scope="module")
def orc_mod():
    import oracle
    oracle.build()
    return oracle


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _sub(inp, idx):
    out = dict(inp)
    out["x0"] = inp["x0"][idx]
    out["T"] = inp["T"][idx]
    if inp["ctrl"] is not None:
        out["ctrl"] = inp["ctrl"][idx]
    return out


def gpu_rollout(dmx, model, inp, tape=False, **kw):
    ctrl = None if inp["ctrl"] is None else _dev(np.transpose(inp["ctrl"], (1, 2, 0)))   # [B,NI,nu] -> [NI,nu,B]
    args = dict(NI=inp["NI"], rtol=inp["rtol"], atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"])
    args.update(kw)
    out = dmx.rollout(model, _dev(inp["x0"].T), _dev(inp["T"]), ctrl=ctrl, tape=tape, **args)
    res = {k: v.cpu().numpy() for k, v in out.items() if k != "tape" and v is not None}
    res["xT"] = res["xT"].T
    if "xb" in res:
        res["xb"] = np.transpose(res["xb"], (2, 0, 1))
    if tape:
        hlog, n, ck = out["tape"].read(checkpoints=True)
        res["hlog"] = hlog.cpu().numpy().T
        res["tape_n"] = n.cpu().numpy()
        res["ckpt"] = np.transpose(ck.cpu().numpy(), (2, 0, 1))      # [B, ncheck, nx+1]
    return res


def oracle_free(orc_mod, scene, inp, want_xb=False, method="dopri5"):
    m = orc_mod.OracleModel(scene)
    return m.batch_rollout(inp["x0"], inp["T"], ctrl=inp["ctrl"], NI=inp["NI"], rtol=inp["rtol"], atol=inp["atol"],
                           h0=inp["h0"], max_steps=inp["max_steps"], want_xb=want_xb, method=method)


def _sel(x, comps):
    return x if comps is None else np.asarray(x)[..., comps]


def assert_replay_parity(orc_mod, scene, inp, g, envs=None, method="dopri5", comps=None):
    """The oracle replays each environment's GPU step sequence (state
    components comps, default all)."""
    m = orc_mod.OracleModel(scene)
    envs = range(len(inp["x0"])) if envs is None else envs
    worst = 0.0
    for e in envs:
        n = int(g["tape_n"][e])
        assert n == g["nsteps"][e]
        ctrl = None if inp["ctrl"] is None else inp["ctrl"][e]
        xT, xb = m.replay(inp["x0"][e], g["hlog"][e, :n], ctrl=ctrl, T=float(inp["T"][e]), NI=inp["NI"],
                          method=method)
        worst = max(worst, rel_err(_sel(g["xT"][e], comps), _sel(xT, comps)))
        if "xb" in g:
            for k in range(inp["NI"] + 1):
                worst = max(worst, rel_err(_sel(g["xb"][e, k], comps), _sel(xb[k], comps)))
    assert worst < TOL_REPLAY, f"replay-mode relative error {worst:.3e}"
    return worst


def _interval(T, NI, t):
    k = 0
    while k + 1 < NI and t >= (T if k + 1 >= NI else T * (k + 1) / NI):
        k += 1
    return k


def assert_stepwise_parity(orc_mod, scene, inp, g, envs=None, check_valid=True, method="dopri5", comps=None):
    """Each accepted GPU step, started from the GPU's state, against one oracle
    step of the same size (tape with checkpoint interval 1); and the oracle's
    error norm of each of those steps is <= 1 (the step would be accepted)."""
    m = orc_mod.OracleModel(scene)
    nx = m.nx
    envs = range(len(inp["x0"])) if envs is None else envs
    worst, count, worst_err = 0.0, 0, 0.0
    for e in envs:
        n = int(g["tape_n"][e])
        ck = g["ckpt"][e]
        T = float(inp["T"][e])
        for s_ in range(n):
            xs, ts, h = ck[s_, :nx], ck[s_, nx], g["hlog"][e, s_]
            ctrl = None
            if inp["ctrl"] is not None:
                ctrl = inp["ctrl"][e][_interval(T, inp["NI"], ts)][None, :]
            xo, _ = m.replay(xs, [h], ctrl=ctrl, T=h, NI=1, method=method)
            worst = max(worst, rel_err(_sel(ck[s_ + 1, :nx], comps), _sel(xo, comps)))
            # the GPU's step sequence is a valid one: the oracle's error norm accepts each step
            if check_valid:
                err = m.step_error(xs, h, u=None if ctrl is None else ctrl[0], rtol=inp["rtol"], atol=inp["atol"],
                                   method=method)
                worst_err = max(worst_err, err)
            count += 1
    assert count > 0
    assert worst < TOL_STEP, f"per-step relative error {worst:.3e} over {count} steps"
    if check_valid:
        assert worst_err <= 1.0 + 1e-9, f"an accepted GPU step has oracle error norm {worst_err}"
    return worst


def assert_step_statistics(g, o):
    """Chaotic workloads (tumbling boxes): free-running states are not compared
    per environment (see the module note); statuses must agree and the
    accepted-step counts agree in distribution."""
    np.testing.assert_array_equal(g["status"], o["status"])
    ratio = g["nsteps"] / np.maximum(o["nsteps"], 1)
    assert abs(np.median(ratio) - 1) < 0.05 and abs(g["nsteps"].mean() / o["nsteps"].mean() - 1) < 0.05


def assert_free_parity(g, o, comps=None, ratio_tol=0.1):
    np.testing.assert_array_equal(g["status"], o["status"])
    err = max(rel_err(_sel(g["xT"][e], comps), _sel(o["xT"][e], comps)) for e in range(len(o["xT"])))
    assert err < TOL_FREE, f"free-running relative error {err:.3e}"
    ratio = g["nsteps"] / np.maximum(o["nsteps"], 1)
    assert np.all(np.abs(ratio - 1) < ratio_tol), ratio


# ---------------------------------------------------------------- right-hand side
SEEDS = {"ball": 11, "box": 12, "chain_cube": 13, "quadruped": 14}


def _axis_clear(om, q, scene):
    """Every capsule-box slot keeps the capsule axis 10 mm outside the box: a
    capsule axis inside a box puts the minimum of the (piecewise-linear) box
    distance field on a kink, where the contact normal is not unique."""
    ct = om.contacts(q)
    for p_i, p in enumerate(scene["pairs"]):
        if p["geom2"] >= 0:
            slot = sum(1 if (pp["geom2"] >= 0 or scene["geoms"][pp["geom1"]]["type"] == "sphere") else
                       (2 if scene["geoms"][pp["geom1"]]["type"] == "capsule" else 8) for pp in scene["pairs"][:p_i])
            if ct[slot, 0] < -scene["geoms"][p["geom1"]]["size"][0] + 0.01:
                return False
    return True


def _random_states(scene, B, seed, om=None):
    """States near contact: free bodies 0-3 mm into the plane or just above,
    hinges within +-0.5 rad; states whose capsule axis comes within 10 mm of a
    box are drawn again (see _axis_clear)."""
    q, v, u = _draw_states(scene, B, seed)
    if om is not None:
        for e in range(B):
            k = 0
            while not _axis_clear(om, q[e], scene):
                k += 1
                q[e] = _draw_states(scene, 1, seed * 1000 + e * 50 + k)[0][0]
    return q, v, u


def _draw_states(scene, B, seed):
    g = np.random.default_rng(seed)
    nq = sum(7 if b["joint"] == "free" else 1 for b in scene["bodies"])
    nv = sum(6 if b["joint"] == "free" else 1 for b in scene["bodies"])
    q = np.tile(np.array(scene["qpos0"], float), (B, 1))
    qa = 0
    for b in scene["bodies"]:
        if b["joint"] == "free":
            q[:, qa:qa + 2] += g.normal(scale=0.1, size=(B, 2))
            z0 = q[0, qa + 2]
            q[:, qa + 2] = z0 + g.uniform(-0.003, 0.002, B)
            qq = g.normal(size=(B, 4)) * 0.05
            qq[:, 0] += 1.0
            q[:, qa + 3:qa + 7] = qq / np.linalg.norm(qq, axis=1, keepdims=True)
            qa += 7
        else:
            q[:, qa] = g.uniform(-0.5, 0.5, B)
            qa += 1
    v = g.normal(scale=0.5, size=(B, nv))
    u = g.normal(size=(B, max(1, len(scene["actuators"]))))
    return q, v, u


@pytest.mark.parametrize("cfd", [False, True])
@pytest.mark.parametrize("name", ["ball", "box", "chain_cube", "quadruped"])
def test_rhs_matches_oracle(dmx, orc_mod, name, cfd):
    sc = W.SCENES[name](**CFD_OPT) if cfd else W.SCENES[name]()
    B = 96
    om = orc_mod.OracleModel(sc)
    q, v, u = _random_states(sc, B, SEEDS[name], om)
    gm = dmx.Model(sc)
    ref = np.array([om.rhs(q[e], v[e], u[e], cfd=cfd) for e in range(B)])
    nrows = np.array([om.rhs(q[e], v[e], u[e], cfd=cfd, detail=True)[1]["nr"] for e in range(B)])
    assert nrows.max() > 0
    for lanes in ((8, 16, 32) if name == "chain_cube" else (4, 8, 16, 32)):   # wider lanes where the workspace is large
        a, info = dmx.eval_rhs(gm, _dev(q.T), _dev(v.T), _dev(u[:, :gm.nu].T) if gm.nu else None, cfd=cfd, lanes=lanes)
        a = a.cpu().numpy().T
        info = info.cpu().numpy()
        assert np.all(info[0] == 0)
        np.testing.assert_array_equal(info[1], nrows)
        err = max(rel_err(a[e], ref[e]) for e in range(B))
        assert err < TOL_RHS, f"lanes {lanes}: {err:.3e}"


# ---------------------------------------------------------------- trajectories
def _short(inp, T=0.05):
    out = dict(inp)
    out["T"] = np.minimum(inp["T"], T)
    return out


def test_ball_batch(dmx, orc_mod):
    """Bouncing balls, the full batch of 16 (T = 1 s, rtol 1e-6, atol 1e-8):
    non-chaotic, so the whole trajectory is replayed at 1e-9."""
    sc, inp = W.ball_scene(), W.ball_inputs(16)
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp, tape=True, K=1)
    assert_stepwise_parity(orc_mod, sc, inp, g)
    assert_replay_parity(orc_mod, sc, inp, g)
    assert_free_parity(gpu_rollout(dmx, m, inp), oracle_free(orc_mod, sc, inp))


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_box_push_every_lane_count(dmx, orc_mod, lanes):
    """Box pushes (8 vertex contacts, pyramidal friction): 100 environments
    (several warps and a ragged tail) with each lane count."""
    sc = W.box_scene()
    inp = _sub(W.box_push_inputs(4096), np.arange(100))
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp, tape=True, K=1, lanes=lanes)
    assert_stepwise_parity(orc_mod, sc, inp, g)
    f = gpu_rollout(dmx, m, inp, lanes=lanes)
    np.testing.assert_array_equal(f["xT"], g["xT"])          # the tape does not change the arithmetic
    assert_step_statistics(f, oracle_free(orc_mod, sc, inp))
    s = _short(inp)
    assert_replay_parity(orc_mod, sc, s, gpu_rollout(dmx, m, s, tape=True, lanes=lanes))


def test_box_push_full_batch_sampled(dmx, orc_mod):
    """The benchmark configuration (4096 environments, persistent form,
    autotuned lanes): 64 sampled environments, every step and free-running."""
    sc, inp = W.box_scene(), W.box_push_inputs(4096)
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp)
    assert np.all(g["status"] == 0)
    gt = gpu_rollout(dmx, m, dict(inp, max_steps=2500), tape=True, K=1)
    np.testing.assert_array_equal(g["xT"], gt["xT"])
    idx = np.sort(np.random.default_rng(0).choice(4096, 64, replace=False))
    assert_stepwise_parity(orc_mod, sc, inp, gt, envs=idx)
    sub = _sub(inp, idx)
    assert_step_statistics({k: v[idx] for k, v in g.items()}, oracle_free(orc_mod, sc, sub))


def test_chain_cube(dmx, orc_mod):
    """Arm + cube with piecewise-constant torques (0.04 s intervals as in the
    2 s / 50-interval workload), interval-boundary states included."""
    sc = W.chain_cube_scene()
    inp = W.chain_inputs(24, T=0.4, NI=10)
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp, tape=True, K=1, want_xb=True)
    assert_stepwise_parity(orc_mod, sc, inp, g)
    assert_free_parity(gpu_rollout(dmx, m, inp), oracle_free(orc_mod, sc, inp))
    s = W.chain_inputs(24, T=0.08, NI=2)
    assert_replay_parity(orc_mod, sc, s, gpu_rollout(dmx, m, s, tape=True, want_xb=True))


def test_quadruped(dmx, orc_mod):
    sc = W.quadruped_scene()
    inp = W.quadruped_inputs(16)
    inp["T"] = np.minimum(inp["T"], 0.6)
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp, tape=True, K=1)
    assert_stepwise_parity(orc_mod, sc, inp, g)
    assert_free_parity(gpu_rollout(dmx, m, inp), oracle_free(orc_mod, sc, inp))
    s = _short(inp)
    assert_replay_parity(orc_mod, sc, s, gpu_rollout(dmx, m, s, tape=True))


def arm_tilt_states(orc_mod, B, seed):
    """States of the tilted arm (capsule ends pressed into the plane) along
    the oracle's trajectories, jittered by 1e-4 (hinges) / 1e-3 (velocities)."""
    sc = W.arm_tilt_scene()
    om = orc_mod.OracleModel(sc)
    inp = W.arm_tilt_inputs(B, seed=seed)
    g = np.random.default_rng(seed)
    Q, V, U = [], [], []
    for e in range(B):
        r = om.rollout(inp["x0"][e], ctrl=inp["ctrl"][e], T=0.5, NI=inp["NI"])
        xb = r["xb"][1 + e % inp["NI"]]
        Q.append(xb[:om.nq] + 1e-4 * g.normal(size=om.nq) * (np.arange(om.nq) < 7))
        V.append(xb[om.nq:] + 1e-3 * g.normal(size=om.nv))
        U.append(inp["ctrl"][e][e % inp["NI"]])
    return sc, np.array(Q), np.array(V), np.array(U)


@pytest.mark.parametrize("cfd", [False, True])
def test_arm_tilt_rhs_matches_oracle(dmx, orc_mod, cfd):
    """Capsule-plane penetration with friction on hinge chains: the tilted
    arm's links pressed into the plane at states along its trajectories.
    The hinges move the pressed capsule ends almost parallel to the plane
    (the tilt is 0.015 rad), so the normal rows' Jacobians are small against
    their forces and the right-hand side is ill-conditioned: the oracle's own
    value moves by ~3e-11 (up to 2e-10) when q and v move by 1e-15 relative.
    Each state's bar is therefore max(1e-11, 10x that measured floor)."""
    sc, q, v, u = arm_tilt_states(orc_mod, 48, 31)
    if cfd:
        sc = W.arm_tilt_scene(**CFD_OPT)
    om = orc_mod.OracleModel(sc)
    plane = np.array([om.contacts(q[e])[-14:, 0].min() for e in range(len(q))])
    assert (plane < 0).mean() > 0.9                         # capsule ends in the plane
    ref = np.array([om.rhs(q[e], v[e], u[e], cfd=cfd) for e in range(len(q))])
    nrows = np.array([om.rhs(q[e], v[e], u[e], cfd=cfd, detail=True)[1]["nr"] for e in range(len(q))])
    rng = np.random.default_rng(0)
    floor = np.zeros(len(q))
    for e in range(len(q)):
        for _ in range(4):
            qp = q[e] * (1 + 1e-15 * rng.normal(size=q.shape[1]))
            vp = v[e] * (1 + 1e-15 * rng.normal(size=v.shape[1]))
            floor[e] = max(floor[e], rel_err(om.rhs(qp, vp, u[e], cfd=cfd), ref[e]))
    assert np.median(floor) < 1e-9
    bar = np.maximum(TOL_RHS, 10 * floor)
    gm = dmx.Model(sc)
    for lanes in (8, 16, 32):
        a, info = dmx.eval_rhs(gm, _dev(q.T), _dev(v.T), _dev(u.T), cfd=cfd, lanes=lanes)
        a, info = a.cpu().numpy().T, info.cpu().numpy()
        assert np.all(info[0] == 0)
        np.testing.assert_array_equal(info[1], nrows)
        ratio = max(rel_err(a[e], ref[e]) / bar[e] for e in range(len(q)))
        assert ratio < 1.0, f"lanes {lanes}: {ratio:.3f} of the per-state bar"


def test_arm_tilt_trajectories(dmx, orc_mod):
    """Tilted arm over 0.5 s (10 torque intervals): every step, free running,
    and the replayed first 50 ms."""
    sc = W.arm_tilt_scene()
    inp = W.arm_tilt_inputs(24)
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp, tape=True, K=1, want_xb=True)
    assert np.all(g["status"] == 0)
    assert_stepwise_parity(orc_mod, sc, inp, g)
    assert_free_parity(gpu_rollout(dmx, m, inp), oracle_free(orc_mod, sc, inp))
    s = dict(inp, T=np.full(24, 0.05), NI=1, ctrl=inp["ctrl"][:, :1])
    assert_replay_parity(orc_mod, sc, s, gpu_rollout(dmx, m, s, tape=True, want_xb=True))


# ---------------------------------------------------------------- GPU invariants and edges
@pytest.mark.parametrize("form", ["step", "graph"])
def test_plain_forms_bitwise_equal_persistent(dmx, form):
    sc = W.box_scene()
    inp = _sub(W.box_push_inputs(4096), np.arange(37))
    m = dmx.Model(sc)
    a = gpu_rollout(dmx, m, inp, lanes=8)
    b = gpu_rollout(dmx, m, inp, lanes=8, form=form)
    np.testing.assert_array_equal(a["xT"], b["xT"])
    np.testing.assert_array_equal(a["nsteps"], b["nsteps"])


def test_environment_alone_equals_in_batch(dmx):
    """Per-environment step sizes (Fig. 14): an environment's result does not
    depend on the others (bitwise)."""
    sc, inp = W.box_scene(), W.box_push_inputs(4096)
    m = dmx.Model(sc)
    batch = gpu_rollout(dmx, m, _sub(inp, np.arange(64)), lanes=8)
    for e in (0, 17, 63):
        alone = gpu_rollout(dmx, m, _sub(inp, np.array([e])), lanes=8)
        np.testing.assert_array_equal(alone["xT"][0], batch["xT"][e])
        assert alone["nsteps"][0] == batch["nsteps"][e]


def test_status_codes_and_empty_batch(dmx):
    import torch
    sc, inp = W.ball_scene(), W.ball_inputs(4)
    m = dmx.Model(sc)
    x0 = inp["x0"].copy()
    x0[1, 2] = np.nan
    g = gpu_rollout(dmx, m, dict(inp, x0=x0))
    assert g["status"][1] == 3 and g["nsteps"][1] == 0
    assert np.all(g["status"][[0, 2, 3]] == 0)
    g = gpu_rollout(dmx, m, inp, max_steps=5)
    assert np.all(g["status"] == 1)
    out = dmx.rollout(m, torch.zeros((13, 0), dtype=torch.float64, device="cuda"),
                      torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert out["xT"].shape == (13, 0)


def test_host_buffer_call_equals_device_call(dmx):
    sc = W.box_scene()
    inp = _sub(W.box_push_inputs(4096), np.arange(50))
    m = dmx.Model(sc)
    d = gpu_rollout(dmx, m, inp, lanes=8)
    h = dmx.rollout_host(m, np.ascontiguousarray(inp["x0"].T), np.ascontiguousarray(inp["T"]), lanes=8)
    np.testing.assert_array_equal(h["xT"].T, d["xT"])


def test_model_inverse_weights_match_oracle(dmx, orc_mod):
    for name in ("ball", "box", "chain_cube", "quadruped", "billiard", "capsules"):
        sc = W.SCENES[name]()
        g = dmx.Model(sc).info()["invw"]
        o = orc_mod.OracleModel(sc)
        np.testing.assert_allclose(g, [o.body_invw(b) for b in range(o.nbody)], rtol=1e-12)


# ---------------------------------------------------------------- step-size control
def test_step_size_sequence_equals_oracle(dmx, orc_mod):
    """The GPU's controller against the oracle's pinned one: on the torque-free
    symmetric top (error norm a function of h alone, absolute tolerance only;
    tests/test_oracle_step_control.py) both take the same accepted step sizes,
    through the PID transient, the rejections (one retry, and two when the
    first retry is clipped at 0.2), the growth clip at 10 and the fixed point.
    From h0 = 1 us the first error norms are rounding noise (1e-14 .. 1e-9 of
    atol): there only the steps the floor and the clip fix exactly are
    compared."""
    sc = W.box_scene(gravity=(0.0, 0.0, 0.0))
    sc["bodies"][0]["inertia"] = [0.1, 0.1, 0.3]
    sc["pairs"] = []
    om = orc_mod.OracleModel(sc)
    gm = dmx.Model(sc)
    x0 = np.array([0, 0, 1.0, 1, 0, 0, 0, 0, 0, 0, 1.0, 0.5, 4.0])
    for h0 in (1e-6, 5e-3, 0.03, 0.1):
        inp = {"x0": x0[None, :], "ctrl": None, "T": np.array([1.0]), "NI": 1, "rtol": 0.0, "atol": 1e-8,
               "h0": h0, "max_steps": 20000}
        g = gpu_rollout(dmx, gm, inp, tape=True)
        o = om.rollout(x0, T=1.0, rtol=0.0, atol=1e-8, h0=h0)
        n = int(g["tape_n"][0])
        if h0 < 1e-4:   # (the kernel forms the factor as one exponential of logs: an ulp apart)
            np.testing.assert_allclose(g["hlog"][0, :3], o["hlog"][:3], rtol=1e-14)
            continue
        assert n == o["nsteps"] and g["nrej"][0] == o["nrej"]
        np.testing.assert_allclose(g["hlog"][0, :n], o["hlog"], rtol=1e-7)   # error norms of 1e-11 differences


# ---------------------------------------------------------------- other schemes (Fig. 12, Sec. 3.1)
@pytest.mark.parametrize("method", ["tsit5", "euler"])
def test_other_schemes_match_oracle(dmx, orc_mod, method):
    """Tsitouras 5(4) with the PID controller and fixed-step semi-implicit Euler
    (h0 = 1 ms): every accepted step against one oracle step of the same
    scheme and size, whole-trajectory replay, and free-running step sequences
    (balls: states and step counts; the fixed-step scheme takes exactly the
    same steps on both sides) on balls, box pushes and the arm."""
    sc, inp = W.ball_scene(), W.ball_inputs(16)
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp, tape=True, K=1, method=method)
    assert_stepwise_parity(orc_mod, sc, inp, g, method=method)
    assert_replay_parity(orc_mod, sc, inp, g, method=method)
    f = gpu_rollout(dmx, m, inp, method=method)
    o = oracle_free(orc_mod, sc, inp, method=method)
    assert_free_parity(f, o)
    if method == "euler":
        np.testing.assert_array_equal(f["nsteps"], o["nsteps"])
        assert np.all(f["nrej"] == 0)
    sc = W.box_scene()
    inp = _sub(W.box_push_inputs(4096), np.arange(40))
    m = dmx.Model(sc)
    for lanes in (4, 8):
        g = gpu_rollout(dmx, m, _short(inp, 0.1), tape=True, K=1, lanes=lanes, method=method)
        assert_stepwise_parity(orc_mod, sc, _short(inp, 0.1), g, method=method)
    s = _short(inp)
    assert_replay_parity(orc_mod, sc, s, gpu_rollout(dmx, m, s, tape=True, method=method), method=method)
    sc = W.chain_cube_scene()
    inp = W.chain_inputs(12, T=0.2, NI=5)
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp, tape=True, K=1, want_xb=True, method=method)
    assert_stepwise_parity(orc_mod, sc, inp, g, method=method)


def test_scheme_forms_bitwise_equal(dmx):
    """Every launch form runs the same scheme: persistent, per-attempt and
    graph-replayed forms give bitwise-equal Tsit5 and Euler results."""
    sc = W.box_scene()
    inp = _sub(W.box_push_inputs(4096), np.arange(29))
    m = dmx.Model(sc)
    for method in ("tsit5", "euler"):
        a = gpu_rollout(dmx, m, inp, lanes=8, method=method)
        for form in ("step", "graph"):
            b = gpu_rollout(dmx, m, inp, lanes=8, form=form, method=method)
            np.testing.assert_array_equal(a["xT"], b["xT"])
            np.testing.assert_array_equal(a["nsteps"], b["nsteps"])


# ---------------------------------------------------------------- sphere / capsule pairs (Sec. 4 billiard)
def pair_states(orc_mod, name, B, seed):
    """States of seeded billiard / capsule throws at which some pair is within
    3 mm (approaching, in contact or separating), from the oracle's own
    trajectories, jittered by 1e-4."""
    sc = W.SCENES[name]()
    om = orc_mod.OracleModel(sc)
    inp = W.INPUTS[name](64, seed=seed)
    g = np.random.default_rng(seed)
    Q, V = [], []
    for x0 in inp["x0"]:
        r = om.rollout(x0, T=float(inp["T"][0]), NI=80)
        for xb in r["xb"]:
            if om.contacts(xb[:om.nq])[:, 0].min() < 3e-3:
                Q.append(xb[:om.nq] + 1e-4 * g.normal(size=om.nq))
                V.append(xb[om.nq:] + 1e-4 * g.normal(size=om.nv))
        if len(Q) >= B:
            break
    q = np.array(Q[:B])
    for k in range(len(sc["bodies"])):
        q[:, 7 * k + 3:7 * k + 7] /= np.linalg.norm(q[:, 7 * k + 3:7 * k + 7], axis=1, keepdims=True)
    return sc, q, np.array(V[:B])


@pytest.mark.parametrize("cfd", [False, True])
@pytest.mark.parametrize("name", ["billiard", "capsules"])
def test_pair_rhs_matches_oracle(dmx, orc_mod, name, cfd):
    sc, q, v = pair_states(orc_mod, name, 64, 21)
    if cfd:
        sc = W.SCENES[name](**CFD_OPT)
    om = orc_mod.OracleModel(sc)
    ref = np.array([om.rhs(q[e], v[e], cfd=cfd) for e in range(len(q))])
    det = [om.rhs(q[e], v[e], cfd=cfd, detail=True)[1] for e in range(len(q))]
    nrows = np.array([d["nr"] for d in det])
    pushed = np.array([d["nr"] > 0 and d["f"].max() > 0 for d in det])
    assert pushed.sum() >= 8
    gm = dmx.Model(sc)
    for lanes in (4, 8, 32):
        a, info = dmx.eval_rhs(gm, _dev(q.T), _dev(v.T), cfd=cfd, lanes=lanes)
        a, info = a.cpu().numpy().T, info.cpu().numpy()
        assert np.all(info[0] == 0)
        np.testing.assert_array_equal(info[1], nrows)
        # zero gravity: a contact-free state's right-hand side is the
        # gyroscopic term alone (exactly zero for the balls), which both sides
        # compute as rounding residue of the cancelling spatial-velocity terms
        # (1e-14 rad/s^2 at 1 m/s); errors are measured against >= 1 m/s^2
        scale = np.maximum(np.maximum(np.abs(ref), np.abs(ref).max(axis=1, keepdims=True)), 1.0)
        err = float((np.abs(a - ref) / scale).max())
        assert err < TOL_RHS, f"lanes {lanes}: {err:.3e}"
        err_c = max(rel_err(a[e], ref[e]) for e in np.nonzero(pushed)[0])
        assert err_c < TOL_RHS, f"lanes {lanes}, states with contact force: {err_c:.3e}"


# Positions and linear velocities of the two balls.  The frictionless balls'
# orientations and spins are physically inert (exactly identity and zero);
# computed, they are rounding residue.  In the shots where one 0.37 s step
# carries the cue ball through the target, only the second stage sees the
# contact (2.8e3 m/s^2); its weights in the solution and in the error
# estimate are zero, so the hit cancels (both sides tunnel), but its kick
# puts the later stage states hundreds of metres from the origin, where the
# cancelling spatial-velocity terms leave 1e-7 rad/s^2 of spin residue that
# differs with the summation order (Sec. 4 and App. C.4 discuss the adaptive
# solver seeing an interaction only at its stage states).
BILLIARD_TRANS = [0, 1, 2, 7, 8, 9, 14, 15, 16, 20, 21, 22]


@pytest.mark.parametrize("name", ["billiard", "capsules"])
def test_pair_trajectories_match_oracle(dmx, orc_mod, name):
    """Billiard shots (head-on to glancing, some misses) and capsule throws:
    every accepted step, the whole replayed trajectory, and free-running final
    states of the non-chaotic billiard."""
    sc, inp = W.SCENES[name](), W.INPUTS[name](16)
    m = dmx.Model(sc)
    g = gpu_rollout(dmx, m, inp, tape=True, K=1)
    assert np.all(g["status"] == 0)
    comps = BILLIARD_TRANS if name == "billiard" else None
    if name == "billiard":
        # the error norm of a tunnelling step carries the spin residue too
        # (above atol, order-dependent), so its acceptance is checked on the
        # shots that hit (dozens of steps; a tunnelling shot takes 5 or 6)
        hit = [e for e in range(len(inp["x0"])) if g["tape_n"][e] >= 15]
        tun = [e for e in range(len(inp["x0"])) if g["tape_n"][e] < 15]
        assert len(hit) >= 8 and len(tun) >= 2
        assert_stepwise_parity(orc_mod, sc, inp, g, envs=hit, comps=comps)
        assert_stepwise_parity(orc_mod, sc, inp, g, envs=tun, comps=comps, check_valid=False)
    else:
        assert_stepwise_parity(orc_mod, sc, inp, g)
    assert_replay_parity(orc_mod, sc, inp, gpu_rollout(dmx, m, inp, tape=True), comps=comps)
    if name == "billiard":
        # free running, the spin residue enters every error norm: the step
        # sequences part (a few steps in 50) while the balls' motion agrees
        assert_free_parity(gpu_rollout(dmx, m, inp), oracle_free(orc_mod, sc, inp), comps=comps, ratio_tol=0.25)
