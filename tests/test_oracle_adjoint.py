"""Pins of the oracle's discrete adjoint (discretize-then-optimize over the
accepted steps) and of the straight-through CFD gradient: closed forms,
frozen-step central differences, and the properties the paper states for the
straight-through estimator (Sec. 4, App. C.4)."""

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W
from tests.conftest import rel_err

CFD_OPT = dict(W.CFD_OPTIONS)


def test_ballistic_gradient_closed_form(orc):
    m = orc.OracleModel(W.ball_scene())
    x0 = np.array([0.1, -0.2, 2.0, 1, 0, 0, 0, 0.7, -0.4, 1.5, 0, 0, 0])
    T = 0.4
    xbar = np.zeros(13); xbar[2] = 1.0                     # L = z_T
    g = m.rollout_grad(x0, xbar, T=T)["x0_bar"]
    ref = np.zeros(13); ref[2] = 1.0; ref[9] = T
    np.testing.assert_allclose(g, ref, atol=1e-13)
    xbar = np.zeros(13); xbar[0] = 1.0; xbar[7] = 2.0      # L = x_T + 2 vx_T
    g = m.rollout_grad(x0, xbar, T=T)["x0_bar"]
    ref = np.zeros(13); ref[0] = 1.0; ref[7] = T + 2.0
    np.testing.assert_allclose(g, ref, atol=1e-13)


def _frozen_fd(m, x0, hlog, wT, ctrl=None, T=1.0, NI=1, eps=1e-6, wb=None, method="dopri5"):
    """Central differences of <wT, xT> (+ sum_k <wb_k, x(t_k)>) of the replayed
    (frozen-step) discrete map w.r.t. x0 and the controls."""
    def L(x, c):
        xT, xb = m.replay(x, hlog, ctrl=c, T=T, NI=NI, method=method)
        val = wT @ xT
        if wb is not None:
            val += (wb * xb).sum()
        return val
    gx = np.zeros(m.nx)
    for i in range(m.nx):
        e = np.zeros(m.nx); e[i] = eps
        gx[i] = (L(x0 + e, ctrl) - L(x0 - e, ctrl)) / (2 * eps)
    gu = None
    if ctrl is not None and m.nu:
        gu = np.zeros_like(ctrl)
        for idx in np.ndindex(ctrl.shape):
            e = np.zeros_like(ctrl); e[idx] = eps
            gu[idx] = (L(x0, ctrl + e) - L(x0, ctrl - e)) / (2 * eps)
    return gx, gu


def test_step_jacobian_matches_differences(orc):
    m = orc.OracleModel(W.box_scene())
    x0 = W.box_push_inputs(1, seed=5)["x0"][0]
    r = m.rollout(x0, T=0.02)
    q, v = r["xT"][:7], r["xT"][7:]
    h = 1e-3
    Jx, _ = m.step_jacobian(q, v, None, h)
    eps = 1e-7
    for i in range(13):
        e = np.zeros(13); e[i] = eps
        xp, _ = m.replay(r["xT"] + e, [h], T=h)
        xm, _ = m.replay(r["xT"] - e, [h], T=h)
        np.testing.assert_allclose(Jx[:, i], (xp - xm) / (2 * eps), atol=1e-6)


@pytest.mark.parametrize("seed", range(3))
def test_ball_bounce_gradient_frozen_steps(orc, seed):
    m = orc.OracleModel(W.ball_scene())
    x0 = W.ball_inputs(3, seed=seed)["x0"][seed]
    r = m.rollout(x0, T=1.0)
    w = np.zeros(13); w[2] = 1.0; w[7] = 0.3; w[9] = -0.5
    g = m.rollout_grad(x0, w, T=1.0)
    np.testing.assert_array_equal(g["xT"], r["xT"])
    assert _best_fd_err(m, x0, r["hlog"], w, g) < 1e-5


def _best_fd_err(m, x0, hlog, w, g, **kw):
    """Stiff contact makes the frozen-step map strongly curved: central
    differences converge to the derivative as eps shrinks, so take the best
    of a small eps sweep (truncation vs round-off)."""
    errs = []
    for eps in (1e-6, 1e-7, 1e-8):
        fdx, fdu = _frozen_fd(m, x0, hlog, w, eps=eps, **kw)
        e = rel_err(g["x0_bar"], fdx)
        if fdu is not None:
            e = max(e, rel_err(g["ctrl_bar"].ravel(), fdu.ravel()))
        errs.append(e)
    return min(errs)


@pytest.mark.parametrize("T", [0.01, 0.1])
def test_box_gradient_frozen_steps(orc, T):
    """Box launched by a push at its base (tumbling, sliding and landing on
    corners): adjoint vs central differences of the replayed map."""
    m = orc.OracleModel(W.box_scene())
    x0 = np.array([0, 0, 0.0497, 1, 0, 0, 0, 2.0, 0.5, 0, 0, 0, 0.0])
    x1 = m.rollout(x0, T=0.02)["xT"]
    r = m.rollout(x1, T=T)
    w = np.random.default_rng(1).normal(size=13)
    g = m.rollout_grad(x1, w, T=T)
    assert _best_fd_err(m, x1, r["hlog"], w, g, T=T) < 1e-5


def test_chain_control_gradient_frozen_steps(orc):
    """Chain + cube, piecewise-constant torques: gradient w.r.t. x0 and every
    control of every interval, with interval-boundary cotangents."""
    sc = W.chain_cube_scene()
    m = orc.OracleModel(sc)
    inp = W.chain_inputs(1, T=0.3, NI=6)
    x0, ctrl = inp["x0"][0], inp["ctrl"][0]
    r = m.rollout(x0, ctrl=ctrl, T=0.3, NI=6)
    g_ = np.random.default_rng(2)
    w = g_.normal(size=m.nx)
    wb = g_.normal(size=(7, m.nx))
    g = m.rollout_grad(x0, w, ctrl=ctrl, T=0.3, NI=6, xb_bar=wb)
    # the cube starts resting on the plane, where pyramid rows sit at the edge of
    # the active set (kinks of the map): compare the arm's state and the controls
    arm = list(range(7)) + list(range(14, 21))
    best = []
    for eps in (1e-6, 1e-7):
        fdx, fdu = _frozen_fd(m, x0, r["hlog"], w, ctrl=ctrl, T=0.3, NI=6, wb=wb, eps=eps)
        best.append(max(rel_err(g["x0_bar"][arm], fdx[arm]), rel_err(g["ctrl_bar"].ravel(), fdu.ravel())))
    assert min(best) < 1e-5


def test_quadruped_gradient_frozen_steps(orc):
    sc = W.quadruped_scene()
    m = orc.OracleModel(sc)
    inp = W.quadruped_inputs(1)
    x0, ctrl = inp["x0"][0], inp["ctrl"][0]
    T = 0.25
    r = m.rollout(x0, ctrl=ctrl, T=T)
    w = np.zeros(m.nx); w[0:3] = [1.0, 0.5, -0.7]
    g = m.rollout_grad(x0, w, ctrl=ctrl, T=T)
    assert _best_fd_err(m, x0, r["hlog"], w, g, ctrl=ctrl, T=T) < 1e-5


def test_gradient_converges_with_tolerance(orc):
    """Adaptive integration drives the discrete gradient towards the gradient of
    the continuous flow as the tolerance shrinks (Sec. 3.1, Fig. 5): for a ball
    in the middle of its impact, the error against a 1e-12 reference falls by
    more than an order of magnitude from rtol 1e-6 to 1e-10."""
    m = orc.OracleModel(W.ball_scene())
    x0 = np.array([0, 0, 0.6, 1, 0, 0, 0, 0.3, 0, -0.5, 0, 0, 0.0])
    w = np.zeros(13); w[2] = 1.0; w[9] = 0.1
    g = {rt: m.rollout_grad(x0, w, T=0.33, rtol=rt, atol=rt * 1e-2)["x0_bar"] for rt in (1e-6, 1e-10, 1e-12)}
    e6, e10 = rel_err(g[1e-6], g[1e-12]), rel_err(g[1e-10], g[1e-12])
    assert e10 < 0.05 and e10 < e6 / 10


# ---------------------------------------------------------------- straight-through CFD
def test_cfd_does_not_change_the_forward_pass(orc):
    m = orc.OracleModel(W.box_scene(**CFD_OPT))
    x0 = W.box_push_inputs(2, seed=3)["x0"][0]
    w = np.ones(13)
    a = m.rollout_grad(x0, w, T=0.3, cfd=False)
    b = m.rollout_grad(x0, w, T=0.3, cfd=True)
    np.testing.assert_array_equal(a["xT"], b["xT"])
    assert np.abs(a["x0_bar"] - b["x0_bar"]).max() > 1e-6


def test_cfd_gradient_equals_plain_gradient_without_near_contacts(orc):
    m = orc.OracleModel(W.ball_scene(**CFD_OPT))
    x0 = np.array([0, 0, 3.0, 1, 0, 0, 0, 0.3, 0.2, 1.0, 0, 0, 0])   # stays above w_c
    w = np.zeros(13); w[2] = 1.0; w[0] = 0.5
    a = m.rollout_grad(x0, w, T=0.4, cfd=False)["x0_bar"]
    b = m.rollout_grad(x0, w, T=0.4, cfd=True)["x0_bar"]
    np.testing.assert_array_equal(a, b)


def test_cfd_gives_informative_gradient_before_contact(orc):
    """A ball gliding just above the plane (no gravity) never touches it: the
    plain gradient of its final height w.r.t. its initial height is exactly 1,
    the CFD gradient sees the plane within w_c (Sec. 4, billiard example)."""
    m = orc.OracleModel(W.ball_scene(gravity=(0.0, 0.0, 0.0), **CFD_OPT))
    x0 = np.array([0, 0, 0.12, 1, 0, 0, 0, 1.0, 0, 0, 0, 0, 0])
    w = np.zeros(13); w[2] = 1.0
    plain = m.rollout_grad(x0, w, T=0.5, cfd=False)
    cfd = m.rollout_grad(x0, w, T=0.5, cfd=True)
    assert abs(plain["x0_bar"][2] - 1.0) < 1e-14 and abs(plain["x0_bar"][9] - 0.5) < 1e-14
    np.testing.assert_array_equal(plain["xT"], cfd["xT"])
    # the CFD rows (damping term of a_ref, d(r) > 0 within w_c) react to the
    # normal velocity: dz_T/dvz_0 departs from the free-flight value T
    assert abs(cfd["x0_bar"][9] - 0.5) > 1e-2
    assert np.all(np.isfinite(cfd["x0_bar"]))


def test_cfd_step_jacobian_uses_cfd_rhs_at_the_plain_states(orc):
    """With cfd, the derivative of one step is the derivative of the DOPRI5
    step built from F~, but evaluated at the stage states of F (compare the
    one-stage case h -> small: J ~ I + h [0 I; dF~/dq dF~/dv])."""
    sc = W.ball_scene(gravity=(0.0, 0.0, 0.0), **CFD_OPT)
    m = orc.OracleModel(sc)
    q = np.array([0, 0, 0.12, 1, 0, 0, 0]); v = np.array([1.0, 0, -0.1, 0, 0, 0])
    h = 1e-7
    Jx, _ = m.step_jacobian(q, v, None, h, cfd=True)
    Jq, Jv, _ = m.rhs_jacobian(q, v, None, cfd=True)
    np.testing.assert_allclose((Jx[7:, :7]) / h, Jq, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose((Jx[7:, 7:] - np.eye(6)) / h, Jv, rtol=1e-5, atol=1e-6)


def _replay_grads(m, inp, xT_bar, x0):
    B = len(x0)
    H, N = [], []
    for e in range(B):
        r = m.rollout(inp["x0"][e], T=float(inp["T"][e]), rtol=inp["rtol"], atol=inp["atol"], h0=inp["h0"],
                      max_steps=inp["max_steps"])
        H.append(r["hlog"]); N.append(r["nsteps"])
    hl = np.zeros((B, max(N)))
    for e in range(B):
        hl[e, :N[e]] = H[e]
    return m.batch_replay_grad(x0, inp["T"], hl, N, xT_bar)["x0_bar"]


def test_gradient_conditioning_floor(orc):
    """How far rounding alone can move the frozen-step gradient of box pushes:
    the x0 gradient at x0 and at x0 (1 + 1e-16 noise), along the same step
    sizes.  Over 0.1 s the change stays far below the 1e-6 gradient bar; over
    0.3 s it reaches that bar (products of a few hundred Jacobians of the
    stiff sliding-contact map), which is why the GPU gradient tests of box
    pushes integrate 0.1 s."""
    m = orc.OracleModel(W.box_scene())
    floors = {}
    for T in (0.1, 0.3):
        inp = W.box_push_inputs(24, seed=5, T=T)
        w = np.random.default_rng(1).normal(size=(24, 13))
        g0 = _replay_grads(m, inp, w, inp["x0"])
        worst = 0.0
        for trial in range(3):
            x1 = inp["x0"] * (1 + 1e-16 * np.random.default_rng(trial).normal(size=inp["x0"].shape))
            g1 = _replay_grads(m, inp, w, x1)
            worst = max(worst, max(rel_err(g1[e], g0[e]) for e in range(24)))
        floors[T] = worst
    assert floors[0.1] < 1e-8, floors
    assert floors[0.3] > 1e-7, floors


def test_arm_gradient_conditioning_floor_at_full_horizon(orc):
    """The same question for the arm pushing the cube over its full 2 s
    horizon (50 torque intervals, as timed by the benchmark): the control and
    x0 gradients of the squared cube-to-goal distance plus a random cotangent
    on the final coordinates, at x0 and at x0 moved by 1e-15 (relative and
    absolute), along the same step sizes, move by less than 1e-7.  So the
    1e-6 gradient bar can be checked at the full horizon."""
    sc = W.chain_cube_scene()
    m = orc.OracleModel(sc)
    inp = W.chain_inputs(16384)
    idx = np.array([0, 5])                       # the arm reaches the cube in both
    x0, ctrl, T = inp["x0"][idx], inp["ctrl"][idx], inp["T"][idx]
    H, N, xT = [], [], []
    for e in range(len(idx)):
        r = m.rollout(x0[e], ctrl=ctrl[e], T=float(T[e]), NI=50)
        assert r["status"] == 0
        H.append(r["hlog"]); N.append(r["nsteps"]); xT.append(r["xT"])
    hl = np.zeros((len(idx), max(N)))
    for e in range(len(idx)):
        hl[e, :N[e]] = H[e]
    xT_bar = 0.1 * np.random.default_rng(9).normal(size=(len(idx), m.nx))
    xT_bar[:, 7:10] += 2 * (np.array(xT)[:, 7:10] - W.chain_goal())
    g0 = m.batch_replay_grad(x0, T, hl, N, xT_bar, ctrl=ctrl, NI=50)
    assert np.abs(g0["ctrl_bar"]).max() > 0
    rng = np.random.default_rng(10)
    x1 = x0 * (1 + 1e-15 * rng.normal(size=x0.shape)) + 1e-15 * rng.normal(size=x0.shape)
    g1 = m.batch_replay_grad(x1, T, hl, N, xT_bar, ctrl=ctrl, NI=50)
    floor = max(max(rel_err(g1["ctrl_bar"][e].ravel(), g0["ctrl_bar"][e].ravel()),
                    rel_err(g1["x0_bar"][e], g0["x0_bar"][e])) for e in range(len(idx)))
    assert 0 < floor < 1e-7, floor


@pytest.mark.parametrize("method", ["tsit5", "euler"])
def test_other_schemes_gradient_frozen_steps(orc, method):
    """The discrete adjoint of the Tsitouras scheme and of fixed-step
    semi-implicit Euler (h = 1 ms): ball bounce and arm controls against
    central differences of the replayed map."""
    m = orc.OracleModel(W.ball_scene())
    x0 = W.ball_inputs(3, seed=1)["x0"][1]
    r = m.rollout(x0, T=1.0, method=method)
    assert r["status"] == 0
    w = np.zeros(13); w[2] = 1.0; w[7] = 0.3; w[9] = -0.5
    g = m.rollout_grad(x0, w, T=1.0, method=method)
    np.testing.assert_array_equal(g["xT"], r["xT"])
    assert _best_fd_err(m, x0, r["hlog"], w, g, method=method) < 1e-5
    sc = W.chain_cube_scene()
    m = orc.OracleModel(sc)
    inp = W.chain_inputs(1, T=0.2, NI=4)
    x0, ctrl = inp["x0"][0], inp["ctrl"][0]
    r = m.rollout(x0, ctrl=ctrl, T=0.2, NI=4, method=method)
    w = np.random.default_rng(2).normal(size=m.nx)
    g = m.rollout_grad(x0, w, ctrl=ctrl, T=0.2, NI=4, method=method)
    arm = list(range(7)) + list(range(14, 21))
    best = []
    for eps in (1e-6, 1e-7):
        fdx, fdu = _frozen_fd(m, x0, r["hlog"], w, ctrl=ctrl, T=0.2, NI=4, eps=eps, method=method)
        best.append(max(rel_err(g["x0_bar"][arm], fdx[arm]), rel_err(g["ctrl_bar"].ravel(), fdu.ravel())))
    assert min(best) < 1e-5


# ------------------------------------------------------------------ model-parameter gradients (Sec. 5.1, App. E.2)
PARAM_NAMES = ["t_c", "phi_d", "d_o", "d_w", "width", "midpoint"]


def _boxes(sc):
    return [g for g, gm in enumerate(sc["geoms"]) if gm["type"] == "box"]


def _perturbed_scene(make, k, delta):
    """Scene from make() with model parameter k moved by delta (order:
    t_c, phi_d, d_o, d_w, width, midpoint, mu of each pair, the mass of each
    body with its inertia scaled in proportion, then the side length (2 x the
    x half size) of each box geom: half sizes scaled together, and the
    inertia of a body whose only geom is the box by the square)."""
    sc = make()
    o = sc["options"]
    npair, nbody = len(sc["pairs"]), len(sc["bodies"])
    if k < 2:
        o["solref"][k] += delta
    elif k < 6:
        o["solimp"][k - 2] += delta
    elif k < 6 + npair:
        sc["pairs"][k - 6]["mu"] += delta
    elif k < 6 + npair + nbody:
        b = sc["bodies"][k - 6 - npair]
        f = (b["mass"] + delta) / b["mass"]
        b["mass"] += delta
        b["inertia"] = [f * x for x in b["inertia"]]
    else:
        g = _boxes(sc)[k - 6 - npair - nbody]
        gm = sc["geoms"][g]
        lam = (2 * gm["size"][0] + delta) / (2 * gm["size"][0])
        gm["size"] = [lam * x for x in gm["size"]]
        if sum(1 for q in sc["geoms"] if q["body"] == gm["body"]) == 1:
            b = sc["bodies"][gm["body"]]
            b["inertia"] = [lam * lam * x for x in b["inertia"]]
    return sc


def _param_value(sc, k):
    o = sc["options"]
    npair, nbody = len(sc["pairs"]), len(sc["bodies"])
    if k < 2:
        return o["solref"][k]
    if k < 6:
        return o["solimp"][k - 2]
    if k < 6 + npair:
        return sc["pairs"][k - 6]["mu"]
    if k < 6 + npair + nbody:
        return sc["bodies"][k - 6 - npair]["mass"]
    return 2 * sc["geoms"][_boxes(sc)[k - 6 - npair - nbody]]["size"][0]


def _param_fd(orc, make, x0, hlog, w, T, k, rel=1e-6, ctrl=None, NI=1):
    """Central difference of <w, xT> of the frozen-step map (the given step
    sizes replayed) w.r.t. model parameter k."""
    eps = rel * max(abs(_param_value(make(), k)), 1e-3)
    vals = []
    for sgn in (1.0, -1.0):
        m = orc.OracleModel(_perturbed_scene(make, k, sgn * eps))
        xT, _ = m.replay(x0, hlog, ctrl=ctrl, T=T, NI=NI)
        vals.append(w @ xT)
    return (vals[0] - vals[1]) / (2 * eps)


@pytest.mark.parametrize("name", ["ball", "box"])
def test_parameter_gradient_frozen_steps(orc, name):
    """p_bar of the discrete adjoint (solref, solimp, friction, mass, box side)
    against central differences of the frozen-step map over models with one
    parameter moved."""
    make = W.SCENES[name]
    m = orc.OracleModel(make())
    if name == "ball":
        x0, T = W.ball_inputs(3, seed=2)["x0"][2], 1.0
    else:
        x0, T = np.array([0, 0, 0.0497, 1, 0, 0, 0, 1.2, 0.4, 0, 0, 0, 0.0]), 0.15
    r = m.rollout(x0, T=T)
    w = np.random.default_rng(4).normal(size=13)
    n = np.array([len(r["hlog"])], dtype=np.int32)
    g = m.batch_replay_grad(x0[None], np.array([T]), r["hlog"][None], n, w[None], params=True)
    pb = g["p_bar"][0]
    assert len(pb) == m.nparams() == 8 + (name == "box")
    for k in range(m.nparams()):
        if name == "ball" and k == 6:
            assert pb[k] == 0.0                      # frictionless: mu enters no row
            continue
        # stiff contact curves the frozen-step map: best of a small eps sweep
        # (truncation vs round-off), as for the state gradients
        errs = []
        for rel in (1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9):
            fd = _param_fd(orc, make, x0, r["hlog"], w, T, k, rel=rel)
            errs.append(abs(pb[k] - fd) / max(abs(fd), np.abs(pb).max() * 1e-2))
        assert min(errs) < 2e-5, (k, pb[k], errs)


def test_rest_height_parameter_gradient(orc):
    """A ball settled on the plane sits at R + r_rest(theta), where r_rest is
    the root of k d(r)^2 (-r) = g (1 - d(r)) (a = 0, J v = 0; k = 1/(d_w^2 t_c^2
    phi_d^2), d the solimp spline): the adjoint's gradient of the final height
    w.r.t. (t_c, phi_d, d_o, d_w, width, midpoint) equals d r_rest / d theta,
    computed here from that scalar equation alone (brentq roots of perturbed
    equations).  The mass drops out: the contact force m g equals
    (a_ref + g) / (R + 1/m) with R = A_hat (1 - d) / d, and the ball's A_hat is
    1/m, so a_ref = g (1 - d) / d whatever m; the mass gradient vanishes only
    if both the inertia's and A_hat's dependence on the mass are carried
    (either alone gives a non-zero gradient, the two of opposite sign).  The adaptive
    steps at rest leave velocities of ~1e-9 m/s, so the comparison holds to
    1e-3 relative (a missing term or a sign is O(1))."""
    from scipy.optimize import brentq
    sc = W.ball_scene()
    m0 = sc["bodies"][0]["mass"]
    base = [*sc["options"]["solref"], *sc["options"]["solimp"][:4]]
    pw = sc["options"]["solimp"][4]

    def spline(x, mid):
        return x ** pw / mid ** (pw - 1) if x <= mid else 1 - (1 - x) ** pw / (1 - mid) ** (pw - 1)

    def r_rest(th):
        tc, ph, do, dw, wd, mid = th
        k = 1.0 / (dw ** 2 * tc ** 2 * ph ** 2)
        d = lambda r: min(max(do + (dw - do) * spline(min(abs(r) / wd, 1.0), mid), 0.0), 0.9999)
        return brentq(lambda r: k * d(r) ** 2 * (-r) - 9.81 * (1 - d(r)), -0.0009, -1e-6, xtol=1e-18, rtol=1e-15)

    m = orc.OracleModel(sc)
    x0 = np.array([0, 0, 0.3, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0])
    T = 2.0
    r = m.rollout(x0, T=T)
    w = np.zeros(13); w[2] = 1.0
    n = np.array([len(r["hlog"])], dtype=np.int32)
    pb = m.batch_replay_grad(x0[None], np.array([T]), r["hlog"][None], n, w[None], params=True)["p_bar"][0]
    # parameter order: the six contact parameters, mu of the pair, the mass
    assert pb[6] == 0.0                                 # frictionless pair
    for k in range(6):
        eps = 1e-6 * max(abs(base[k]), 1e-3)
        hi, lo = list(base), list(base)
        hi[k] += eps; lo[k] -= eps
        ref = (r_rest(hi) - r_rest(lo)) / (2 * eps)
        assert abs(pb[k] - ref) <= 1e-3 * abs(ref), (PARAM_NAMES[k], pb[k], ref)
    # relative sensitivities theta dz/dtheta: the mass's vanishes
    rel = np.abs(pb[:6] * np.array(base))
    assert abs(pb[7] * m0) <= 1e-3 * rel.max(), (pb[7], rel)


def test_cube_rest_height_side_gradient(orc):
    """A cube settled flat on the plane rests at z = l/2 + r_rest: the
    penetration r_rest solves the same per-vertex equilibrium whatever the
    side l (the vertices move horizontally with it, and the inverse weight of
    the free body is 1/m, independent of its inertia), so dz/dl = 1/2; and,
    as for the ball, the mass leaves z unchanged.  Pins the side length's
    path through the vertex positions and the inertia scaling."""
    sc = W.box_scene()
    m = orc.OracleModel(sc)
    x0 = np.array([0, 0, 0.06, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0.0])
    T = 1.0
    r = m.rollout(x0, T=T)
    w = np.zeros(13); w[2] = 1.0
    n = np.array([len(r["hlog"])], dtype=np.int32)
    pb = m.batch_replay_grad(x0[None], np.array([T]), r["hlog"][None], n, w[None], params=True)["p_bar"][0]
    assert len(pb) == 9                                  # 6 contact, mu, mass, side
    assert abs(pb[8] - 0.5) < 1e-9, pb[8]
    assert abs(pb[7] * sc["bodies"][0]["mass"]) < 1e-12, pb[7]


def test_capsule_box_side_gradient(orc):
    """The side length through the capsule-box distance: the arm's last link
    pressed 0.5 mm into a vertical edge of the yawed cube (zero gravity, so
    that contact alone acts), loss on the whole state after 10 ms; p_bar of
    the side against central differences of the frozen-step map over models
    with the box scaled (the implicit-function derivative of the minimiser
    along the link and the distance field both carry the box size)."""
    make = lambda: W.chain_cube_scene(gravity=(0.0, 0.0, 0.0))
    m = orc.OracleModel(make())
    k = m.nparams() - 1                                   # the cube's side
    yaw = 0.4
    x0 = np.zeros(27)
    x0[7:10] = [1.95, 0.09, 0.06]
    x0[10:14] = [np.cos(yaw / 2), 0, 0, np.sin(yaw / 2)]
    assert -1e-3 < m.contacts(x0[:14])[14, 0] < 0            # the last link's capsule-box slot
    ctrl = np.zeros((1, 7))
    T = 0.01
    r = m.rollout(x0, ctrl=ctrl, T=T, NI=1)
    w = np.random.default_rng(3).normal(size=27)
    n = np.array([r["nsteps"]], dtype=np.int32)
    pb = m.batch_replay_grad(x0[None], np.array([T]), r["hlog"][None], n, w[None], ctrl=ctrl[None], NI=1,
                             params=True)["p_bar"][0]
    errs = []
    for rel in (1e-6, 1e-7, 1e-8):
        fd = _param_fd(orc, make, x0, r["hlog"][:r["nsteps"]], w, T, k, rel=rel, ctrl=ctrl, NI=1)
        errs.append(abs(pb[k] - fd) / abs(fd))
    assert min(errs) < 1e-7, (pb[k], errs)


def _param_floor(orc, name, inp):
    """Largest change of the parameter gradient when x0 moves by 1e-15
    (relative and absolute), along the same step sizes."""
    m = orc.OracleModel(W.SCENES[name]())
    B = len(inp["x0"])
    H, N = [], []
    for e in range(B):
        r = m.rollout(inp["x0"][e], ctrl=None if inp["ctrl"] is None else inp["ctrl"][e], T=float(inp["T"][e]),
                      NI=inp["NI"])
        H.append(r["hlog"]); N.append(r["nsteps"])
    hl = np.zeros((B, max(N)))
    for e in range(B):
        hl[e, :N[e]] = H[e]
    w = np.random.default_rng(17).normal(size=(B, m.nx))
    n = np.array(N, dtype=np.int32)
    g0 = m.batch_replay_grad(inp["x0"], inp["T"], hl, n, w, ctrl=inp["ctrl"], NI=inp["NI"], params=True)
    rng = np.random.default_rng(3)
    x1 = inp["x0"] * (1 + 1e-15 * rng.normal(size=inp["x0"].shape)) + 1e-15 * rng.normal(size=inp["x0"].shape)
    g1 = m.batch_replay_grad(x1, inp["T"], hl, n, w, ctrl=inp["ctrl"], NI=inp["NI"], params=True)
    return max(rel_err(g1["p_bar"][e], g0["p_bar"][e]) for e in range(B))


def test_parameter_gradient_conditioning_floor(orc):
    """Where the contact-parameter gradient is defined to rounding: with the
    arm's cube dropped onto the plane, the quadruped (0.3 s) and tumbling
    boxes, 1e-15 perturbations of x0 move p_bar by less than 1e-8; with the
    cube resting on the plane or boxes sliding flat on a face (friction rows
    of coplanar contacts at the edge of the active set) they move it by more
    than 1e-4, so the GPU parameter-gradient tests use the former inputs."""
    from tests.test_gpu_adjoint import param_inputs
    for name in ("chain_cube", "quadruped", "box"):
        assert _param_floor(orc, name, param_inputs(name)) < 1e-8, name
    rest = W.chain_inputs(6, T=0.2, NI=4)
    slow = W.box_push_inputs(12, seed=5, T=0.1)
    assert max(_param_floor(orc, "chain_cube", rest), _param_floor(orc, "box", slow)) > 1e-4
