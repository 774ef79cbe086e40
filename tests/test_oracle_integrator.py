"""Pins of the oracle's adaptive DOPRI5 rollout against closed-form motions
(ballistic flight, torque-free symmetric top, damped hinge), its convergence
order, the stiff-contact rest height, conservation laws of a frictionless
bounce, Coulomb-like sliding friction, and its status codes."""

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2506_14186_gb300 import workloads as W


def test_ballistic_flight_is_exact(orc):
    """No contact: the motion is quadratic in t, which DOPRI5 integrates exactly."""
    m = orc.OracleModel(W.ball_scene())
    x0 = np.array([0.1, -0.2, 2.0, 1, 0, 0, 0, 0.7, -0.4, 1.5, 0, 0, 0])
    T = 0.5
    r = m.rollout(x0, T=T)
    assert r["status"] == 0
    np.testing.assert_allclose(r["xT"][:3], [0.1 + 0.7 * T, -0.2 - 0.4 * T, 2.0 + 1.5 * T - 0.5 * 9.81 * T * T], atol=1e-14)
    np.testing.assert_allclose(r["xT"][7:10], [0.7, -0.4, 1.5 - 9.81 * T], atol=1e-14)


def _top_scene(I1=0.1, I3=0.3):
    sc = W.box_scene(gravity=(0.0, 0.0, 0.0))
    sc["bodies"][0]["inertia"] = [I1, I1, I3]
    sc["pairs"] = []
    return sc


def _top_exact(w0, t, I1=0.1, I3=0.3):
    lam = (I3 - I1) / I1 * w0[2]
    c, s = np.cos(lam * t), np.sin(lam * t)
    return np.array([w0[0] * c - w0[1] * s, w0[0] * s + w0[1] * c, w0[2]])


def test_torque_free_symmetric_top(orc):
    """Body-frame angular velocity of a free symmetric top precesses at
    (I3 - I1)/I1 w3 (Euler's equations; closed form)."""
    m = orc.OracleModel(_top_scene())
    w0 = np.array([1.0, 0.5, 4.0])
    x0 = np.concatenate([[0, 0, 1.0, 1, 0, 0, 0, 0, 0, 0], w0])
    r = m.rollout(x0, T=1.0, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(r["xT"][10:13], _top_exact(w0, 1.0), atol=1e-9)


def test_fifth_order_convergence(orc):
    """Fixed steps (replay of a constant step list): the global error of the
    angular velocity falls by ~2^5 per halving of h."""
    m = orc.OracleModel(_top_scene())
    w0 = np.array([1.0, 0.5, 4.0])
    x0 = np.concatenate([[0, 0, 1.0, 1, 0, 0, 0, 0, 0, 0], w0])
    errs = []
    for n in (8, 16, 32):
        xT, _ = m.replay(x0, np.full(n, 1.0 / n), T=1.0)
        errs.append(np.abs(xT[10:13] - _top_exact(w0, 1.0)).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 20 < e1 / e2 < 50


def test_damped_hinge_exponential_decay(orc):
    """Single z-axis hinge with damping b and no gravity torque: w(t) = w0 exp(-b t / I)."""
    sc = W.chain_cube_scene()
    sc["bodies"] = [sc["bodies"][0]]
    sc["bodies"][0]["damping"] = 0.3
    sc["geoms"] = [sc["geoms"][0]]
    sc["pairs"] = []
    sc["actuators"] = []
    sc["qpos0"] = [0.0]
    m = orc.OracleModel(sc)
    I = m.mass(np.zeros(1))[0, 0]
    r = m.rollout(np.array([0.2, 2.0]), T=1.5, rtol=1e-11, atol=1e-12)
    w = 2.0 * np.exp(-0.3 * 1.5 / I)
    assert abs(r["xT"][1] - w) < 1e-9
    assert abs(r["xT"][0] - (0.2 + 2.0 * I / 0.3 * (1 - np.exp(-0.3 * 1.5 / I)))) < 1e-9


def test_rest_height_of_stiff_contact(orc):
    """At rest a = 0 and J v = 0: the single-row solve reduces to
    k d(r)^2 (-r) = g (1 - d(r)) (from a_ref and R with A_hat = 1/m); the settled
    ball sits at R + r_rest with r_rest the root of that scalar equation."""
    sc = W.ball_scene()
    m = orc.OracleModel(sc)
    tc, damp = sc["options"]["solref"]
    dw = sc["options"]["solimp"][1]
    k = 1.0 / (dw ** 2 * tc ** 2 * damp ** 2)
    r_rest = brentq(lambda r: k * m.impedance(r) ** 2 * (-r) - 9.81 * (1 - m.impedance(r)), -0.0009, -1e-6, xtol=1e-16)
    assert -4e-4 < r_rest < -3.5e-4
    x0 = np.array([0, 0, 0.3, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0])
    res = m.rollout(x0, T=3.0)
    assert res["status"] == 0
    assert abs(res["xT"][2] - (0.1 + r_rest)) < 1e-8
    # and the right-hand side vanishes at the analytic rest state
    a = m.rhs(np.array([0, 0, 0.1 + r_rest, 1, 0, 0, 0]), np.zeros(6))
    assert abs(a[2]) < 1e-9


def test_frictionless_bounce_invariants(orc):
    """Normal forces through the COM: horizontal and angular velocity are exactly
    conserved; the critically damped contact never adds energy (compared at
    out-of-contact instants, where no energy is stored in the contact)."""
    m = orc.OracleModel(W.ball_scene())
    g = np.random.default_rng(13)
    inp = W.ball_inputs(6, seed=13)
    for x0 in inp["x0"]:
        x0 = x0.copy()
        x0[10:13] = g.normal(size=3)
        r = m.rollout(x0, T=1.0, NI=20)
        assert r["status"] == 0
        xb = r["xb"]
        np.testing.assert_allclose(xb[:, 7:9], np.broadcast_to(x0[7:9], xb[:, 7:9].shape), atol=1e-12)
        np.testing.assert_allclose(xb[:, 10:13], np.broadcast_to(x0[10:13], xb[:, 10:13].shape), atol=1e-12)
        E = 0.5 * (xb[:, 9] ** 2) + 9.81 * xb[:, 2]
        free = xb[:, 2] > 0.1            # out of contact: no energy stored in the contact
        assert np.all(np.diff(E[free]) <= 1e-6 * E[0])
        assert E[-1] <= E[0]
        assert E[-1] >= 9.81 * (0.1 - 4e-4)


def test_sliding_box_decelerates_at_mu_g(orc):
    """Box sliding on the plane: the pyramidal soft friction decelerates it at
    about mu g (2 %), and a box at rest stays at rest."""
    m = orc.OracleModel(W.box_scene(mu=0.5))
    x0 = np.array([0, 0, 0.0497, 1, 0, 0, 0, 1.5, 0, 0, 0, 0, 0])
    r = m.rollout(x0, T=0.2, NI=20)
    vx = r["xb"][:, 7]
    t = np.linspace(0, 0.2, 21)
    acc = np.polyfit(t[4:18], vx[4:18], 1)[0]
    assert abs(acc + 0.5 * 9.81) < 0.02 * 0.5 * 9.81
    rest = np.array([0, 0, 0.0497, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0])
    r = m.rollout(rest, T=1.0)
    assert np.abs(r["xT"][7:13]).max() < 1e-6
    assert np.abs(r["xT"][:2]).max() < 1e-7


def test_replay_reproduces_adaptive_rollout(orc):
    m = orc.OracleModel(W.box_scene())
    inp = W.box_push_inputs(3)
    for x0 in inp["x0"]:
        r = m.rollout(x0, T=1.0)
        xT, _ = m.replay(x0, r["hlog"], T=1.0)
        np.testing.assert_array_equal(xT, r["xT"])


def test_status_codes(orc):
    m = orc.OracleModel(W.ball_scene())
    x0 = W.ball_inputs(1)["x0"][0]
    assert m.rollout(x0, T=1.0, max_steps=10)["status"] == 1
    bad = x0.copy(); bad[2] = np.nan
    r = m.rollout(bad, T=1.0)
    assert r["status"] == 3 and r["nsteps"] == 0


def test_control_interval_boundaries_are_hit_exactly(orc):
    """Steps never straddle a control change: the interval boundary states are
    states of accepted steps, and the step count covers every boundary."""
    sc = W.chain_cube_scene()
    m = orc.OracleModel(sc)
    inp = W.chain_inputs(1, T=0.4, NI=8)
    r = m.rollout(inp["x0"][0], ctrl=inp["ctrl"][0], T=0.4, NI=8)
    assert r["status"] == 0
    t = np.concatenate([[0.0], np.cumsum(r["hlog"])])
    for k in range(1, 9):
        assert np.min(np.abs(t - 0.4 * k / 8)) < 1e-12


def test_chaos_floor(orc):
    """How far rounding-level differences travel in the box-push workload: the
    oracle's own replay (same step sizes) from x0 perturbed by 1e-15 relative
    moves by more than 1e-9 at T = 1 s (tumbling contact dynamics amplify it),
    while at 50 ms it stays below 1e-10.  Trajectory parity against another
    implementation is therefore checked per step and on short horizons."""
    from tests.conftest import rel_err
    sc, inp = W.box_scene(), W.box_push_inputs(4096)
    m = orc.OracleModel(sc)
    g = np.random.default_rng(3)
    far, near = [], []
    for e in range(8):
        x0 = inp["x0"][e]
        r = m.rollout(x0, T=1.0)
        r5 = m.rollout(x0, T=0.05)
        xp = x0 * (1 + 1e-15 * g.standard_normal(13))
        far.append(rel_err(m.replay(xp, r["hlog"], T=1.0)[0], r["xT"]))
        near.append(rel_err(m.replay(xp, r5["hlog"], T=0.05)[0], r5["xT"]))
    assert max(far) > 1e-9
    assert max(near) < 1e-10


# ------------------------------------------------------------------ other schemes (Fig. 12, Sec. 3.1)
def _hinge_scene(damping=0.3):
    sc = W.chain_cube_scene()
    sc["bodies"] = [sc["bodies"][0]]
    sc["bodies"][0]["damping"] = damping
    sc["geoms"] = [sc["geoms"][0]]
    sc["pairs"] = []
    sc["actuators"] = []
    sc["qpos0"] = [0.0]
    return sc


def test_semi_implicit_euler_closed_form(orc):
    """Damped hinge, v' = -c v with c = b / I: semi-implicit Euler gives
    v_n = v0 (1 - h c)^n and q_n = q0 + h sum_{k=1..n} v_k (the position takes
    the new velocity), exactly; the last step of the horizon is shortened."""
    m = orc.OracleModel(_hinge_scene())
    I = m.mass(np.zeros(1))[0, 0]
    c = 0.3 / I
    h, T = 0.01, 0.255
    r = m.rollout(np.array([0.2, 2.0]), T=T, h0=h, method="euler")
    assert r["status"] == 0 and r["nrej"] == 0
    hl = r["hlog"]
    assert len(hl) == 26 and np.all(hl[:25] == h) and abs(hl[25] - 0.005) < 1e-15
    v, q = 2.0, 0.2
    for hk in hl:
        v = v * (1 - hk * c)
        q = q + hk * v
    assert abs(r["xT"][1] - v) < 1e-14 and abs(r["xT"][0] - q) < 1e-14


def test_tsit5_step_is_the_stability_polynomial(orc):
    """On the linear damped hinge one Tsit5 step multiplies v by
    R(z) = 1 + z b^T (I - z A)^-1 1 (z = -h c) of the published tableau."""
    from tests.test_oracle_tableau import _golden_tsit5
    a, b, _, _ = _golden_tsit5()
    m = orc.OracleModel(_hinge_scene())
    c = 0.3 / m.mass(np.zeros(1))[0, 0]
    for h in (0.02, 0.05, 0.2, 0.7):                 # z from -0.2 to -7 (outside the stability region)
        z = -h * c
        R = 1 + z * b @ np.linalg.solve(np.eye(7) - z * a, np.ones(7))
        xT, _ = m.replay(np.array([0.0, 1.5]), [h], T=1e3, method="tsit5")
        assert abs(xT[1] - 1.5 * R) < 1e-13 * max(1.0, abs(1.5 * R))


@pytest.mark.parametrize("method,order", [("tsit5", 5), ("euler", 1)])
def test_convergence_order_of_other_schemes(orc, method, order):
    """Fixed steps on the torque-free top: the global error of the angular
    velocity falls by ~2^order per halving of h."""
    m = orc.OracleModel(_top_scene())
    w0 = np.array([1.0, 0.5, 4.0])
    x0 = np.concatenate([[0, 0, 1.0, 1, 0, 0, 0, 0, 0, 0], w0])
    ns = (32, 64, 128) if order == 5 else (200, 400, 800)
    errs = []
    for n in ns:
        xT, _ = m.replay(x0, np.full(n, 1.0 / n), T=1.0, method=method)
        errs.append(np.abs(xT[10:13] - _top_exact(w0, 1.0)).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 0.7 * 2 ** order < e1 / e2 < 1.5 * 2 ** order, errs


def test_tsit5_adaptive_rollout_and_controller(orc):
    """Tsit5 with the same PID controller: the ball drop integrates to the
    closed-form rest height, and on the top the accepted error norms settle
    at the PI fixed point 0.9^(5/I) like DOPRI5's."""
    sc = W.ball_scene()
    m = orc.OracleModel(sc)
    x0 = np.array([0, 0, 0.3, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0])
    a = m.rollout(x0, T=3.0)
    b = m.rollout(x0, T=3.0, method="tsit5")
    assert b["status"] == 0 and abs(b["xT"][2] - a["xT"][2]) < 1e-8
    mt = orc.OracleModel(_top_scene())
    xt = np.array([0, 0, 1.0, 1, 0, 0, 0, 0, 0, 0, 1.0, 0.5, 4.0])
    r = mt.rollout(xt, T=1.0, rtol=0.0, atol=1e-8, h0=5e-3, method="tsit5")
    x = xt.copy()
    errs = []
    for h in r["hlog"][:-1]:
        errs.append(mt.step_error(x, h, rtol=0.0, atol=1e-8, method="tsit5"))
        x, _ = mt.replay(x, [h], T=1e3, method="tsit5")
    np.testing.assert_allclose(errs[-10:], 0.9 ** 12.5, rtol=1e-6)
