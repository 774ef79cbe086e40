"""Pins of the oracle's optimize-then-discretize gradient (App. C.2, Eq.
adjoint-equations: the continuous adjoint integrated backward together with
the state, BacksolveAdjoint) and of its straight-through variant with the
CFD right-hand side (App. C.4): closed forms of the continuous gradient
(damped hinge, ballistic flight), agreement with central differences of the
tight-tolerance continuous map (top, billiard hits, arm controls with
interval-boundary cotangents), convergence with the tolerance, and the
billiard behaviour the paper reports (zero plain gradient for a miss,
informative straight-through gradient)."""

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W
from tests.conftest import rel_err
from tests.test_oracle_integrator import _hinge_scene, _top_scene


def _otd(m, x0, w, T, **kw):
    g = m.batch_grad_otd(np.atleast_2d(x0), np.array([T]), np.atleast_2d(w), **kw)
    assert g["status"][0] == 0 and g["back_status"][0] == 0
    return g


def test_damped_hinge_continuous_gradient(orc):
    """v' = -c v: dv_T/dv0 = exp(-c T), dq_T/dv0 = (1 - exp(-c T)) / c,
    dq_T/dq0 = 1 (the continuous map, which OTD approximates to the
    tolerance: 1e-8 at rtol 1e-10)."""
    m = orc.OracleModel(_hinge_scene())
    c = 0.3 / m.mass(np.zeros(1))[0, 0]
    T = 1.0
    x0 = np.array([0.2, 2.0])
    g = _otd(m, x0, [0.0, 1.0], T, rtol=1e-10, atol=1e-12)["x0_bar"][0]
    assert abs(g[1] - np.exp(-c * T)) < 1e-8 * np.exp(-c * T) and g[0] == 0.0
    g = _otd(m, x0, [1.0, 0.0], T, rtol=1e-10, atol=1e-12)["x0_bar"][0]
    assert abs(g[0] - 1.0) < 1e-12 and abs(g[1] - (1 - np.exp(-c * T)) / c) < 1e-9


def test_ballistic_continuous_gradient(orc):
    m = orc.OracleModel(W.ball_scene())
    x0 = np.array([0.1, -0.2, 2.0, 1, 0, 0, 0, 0.7, -0.4, 1.5, 0, 0, 0])
    w = np.zeros(13); w[2] = 1.0; w[7] = 2.0
    g = _otd(m, x0, w, 0.4)["x0_bar"][0]
    ref = np.zeros(13); ref[2] = 1.0; ref[9] = 0.4; ref[7] = 2.0
    np.testing.assert_allclose(g, ref, atol=1e-12)


def _fd_continuous(m, x0, w, T, idx, eps=1e-6, ctrl=None, NI=1, wb=None, rtol=1e-11):
    """Central differences of <w, x(T)> (+ sum_k <wb_k, x(t_k)>) of the
    tight-tolerance free-running rollout (the continuous map)."""
    out = []
    for i in idx:
        vals = []
        for sgn in (1.0, -1.0):
            if i < m.nx:
                x = x0.copy(); x[i] += sgn * eps; c = ctrl
            else:
                x = x0; c = ctrl.copy(); c.reshape(-1)[i - m.nx] += sgn * eps
            r = m.rollout(x, ctrl=c, T=T, NI=NI, rtol=rtol, atol=rtol * 1e-2, h0=1e-4, max_steps=10 ** 6)
            v = w @ r["xT"]
            if wb is not None:
                v += (wb * r["xb"]).sum()
            vals.append(v)
        out.append((vals[0] - vals[1]) / (2 * eps))
    return np.array(out)


def test_top_against_continuous_differences(orc):
    """Torque-free precession over 1 s: the OTD gradient w.r.t. the initial
    velocities equals central differences of the continuous map; it
    converges as the tolerance shrinks.  (The loss leaves the quaternion out:
    its computed value carries the orientation update's step-sequence
    dependent error, which differences of perturbed rollouts would pick up.)"""
    m = orc.OracleModel(_top_scene())
    x0 = np.array([0, 0, 1.0, 1, 0, 0, 0, 0.1, 0, 0, 1.0, 0.5, 4.0])
    w = np.random.default_rng(2).normal(size=13)
    w[3:7] = 0.0
    idx = list(range(7, 13))
    fd = _fd_continuous(m, x0, w, 1.0, idx)
    errs = [rel_err(_otd(m, x0, w, 1.0, rtol=rt, atol=rt * 1e-2)["x0_bar"][0][idx], fd) for rt in (1e-5, 1e-7, 1e-9)]
    assert errs[2] < 1e-6 and errs[0] > errs[2], errs


def test_billiard_hits_against_continuous_differences(orc):
    """Ball-ball hits: the OTD gradient w.r.t. the initial state against central
    differences of the continuous map within 5e-4 at rtol 1e-8, and at every
    tolerance at least 10x closer to it than the discrete adjoint of the same
    forward solve (the DTO gradient differentiates the discretisation; App.
    C.2).  The backward solve runs the collision in reverse (anti-damped),
    which is why it needs its own steps."""
    sc = W.billiard_scene()
    m = orc.OracleModel(sc)
    inp = W.billiard_inputs(8)
    w = np.zeros(26); w[0] = 1.0; w[8] = 0.7; w[1] = -0.4
    idx = [0, 1, 7, 8, 13, 14, 15, 20]
    hits = 0
    for e in range(8):
        x0, T = inp["x0"][e], float(inp["T"][e])
        if m.rollout(x0, T=T)["nsteps"] < 15:
            continue                                   # a miss
        fd = _fd_continuous(m, x0, w, T, idx)
        for rt in (1e-6, 1e-8):
            g = _otd(m, x0, w, T, rtol=rt, atol=rt * 1e-2)["x0_bar"][0]
            d = m.batch_grad(x0[None], np.array([T]), w[None], rtol=rt, atol=rt * 1e-2)["x0_bar"][0]
            e_otd, e_dto = rel_err(g[idx], fd), rel_err(d[idx], fd)
            assert 10 * e_otd < e_dto, (e, rt, e_otd, e_dto)
            if rt == 1e-8:
                assert e_otd < 5e-4, (e, e_otd)
        hits += 1
    assert hits >= 3


def test_billiard_miss_straight_through(orc):
    """A miss by 1 cm over 0.4 s: the plain gradient of the target ball's
    final x w.r.t. the cue ball's state is zero (no contact ever), the
    straight-through OTD gradient with contacts from distance is not, and
    points towards a hit (App. C.4, Sec. 4): moving the cue ball towards the
    target's side, or the target towards the cue line, raises the loss.
    (An adaptive solver sees the interaction only at its stage states: over
    0.5 s the backward steps grow past the 0.1 s window of the approach, as
    the paper notes for the forward steps of DTO.)"""
    sc = W.billiard_scene(**W.CFD_OPTIONS)
    m = orc.OracleModel(sc)
    x0 = W.billiard_inputs(1)["x0"][0].copy()
    x0[8] = 0.11 - x0[1]                               # target 0.11 m off the cue line: a miss by 1 cm
    w = np.zeros(26); w[7] = 1.0                        # loss: target ball's final x
    T = 0.4
    assert m.rollout(x0, T=T)["xT"][7] == x0[7]
    plain = _otd(m, x0, w, T)["x0_bar"][0]
    st = _otd(m, x0, w, T, cfd=True)["x0_bar"][0]
    cue = list(range(0, 7)) + list(range(14, 20))
    assert np.abs(plain[cue]).max() == 0.0
    assert st[1] > 1e-2 and st[8] < -1e-2


def test_arm_controls_against_continuous_differences(orc):
    """Arm + cube, torques over 4 intervals, loss on the final state and on the
    interval-boundary states: OTD control gradients (a_u collected per
    interval, boundary cotangents as jumps) against central differences of the
    continuous map."""
    sc = W.chain_cube_scene()
    m = orc.OracleModel(sc)
    inp = W.chain_inputs(1, T=0.2, NI=4)
    x0, ctrl = inp["x0"][0], inp["ctrl"][0]
    g_ = np.random.default_rng(8)
    w = np.zeros(27); w[:7] = g_.normal(size=7); w[14:21] = g_.normal(size=7)
    wb = np.zeros((5, 27)); wb[:, :7] = g_.normal(size=(5, 7))
    g = m.batch_grad_otd(x0[None], np.array([0.2]), w[None], ctrl=ctrl[None], NI=4, rtol=1e-9, atol=1e-11,
                         xb_bar=wb[None])
    assert g["back_status"][0] == 0
    idx = list(range(27, 27 + 28, 3))
    fd = _fd_continuous(m, x0, w, 0.2, idx, ctrl=ctrl, NI=4, wb=wb)
    got = g["ctrl_bar"][0].ravel()[[i - 27 for i in idx]]
    assert rel_err(got, fd) < 1e-5
    arm = list(range(7)) + list(range(14, 21))
    fdx = _fd_continuous(m, x0, w, 0.2, arm, ctrl=ctrl, NI=4, wb=wb)
    assert rel_err(g["x0_bar"][0][arm], fdx) < 1e-5
