"""GPU optimize-then-discretize gradient (dmx_rollout_grad_otd through the C
ABI; App. C.2, the continuous adjoint integrated backward together with the
state) against the oracle's backsolve from the same final state: the same
scheme, controller and interval clamping on both sides.  On smooth problems
(damped hinge, torque-free top) the backward step counts agree and the
gradients agree to rounding (1e-9 relative per environment, scale
max(|g_i|, ||g||_inf)); the hinge also against its closed form.  Through
contacts the backward state reconstruction runs each damped collision in
reverse, anti-damped, and amplifies rounding: the oracle's own gradient moves
by 1e-9 (arm) to 1e-4 and, for grazing shots, O(1) (billiard) when x0 moves
by 1e-15 relative, and its step counts by ~10%.  There each environment's GPU
gradient must lie within 10x that measured spread of the oracle's (at least
1e-9), and most environments must be well conditioned so that the bar bites:
billiard shots with and without the straight-through CFD adjoint (App. C.4),
arm controls with interval-boundary cotangents."""

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W
from tests.conftest import rel_err
from tests.test_oracle_integrator import _hinge_scene, _top_scene

pytestmark = pytest.mark.gpu
TOL = 1e-9


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


def _both(dmx, orc_mod, sc, x0, T, w, ctrl=None, NI=1, wb=None, cfd=False, rtol=1e-6, atol=1e-8, method="dopri5"):
    """Oracle forward + backsolve; the GPU backsolve from the oracle's xT."""
    om = orc_mod.OracleModel(sc)
    B = len(x0)
    Tv = np.broadcast_to(np.asarray(T, dtype=np.float64), (B,)).copy()
    o = om.batch_grad_otd(x0, Tv, w, ctrl=ctrl, NI=NI, rtol=rtol, atol=atol, cfd=cfd, xb_bar=wb, method=method)
    assert np.all(o["status"] == 0) and np.all(o["back_status"] == 0)
    m = dmx.Model(sc)
    gc = None if ctrl is None else _dev(np.transpose(ctrl, (1, 2, 0)))
    gwb = None if wb is None else _dev(np.transpose(wb, (1, 2, 0)))
    gx, gu, steps, status = dmx.rollout_grad_otd(m, _dev(o["xT"].T), _dev(Tv), _dev(np.asarray(w).T), ctrl=gc, NI=NI,
                                                 xb_bar=gwb, cfd=cfd, rtol=rtol, atol=atol, method=method)
    g = {"x0_bar": gx.cpu().numpy().T, "steps": steps.cpu().numpy(), "status": status.cpu().numpy()}
    if gu is not None:
        g["ctrl_bar"] = np.transpose(gu.cpu().numpy(), (2, 0, 1))
    assert np.all(g["status"] == 0), g["status"]
    return g, o


def _assert_parity(g, o, keys=("x0_bar",)):
    np.testing.assert_array_equal(g["steps"], o["back_steps"])
    for key in keys:
        err = max(rel_err(np.ravel(g[key][e]), np.ravel(o[key][e])) for e in range(len(o[key])))
        assert err < TOL, f"{key}: relative error {err:.3e}"


def _spread(orc_mod, sc, x0, T, w, o, keys, **kw):
    """Per environment: how far the oracle's backsolve gradient moves when x0
    is scaled by 1 + k 1e-15 (k = 1, 2, 3)."""
    om = orc_mod.OracleModel(sc)
    out = np.zeros(len(x0))
    for k in (1, 2, 3):
        p = om.batch_grad_otd(x0 * (1 + k * 1e-15), T, w, **kw)
        for e in range(len(x0)):
            for key in keys:
                out[e] = max(out[e], rel_err(np.ravel(p[key][e]), np.ravel(o[key][e])))
    return out


def _assert_within_spread(g, o, spread, keys=("x0_bar",), min_good=0.5):
    assert np.mean(spread < 1e-4) >= min_good, spread
    for key in keys:
        for e in range(len(spread)):
            err = rel_err(np.ravel(g[key][e]), np.ravel(o[key][e]))
            assert err <= max(10 * spread[e], TOL), f"{key} env {e}: {err:.3e} (oracle spread {spread[e]:.3e})"


def test_damped_hinge_closed_form(dmx, orc_mod):
    """v' = -c v: dv_T/dv0 = exp(-c T) and dq_T/dv0 = (1 - exp(-c T)) / c of the
    continuous map, reached to the tolerance on the GPU."""
    sc = _hinge_scene()
    om = orc_mod.OracleModel(sc)
    c = 0.3 / om.mass(np.zeros(1))[0, 0]
    x0 = np.array([[0.2, 2.0], [0.2, 2.0]])
    w = np.array([[0.0, 1.0], [1.0, 0.0]])
    g, o = _both(dmx, orc_mod, sc, x0, 1.0, w, rtol=1e-10, atol=1e-12)
    e = np.exp(-c)
    assert abs(g["x0_bar"][0][1] - e) < 1e-8 * e and abs(g["x0_bar"][0][0]) < 1e-15
    assert abs(g["x0_bar"][1][0] - 1.0) < 1e-12 and abs(g["x0_bar"][1][1] - (1 - e) / c) < 1e-9
    _assert_parity(g, o)


@pytest.mark.parametrize("method", ["dopri5", "tsit5"])
def test_top_parity(dmx, orc_mod, method):
    """Torque-free precession (quaternion state, gyroscopic right-hand side)."""
    g_ = np.random.default_rng(5)
    B = 8
    x0 = np.zeros((B, 13))
    x0[:, 2] = 1.0
    x0[:, 3] = 1.0
    x0[:, 7:13] = g_.normal(0.0, 1.0, (B, 6))
    x0[:, 12] += 4.0
    w = g_.normal(size=(B, 13))
    g, o = _both(dmx, orc_mod, _top_scene(), x0, 1.0, w, rtol=1e-8, atol=1e-10, method=method)
    _assert_parity(g, o)


@pytest.mark.parametrize("cfd", [False, True])
def test_billiard_parity(dmx, orc_mod, cfd):
    """Billiard shots (hits and misses): the collision run backward, with and
    without the straight-through CFD adjoint."""
    sc = W.billiard_scene(**W.CFD_OPTIONS) if cfd else W.billiard_scene()
    inp = W.billiard_inputs(16)
    w = np.zeros((16, 26)); w[:, 0] = 1.0; w[:, 7] = 0.5; w[:, 8] = 0.7; w[:, 1] = -0.4
    g, o = _both(dmx, orc_mod, sc, inp["x0"], inp["T"], w, cfd=cfd)
    _assert_within_spread(g, o, _spread(orc_mod, sc, inp["x0"], inp["T"], w, o, ("x0_bar",), cfd=cfd))


def test_arm_controls_parity(dmx, orc_mod):
    """Arm + cube, torques over 4 intervals, cotangents on the final state and
    on every interval-boundary state."""
    sc = W.chain_cube_scene()
    inp = W.chain_inputs(4, T=0.2, NI=4)
    g_ = np.random.default_rng(8)
    w = np.zeros((4, 27)); w[:, :7] = g_.normal(size=(4, 7)); w[:, 14:21] = g_.normal(size=(4, 7))
    wb = np.zeros((4, 5, 27)); wb[:, :, :7] = g_.normal(size=(4, 5, 7))
    kw = dict(ctrl=inp["ctrl"], NI=4, rtol=1e-8, atol=1e-10)
    g, o = _both(dmx, orc_mod, sc, inp["x0"], inp["T"], w, wb=wb, **kw)
    keys = ("x0_bar", "ctrl_bar")
    _assert_within_spread(g, o, _spread(orc_mod, sc, inp["x0"], inp["T"], w, o, keys, xb_bar=wb, **kw), keys)


def test_semi_implicit_euler_parity(dmx, orc_mod):
    """The fixed-step scheme backward (h = h0 every step, clamped at the
    horizon): the same step count as the forward and the oracle's gradient to
    rounding on the damped hinge and the top."""
    sc = _hinge_scene()
    x0 = np.array([[0.2, 2.0], [-0.1, 0.5]])
    w = np.array([[0.3, 1.0], [1.0, -0.2]])
    g, o = _both(dmx, orc_mod, sc, x0, 0.5, w, method="euler")
    _assert_parity(g, o)
    assert np.all(g["steps"] == int(round(0.5 / 1e-3)))
    g_ = np.random.default_rng(9)
    x0 = np.zeros((4, 13)); x0[:, 2] = 1.0; x0[:, 3] = 1.0
    x0[:, 7:13] = g_.normal(0.0, 1.0, (4, 6))
    g, o = _both(dmx, orc_mod, _top_scene(), x0, 0.3, g_.normal(size=(4, 13)), method="euler")
    _assert_parity(g, o)


def test_step_budget_status(dmx):
    """A backward solve that runs out of attempts reports MAX_STEPS per
    environment (and leaves the others untouched)."""
    import torch
    sc = _top_scene()
    m = dmx.Model(sc)
    B = 4
    xT = np.zeros((B, 13)); xT[:, 2] = 1.0; xT[:, 3] = 1.0; xT[:, 12] = 4.0
    T = np.array([1.0, 1.0, 1e-4, 1e-4])
    w = np.ones((B, 13))
    gx, _, steps, status = dmx.rollout_grad_otd(m, _dev(xT.T), _dev(T), _dev(w.T), rtol=1e-10, atol=1e-12,
                                                max_steps=5)
    status = status.cpu().numpy()
    assert list(status[:2]) == [1, 1]                   # DMX_ENV_MAX_STEPS
    assert list(status[2:]) == [0, 0]
    assert torch.isfinite(gx).all()
