"""Pins of the oracle's sphere / capsule pair contacts (the billiard of
Sec. 4 and App. C.4; capsule pairs of App. C.1): the signed distance and
normal against brute-force minimisation over the two segments, closed forms
(two spheres, parallel capsules), the contact frame, the right-hand side's
Jacobian against central differences at colliding states, and conservation
of linear and angular momentum through ball-ball and capsule collisions
(internal forces only, no gravity)."""

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W


def _segment(q, k, geom_half):
    """Centre and axis (body x) of the segment of free body k in q."""
    p = q[7 * k:7 * k + 3]
    w, x, y, z = q[7 * k + 3:7 * k + 7] / np.linalg.norm(q[7 * k + 3:7 * k + 7])
    ax = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
    return p, ax, geom_half


def _brute(pa, ua, La, pb, ub, Lb, n=401):
    """Least distance between two segments by a dense grid and local refinement."""
    s = np.linspace(-La, La, n) if La > 0 else np.zeros(1)
    t = np.linspace(-Lb, Lb, n) if Lb > 0 else np.zeros(1)
    P = pa + s[:, None] * ua
    Q = pb + t[:, None] * ub
    d = np.linalg.norm(P[:, None, :] - Q[None, :, :], axis=2)
    i, j = np.unravel_index(np.argmin(d), d.shape)
    from scipy.optimize import minimize
    f = lambda z: np.linalg.norm(pa + z[0] * ua - pb - z[1] * ub)
    r = minimize(f, [s[i], t[j]], bounds=[(-La, La), (-Lb, Lb)], method="L-BFGS-B", options={"ftol": 1e-15, "gtol": 1e-12})
    z = r.x
    return f(z), pa + z[0] * ua - (pb + z[1] * ub)


def test_pair_distance_and_normal_brute_force(orc):
    """Capsule-capsule, sphere-capsule and capsule-sphere slots at seeded
    poses: r + radii = least distance between the segments (1e-9), normal =
    direction from geom 2's closest point to geom 1's (1e-6), frame
    orthonormal and right-handed, position on the normal between the
    surfaces."""
    sc = W.capsules_scene()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(5)
    halves = [0.1, 0.0, 0.1]
    radii = [0.03, 0.04, 0.03]
    for trial in range(20):
        q = np.array(sc["qpos0"], float)
        for k in range(3):
            q[7 * k:7 * k + 3] += g.normal(0.0, 0.08, 3)
            qq = g.normal(size=4)
            q[7 * k + 3:7 * k + 7] = qq / np.linalg.norm(qq)
        ct = m.contacts(q)
        for s, p in enumerate(sc["pairs"]):
            a, b = p["geom1"], p["geom2"]
            pa, ua, La = _segment(q, a, halves[a])
            pb, ub, Lb = _segment(q, b, halves[b])
            dist, dvec = _brute(pa, ua, La, pb, ub, Lb)
            r, pos, n, t1, t2 = ct[s, 0], ct[s, 1:4], ct[s, 4:7], ct[s, 7:10], ct[s, 10:13]
            assert abs(r - (dist - radii[a] - radii[b])) < 1e-9
            np.testing.assert_allclose(n, dvec / np.linalg.norm(dvec), atol=1e-6)
            F = np.stack([n, t1, t2])
            np.testing.assert_allclose(F @ F.T, np.eye(3), atol=1e-12)
            assert np.dot(np.cross(n, t1), t2) > 0.999999
            assert ct[s, 13] == a and ct[s, 14] == b


def test_two_spheres_closed_form(orc):
    """Ball-ball: r = |c1 - c2| - r1 - r2, n along c1 - c2, pos halfway into the overlap."""
    m = orc.OracleModel(W.billiard_scene())
    q = np.array(W.billiard_scene()["qpos0"], float)
    q[7:10] = [0.07, 0.05, -0.02]
    ct = m.contacts(q)[0]
    d = q[0:3] - q[7:10]
    r = np.linalg.norm(d) - 0.1
    n = d / np.linalg.norm(d)
    assert abs(ct[0] - r) < 1e-15
    np.testing.assert_allclose(ct[4:7], n, atol=1e-15)
    np.testing.assert_allclose(ct[1:4], q[0:3] - (0.05 + r / 2) * n, atol=1e-15)


def test_parallel_capsules_closed_form(orc):
    """Two parallel capsules side by side (overlapping along their axes): the
    distance is that of the axes, the normal perpendicular to both."""
    m = orc.OracleModel(W.capsules_scene())
    q = np.array(W.capsules_scene()["qpos0"], float)
    q[0:3] = [0.0, 0.0, 0.0]
    q[14:17] = [0.05, 0.0, 0.061]      # capsule 3 shifted along the shared x axis and lifted
    ct = m.contacts(q)[0]
    assert abs(ct[0] - (0.061 - 0.06)) < 1e-15
    np.testing.assert_allclose(ct[4:7], [0.0, 0.0, -1.0], atol=1e-15)


@pytest.mark.parametrize("name", ["billiard", "capsules"])
def test_pair_rhs_jacobian_matches_differences(orc, name):
    """The right-hand side's forward-mode Jacobian (through the closest-point
    derivatives) against central differences at colliding states."""
    sc = W.SCENES[name]()
    m = orc.OracleModel(sc)
    inp = W.INPUTS[name](6)
    checked = 0
    for x0 in inp["x0"]:
        r = m.rollout(x0, T=float(inp["T"][0]), NI=40)
        for xb in r["xb"]:
            q, v = xb[:m.nq], xb[m.nq:]
            ct = m.contacts(q)
            if ct[:, 0].min() >= -1e-5 or not m.rhs(q, v, detail=True)[1]["active"].any():
                continue                      # no contact force at this state
            Jq, Jv, _ = m.rhs_jacobian(q, v)
            for i in range(m.nq):
                e = np.zeros(m.nq); e[i] = 1e-7
                fd = (m.rhs(q + e, v) - m.rhs(q - e, v)) / 2e-7
                np.testing.assert_allclose(Jq[:, i], fd, rtol=1e-4, atol=1e-4 * np.abs(Jq).max())
            for i in range(m.nv):
                e = np.zeros(m.nv); e[i] = 1e-7
                fd = (m.rhs(q, v + e) - m.rhs(q, v - e)) / 2e-7
                np.testing.assert_allclose(Jv[:, i], fd, rtol=1e-4, atol=1e-4 * np.abs(Jv).max())
            checked += 1
            break
    assert checked >= 3


def _momenta(sc, x):
    nb = len(sc["bodies"])
    P = np.zeros(3); Lm = np.zeros(3)
    for k in range(nb):
        b = sc["bodies"][k]
        c = x[7 * k:7 * k + 3]
        w, qx, qy, qz = x[7 * k + 3:7 * k + 7]
        R = np.array([[1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - w * qz), 2 * (qx * qz + w * qy)],
                      [2 * (qx * qy + w * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - w * qx)],
                      [2 * (qx * qz - w * qy), 2 * (qy * qz + w * qx), 1 - 2 * (qx * qx + qy * qy)]])
        vv = x[7 * nb + 6 * k:7 * nb + 6 * k + 3]
        om = x[7 * nb + 6 * k + 3:7 * nb + 6 * k + 6]     # body frame
        P += b["mass"] * vv
        Lm += b["mass"] * np.cross(c, vv) + R @ (np.array(b["inertia"]) * om)
    return P, Lm


@pytest.mark.parametrize("name", ["billiard", "capsules"])
def test_collisions_conserve_momentum(orc, name):
    """Contacts between free bodies without gravity are internal forces (equal
    and opposite at one point): total linear momentum is the same before and
    after, to the integration tolerance (rtol 1e-10); so is the angular
    momentum of the balls.  (For the spinning capsules the orientation update
    q (x) exp(h sum_j b_j w_j / 2) drops the commutator of the body rates:
    second order in h and not seen by the embedded error estimate, so their
    angular momentum drifts by ~1e-6 even without contacts.)"""
    sc = W.SCENES[name]()
    m = orc.OracleModel(sc)
    inp = W.INPUTS[name](8)
    hits = 0
    for x0 in inp["x0"]:
        r = m.rollout(x0, T=float(inp["T"][0]), rtol=1e-10, atol=1e-12, max_steps=200000)
        assert r["status"] == 0
        P0, L0 = _momenta(sc, x0)
        P1, L1 = _momenta(sc, r["xT"])
        np.testing.assert_allclose(P1, P0, atol=1e-11)
        if name == "billiard":
            np.testing.assert_allclose(L1, L0, atol=1e-10)
        hits += int(np.abs(r["xT"][7 * len(sc["bodies"]):] - x0[7 * len(sc["bodies"]):]).max() > 1e-3)
    assert hits >= 4


@pytest.mark.parametrize("name", ["billiard", "capsules"])
def test_pair_gradient_frozen_steps(orc, name):
    """Discrete adjoint through ball-ball and capsule contacts against central
    differences of the replayed map (every input direction)."""
    from tests.test_oracle_adjoint import _best_fd_err
    sc = W.SCENES[name]()
    m = orc.OracleModel(sc)
    inp = W.INPUTS[name](4)
    e = 0                                       # a hit in both scenes
    x0, T = inp["x0"][e], float(inp["T"][e])
    r = m.rollout(x0, T=T)
    w = np.random.default_rng(6).normal(size=m.nx)
    g = m.rollout_grad(x0, w, T=T)
    assert np.abs(g["x0_bar"]).max() > 0
    assert _best_fd_err(m, x0, r["hlog"], w, g, T=T) < 1e-5
