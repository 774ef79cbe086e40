"""Pins of the oracle's kinematics, mass matrix, bias force and collision
against closed forms, the textbook definitions written independently of the
recursive algorithms, and finite differences of the kinematics."""

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W


def _rand_quat(g):
    q = g.normal(size=4)
    return q / np.linalg.norm(q)


def _rand_state(model, scene, g, vscale=1.0):
    q = np.array(scene["qpos0"], dtype=float)
    qa = 0
    for b in scene["bodies"]:
        if b["joint"] == "free":
            q[qa:qa + 3] += g.normal(scale=0.3, size=3)
            q[qa + 3:qa + 7] = _rand_quat(g)
            qa += 7
        else:
            q[qa] = g.uniform(-1.0, 1.0)
            qa += 1
    v = g.normal(scale=vscale, size=model.nv)
    return q, v


def _quat_mat(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("scene_fn,inertia", [(W.ball_scene, 0.4 * 1.0 * 0.1 ** 2), (W.box_scene, 1.0 * 0.1 ** 2 / 6)])
def test_free_body_mass_matrix_closed_form(orc, scene_fn, inertia):
    m = orc.OracleModel(scene_fn())
    g = np.random.default_rng(0)
    for _ in range(5):
        q = np.concatenate([g.normal(size=3), _rand_quat(g)])
        M = m.mass(q)
        np.testing.assert_allclose(M, np.diag([1, 1, 1, inertia, inertia, inertia]), atol=1e-14)


def test_free_body_bias_closed_form(orc):
    """c = [-m g ; w x I w] for a free body with its COM at the body origin
    (linear velocity in world axes, angular velocity in body axes)."""
    sc = W.box_scene()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(1)
    I = np.array(sc["bodies"][0]["inertia"])
    for _ in range(5):
        q = np.concatenate([g.normal(size=3), _rand_quat(g)])
        v = g.normal(size=6)
        c = m.bias(q, v)
        w = v[3:]
        np.testing.assert_allclose(c[:3], [0, 0, 9.81], atol=1e-12)
        np.testing.assert_allclose(c[3:], np.cross(w, I * w), atol=1e-14)


SCENES = [W.ball_scene, W.box_scene, W.chain_cube_scene, W.quadruped_scene]


@pytest.mark.parametrize("scene_fn", SCENES)
def test_point_jacobian_matches_kinematics_fd(orc, scene_fn):
    """J_lin v and J_ang v equal the finite-difference rates of a body-fixed
    point and of the body orientation along q(eps) = q (+) eps v."""
    sc = scene_fn()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(2)
    q, v = _rand_state(m, sc, g)
    eps = 1e-6
    Rp, pp, _ = m.kinematics(m.integrate_pos(q, eps * v))
    Rm, pm, _ = m.kinematics(m.integrate_pos(q, -eps * v))
    R0, p0, _ = m.kinematics(q)
    for b in range(m.nbody):
        xl = g.normal(scale=0.2, size=3)
        x = p0[b] + R0[b] @ xl
        Jl, Ja = m.point_jacobian(q, b, x)
        vel_fd = ((pp[b] + Rp[b] @ xl) - (pm[b] + Rm[b] @ xl)) / (2 * eps)
        np.testing.assert_allclose(Jl @ v, vel_fd, atol=1e-8 * (1 + np.abs(vel_fd).max()))
        Rdot = (Rp[b] - Rm[b]) / (2 * eps)
        W_ = Rdot @ R0[b].T
        w_fd = np.array([W_[2, 1], W_[0, 2], W_[1, 0]])
        np.testing.assert_allclose(Ja @ v, w_fd, atol=1e-8 * (1 + np.abs(w_fd).max()))


def _body_inertia_world(sc, R):
    return [R[b] @ np.diag(sc["bodies"][b]["inertia"]) @ R[b].T for b in range(len(sc["bodies"]))]


@pytest.mark.parametrize("scene_fn", SCENES)
def test_crba_equals_sum_of_body_jacobian_inertias(orc, scene_fn):
    """CRBA result equals the definition M = sum_b m_b Jc^T Jc + Jw^T I_b Jw."""
    sc = scene_fn()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(3)
    for _ in range(3):
        q, _ = _rand_state(m, sc, g)
        R, p, com = m.kinematics(q)
        Iw = _body_inertia_world(sc, R)
        Mdef = np.zeros((m.nv, m.nv))
        for b in range(m.nbody):
            Jl, Ja = m.point_jacobian(q, b, com[b])
            Mdef += sc["bodies"][b]["mass"] * Jl.T @ Jl + Ja.T @ Iw[b] @ Ja
        M = m.mass(q)
        np.testing.assert_allclose(M, Mdef, atol=1e-12 * np.abs(Mdef).max())
        np.testing.assert_allclose(M, M.T, atol=0)
        assert np.linalg.eigvalsh(M).min() > 0


@pytest.mark.parametrize("scene_fn", SCENES)
def test_kinetic_energy_from_finite_difference_body_velocities(orc, scene_fn):
    sc = scene_fn()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(4)
    q, v = _rand_state(m, sc, g)
    eps = 1e-6
    Rp, _, cp = m.kinematics(m.integrate_pos(q, eps * v))
    Rm, _, cm = m.kinematics(m.integrate_pos(q, -eps * v))
    R0, _, _ = m.kinematics(q)
    Iw = _body_inertia_world(sc, R0)
    ke = 0.0
    for b in range(m.nbody):
        vc = (cp[b] - cm[b]) / (2 * eps)
        W_ = ((Rp[b] - Rm[b]) / (2 * eps)) @ R0[b].T
        w = np.array([W_[2, 1], W_[0, 2], W_[1, 0]])
        ke += 0.5 * sc["bodies"][b]["mass"] * vc @ vc + 0.5 * w @ Iw[b] @ w
    assert abs(0.5 * v @ m.mass(q) @ v - ke) < 1e-8 * max(1.0, ke)


@pytest.mark.parametrize("scene_fn", SCENES)
def test_gravity_force_is_potential_gradient(orc, scene_fn):
    """c(q, 0) = dV/dq along every tangent direction, V = -sum_b m_b g . com_b."""
    sc = scene_fn()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(5)
    q, _ = _rand_state(m, sc, g)
    grav = np.array(sc["options"]["gravity"])
    masses = np.array([b["mass"] for b in sc["bodies"]])

    def V(qq):
        _, _, com = m.kinematics(qq)
        return -(masses[:, None] * com @ grav).sum()

    c0 = m.bias(q, np.zeros(m.nv))
    eps = 1e-6
    for k in range(m.nv):
        e = np.zeros(m.nv); e[k] = eps
        dV = (V(m.integrate_pos(q, e)) - V(m.integrate_pos(q, -e))) / (2 * eps)
        assert abs(c0[k] - dV) < 1e-7 * (1 + abs(dV))


@pytest.mark.parametrize("scene_fn", SCENES)
def test_velocity_product_terms_match_newton_euler_definition(orc, scene_fn):
    """c(q,v) - c(q,0) = sum_b m Jc^T (Jc' v) + Jw^T (I Jw' v + w x I w), with the
    Jacobian rates taken by central differences along q (+) eps v."""
    sc = scene_fn()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(6)
    q, v = _rand_state(m, sc, g)
    eps = 1e-6
    qp, qm = m.integrate_pos(q, eps * v), m.integrate_pos(q, -eps * v)
    R0, p0, com0 = m.kinematics(q)
    Rp, pp, _ = m.kinematics(qp)
    Rm, pm, _ = m.kinematics(qm)
    Iw = _body_inertia_world(sc, R0)
    ref = np.zeros(m.nv)
    for b in range(m.nbody):
        cl = R0[b].T @ (com0[b] - p0[b])          # COM in body coordinates
        Jl0, Ja0 = m.point_jacobian(q, b, com0[b])
        Jlp, Jap = m.point_jacobian(qp, b, pp[b] + Rp[b] @ cl)
        Jlm, Jam = m.point_jacobian(qm, b, pm[b] + Rm[b] @ cl)
        acc = (Jlp - Jlm) @ v / (2 * eps)
        alp = (Jap - Jam) @ v / (2 * eps)
        w = Ja0 @ v
        ref += sc["bodies"][b]["mass"] * Jl0.T @ acc + Ja0.T @ (Iw[b] @ alp + np.cross(w, Iw[b] @ w))
    got = m.bias(q, v) - m.bias(q, np.zeros(m.nv))
    np.testing.assert_allclose(got, ref, atol=1e-6 * (1 + np.abs(ref).max()))


@pytest.mark.parametrize("scene_fn", SCENES)
def test_coriolis_power_identity(orc, scene_fn):
    """v^T M' v = 2 v^T (c(q,v) - c(q,0)) with M' = dM/dt along q (+) t v."""
    sc = scene_fn()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(7)
    q, v = _rand_state(m, sc, g)
    eps = 1e-6
    Md = (m.mass(m.integrate_pos(q, eps * v)) - m.mass(m.integrate_pos(q, -eps * v))) / (2 * eps)
    lhs = v @ Md @ v
    rhs = 2 * v @ (m.bias(q, v) - m.bias(q, np.zeros(m.nv)))
    assert abs(lhs - rhs) < 1e-6 * (1 + abs(lhs))


def test_box_vertex_contacts_closed_form(orc):
    m = orc.OracleModel(W.box_scene())
    g = np.random.default_rng(8)
    for _ in range(3):
        p = g.normal(size=3) * 0.1 + [0, 0, 0.06]
        quat = _rand_quat(g)
        ct = m.contacts(np.concatenate([p, quat]))
        R = _quat_mat(quat)
        for j in range(8):
            s = np.array([0.05 if j & 1 else -0.05, 0.05 if j & 2 else -0.05, 0.05 if j & 4 else -0.05])
            v = p + R @ s
            assert abs(ct[j, 0] - v[2]) < 1e-15
            np.testing.assert_allclose(ct[j, 1:4], v - 0.5 * v[2] * np.array([0, 0, 1]), atol=1e-15)
            np.testing.assert_allclose(ct[j, 4:13], [0, 0, 1, 1, 0, 0, 0, 1, 0], atol=0)


def test_sphere_contact_closed_form(orc):
    m = orc.OracleModel(W.ball_scene())
    ct = m.contacts(np.array([0.3, -0.2, 0.0995, 1, 0, 0, 0]))
    assert abs(ct[0, 0] - (-0.0005)) < 1e-16
    np.testing.assert_allclose(ct[0, 1:4], [0.3, -0.2, -0.00025], atol=1e-16)


def _box_sdf(y, h):
    qd = np.abs(y) - h
    out = np.linalg.norm(np.maximum(qd, 0), axis=-1)
    inside = np.minimum(qd.max(axis=-1), 0)
    return out + inside


def test_capsule_box_distance_brute_force(orc):
    """Signed distance, contact point and normal of the capsule-box pair against
    dense sampling of the capsule axis and the exact box distance field."""
    sc = W.chain_cube_scene()
    m = orc.OracleModel(sc)
    g = np.random.default_rng(9)
    h = np.array([0.05, 0.05, 0.05])
    slot0 = 8           # cube-plane slots come first
    checked = 0
    for trial in range(40):
        q = np.array(sc["qpos0"], dtype=float)
        q[:7] = g.uniform(-0.6, 0.6, 7)
        q[7:10] = [g.uniform(0.8, 2.2), g.uniform(-0.5, 0.6), 0.05 + g.uniform(-0.02, 0.02)]
        q[10:14] = _rand_quat(g) if trial % 2 else [np.cos(0.3 * trial), 0, 0, np.sin(0.3 * trial)]
        R, p, _ = m.kinematics(q)
        ct = m.contacts(q)
        Rb, pb = R[7], p[7]
        for link in range(7):
            cen = p[link] + R[link] @ np.array([0.15, 0, 0])
            u = R[link][:, 0]
            s = np.linspace(-0.15, 0.15, 200001)
            pts = cen[None, :] + s[:, None] * u[None, :]
            d = _box_sdf((pts - pb) @ Rb, h)
            i = int(np.argmin(d))
            r_ref = d[i] - 0.025
            row = ct[slot0 + link]
            # outside the box the distance is smooth along the axis (sampling error is
            # quadratic in the spacing); inside it is piecewise linear (linear error)
            assert abs(row[0] - r_ref) < (1e-8 if d[i] > 0 else 2e-6)
            assert row[0] <= r_ref + 1e-12
            if d[i] > 1e-3 and 0 < i < len(s) - 1:
                # normal = gradient of the distance field at the closest axis point
                x = pts[i]
                e = 1e-6
                grad = np.array([(_box_sdf(((x + e * ax) - pb) @ Rb, h) - _box_sdf(((x - e * ax) - pb) @ Rb, h)) / (2 * e)
                                 for ax in np.eye(3)])
                np.testing.assert_allclose(row[4:7], grad, atol=2e-4)
                checked += 1
            n = row[4:7]
            assert abs(np.linalg.norm(n) - 1) < 1e-12
            assert abs(n @ row[7:10]) < 1e-12 and abs(n @ row[10:13]) < 1e-12
    assert checked > 20


def test_impedance_spline_points(orc):
    """solimp (0, 0.95, 0.001, 0.5, 2): d(0) = d_o, d(-w) = d_w, d(-mid w) =
    d_o + mid (d_w - d_o), x^p / mid^(p-1) below the midpoint; CFD continuation
    (d_c, d_0, w_c, m_c, p_c) = (0, 0.1, 0.05, 1, 4) meets d_0 at r = 0 and d_c at w_c."""
    sc = W.ball_scene(**W.CFD_OPTIONS)
    m = orc.OracleModel(sc)
    assert abs(m.impedance(0.0) - 0.1) < 1e-15
    assert abs(m.impedance(-0.001) - 0.95) < 1e-15
    assert abs(m.impedance(-0.01) - 0.95) < 1e-15
    assert abs(m.impedance(-0.0005) - (0.1 + 0.5 * 0.85)) < 1e-15
    x = 0.25
    assert abs(m.impedance(-0.00025) - (0.1 + 0.85 * x * x / 0.5)) < 1e-15
    x = 0.75
    assert abs(m.impedance(-0.00075) - (0.1 + 0.85 * (1 - (1 - x) ** 2 / 0.5))) < 1e-15
    assert abs(m.impedance(0.0, cfd=True) - 0.1) < 1e-15
    assert abs(m.impedance(0.05, cfd=True) - 0.0) < 1e-15
    assert abs(m.impedance(0.025, cfd=True) - 0.1 * 0.5 ** 4) < 1e-15
    rs = np.linspace(-0.002, 0.0, 2001)
    d = np.array([m.impedance(r) for r in rs])
    assert np.all(np.diff(d) <= 1e-15)      # monotone in the violation


def test_integrate_pos_group_properties(orc):
    m = orc.OracleModel(W.box_scene())
    g = np.random.default_rng(10)
    q = np.concatenate([g.normal(size=3), _rand_quat(g)])
    ax = g.normal(size=3); ax /= np.linalg.norm(ax)
    a = np.concatenate([g.normal(size=3), 0.3 * ax]); b = np.concatenate([g.normal(size=3), 0.5 * ax])
    np.testing.assert_allclose(m.integrate_pos(m.integrate_pos(q, a), b), m.integrate_pos(q, a + b), atol=1e-14)
    # rotation by angle theta about body axis: R(q') = R(q) Rot(axis, theta)
    th = 0.7
    q2 = m.integrate_pos(q, np.concatenate([np.zeros(3), th * ax]))
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rot = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    np.testing.assert_allclose(_quat_mat(q2[3:]), _quat_mat(q[3:]) @ Rot, atol=1e-14)
    # both sides of the small-angle series branch agree with the closed form
    for th in (0.99e-6, 1.01e-6, 3e-9):
        got = m.integrate_pos(q, np.concatenate([np.zeros(3), th * ax]))[3:]
        w, v = q[3], q[4:7]
        ew, ev = np.cos(th / 2), np.sin(th / 2) * ax
        ref = np.concatenate([[w * ew - v @ ev], w * ev + ew * v + np.cross(v, ev)])
        np.testing.assert_allclose(got, ref / np.linalg.norm(ref), atol=2e-16)


@pytest.mark.parametrize("kind", ["motor", "position"])
def test_actuated_hinge_closed_form(orc, kind):
    """One hinge about the world z axis (COM at distance l on the link, gravity
    along the axis, so the bias force vanishes): the applied generalised force
    is gear u for a motor and kp (u - q) - kd v for a position servo, plus the
    joint damping -d v, and the acceleration is that force over the moment of
    inertia about the axis, Izz + m l^2."""
    m_, l, d, gear, kp, kd = 2.0, 0.3, 0.15, 1.7, 40.0, 1.3
    inertia = [0.01, 0.02, 0.03]
    scene = {"name": "hinge", "bodies": [{"parent": -1, "joint": "hinge", "pos": [0.0, 0.0, 0.0],
                                          "quat": [1.0, 0.0, 0.0, 0.0], "axis": [0.0, 0.0, 1.0], "mass": m_,
                                          "com": [l, 0.0, 0.0], "inertia": inertia, "damping": d}],
             "geoms": [], "pairs": [],
             "actuators": [{"type": kind, "body": 0, "gear": gear, "kp": kp, "kd": kd}],
             "options": W._options(), "qpos0": [0.0]}
    om = orc.OracleModel(scene)
    Jz = inertia[2] + m_ * l * l
    g = np.random.default_rng(21)
    for _ in range(5):
        q, v, u = g.uniform(-2, 2, 1), g.uniform(-3, 3, 1), g.uniform(-1, 1, 1)
        tau = gear * u[0] if kind == "motor" else kp * (u[0] - q[0]) - kd * v[0]
        tau -= d * v[0]
        np.testing.assert_allclose(om.applied(q, v, u), [tau], rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(om.rhs(q, v, u), [tau / Jz], rtol=1e-12, atol=1e-13)
