"""Scene descriptions and seeded synthetic inputs for the four rollout workloads.

This module holds input data only (geometry, masses, solver parameters and
seeded random initial states / controls).  It performs none of the method's
arithmetic, imports nothing else from this package, and is the one module that
both the CUDA path and the CPU oracle are fed from.

Scenes are plain dicts:

  bodies    : parent (-1 = world, parents precede children), joint ('free' |
              'hinge'), pos, quat (w, x, y, z) of the body frame in the parent
              frame, axis (hinge, body frame), mass, com (body frame), inertia
              (principal moments about the COM, body axes), damping
  geoms     : type ('sphere' | 'capsule' | 'box'), body, pos, quat, size
              (sphere: radius; capsule: radius, half length along local x;
              box: half extents)
  pairs     : geom1, geom2 (-1 = ground plane z = 0), condim (1 frictionless,
              3 pyramidal friction with 4 edges), mu
  actuators : type ('motor' | 'position'), body (hinge), gear, kp, kd
  options   : gravity, solref (t_c, phi_d), solimp (d_o, d_w, width,
              midpoint, power), solimp_cfd (d_c, d_0, w_c, m_c, p_c),
              softplus width
  qpos0     : reference configuration

Solver parameters follow the paper: solref time constant 0.002 s with damping
ratio 1 (the stiff setting), solimp (0, 0.95, 0.001, 0.5, 2) (Sec. 3 object
tosses, App. E.1), solimp-CFD tuple order (d_c, d_0, w_c, m_c, p_c) (Sec. 4).
"""

from __future__ import annotations

import math

import numpy as np

GRAVITY = (0.0, 0.0, -9.81)
SOLREF = (0.002, 1.0)
SOLIMP = (0.0, 0.95, 0.001, 0.5, 2.0)
SOLIMP_CFD = (0.0, 0.0, 0.05, 1.0, 4.0)
# Contacts from distance (Sec. 4, App. E.3): contact impedance starting at
# d_o = 0.1 and the CFD spline (d_c, d_0, w_c, m_c, p_c) that continues it
# from r = 0 up to the taper width w_c (0.05 m for the 0.1 m cubes here).
CFD_SOLIMP = (0.1, 0.95, 0.001, 0.5, 2.0)
CFD_SOLIMP_CFD = (0.0, 0.1, 0.05, 1.0, 4.0)
CFD_OPTIONS = {"solimp": CFD_SOLIMP, "solimp_cfd": CFD_SOLIMP_CFD}
SOFTPLUS = 1e-3
IDQ = (1.0, 0.0, 0.0, 0.0)


def _options(solimp=SOLIMP, solimp_cfd=SOLIMP_CFD, softplus=SOFTPLUS, gravity=GRAVITY, solref=SOLREF):
    return {"gravity": list(gravity), "solref": list(solref), "solimp": list(solimp),
            "solimp_cfd": list(solimp_cfd), "softplus": float(softplus)}


def _free_body(mass, inertia, parent=-1):
    return {"parent": parent, "joint": "free", "pos": [0.0, 0.0, 0.0], "quat": list(IDQ), "axis": [0.0, 0.0, 1.0],
            "mass": mass, "com": [0.0, 0.0, 0.0], "inertia": list(inertia), "damping": 0.0}


def _hinge_body(parent, pos, axis, mass, com, inertia, damping=0.0, quat=IDQ):
    return {"parent": parent, "joint": "hinge", "pos": list(pos), "quat": list(quat), "axis": list(axis),
            "mass": mass, "com": list(com), "inertia": list(inertia), "damping": damping}


def _geom(gtype, body, size, pos=(0.0, 0.0, 0.0), quat=IDQ):
    s = list(size) + [0.0] * (3 - len(size))
    return {"type": gtype, "body": body, "pos": list(pos), "quat": list(quat), "size": s}


def _pair(g1, g2, condim, mu):
    return {"geom1": g1, "geom2": g2, "condim": condim, "mu": mu}


def sphere_inertia(m, r):
    return [0.4 * m * r * r] * 3


def box_inertia(m, hx, hy, hz):
    a, b, c = 2 * hx, 2 * hy, 2 * hz
    return [m * (b * b + c * c) / 12.0, m * (a * a + c * c) / 12.0, m * (a * a + b * b) / 12.0]


def rod_inertia(m, r, length):
    """Solid cylinder along the local x axis (used for capsule links)."""
    return [0.5 * m * r * r, m * (3 * r * r + length * length) / 12.0, m * (3 * r * r + length * length) / 12.0]


# --------------------------------------------------------------------------- scenes
def ball_scene(radius=0.1, mass=1.0, **opt):
    """Free sphere (6 dof, frictionless) above the ground plane."""
    return {"name": "ball",
            "bodies": [_free_body(mass, sphere_inertia(mass, radius))],
            "geoms": [_geom("sphere", 0, [radius])],
            "pairs": [_pair(0, -1, 1, 0.0)],
            "actuators": [],
            "options": _options(**opt),
            "qpos0": [0.0, 0.0, radius, 1.0, 0.0, 0.0, 0.0]}


def box_scene(half=0.05, mass=1.0, mu=1.0, **opt):
    """Free cube on the ground plane, pyramidal friction, 8 vertex contacts."""
    return {"name": "box",
            "bodies": [_free_body(mass, box_inertia(mass, half, half, half))],
            "geoms": [_geom("box", 0, [half, half, half])],
            "pairs": [_pair(0, -1, 3, mu)],
            "actuators": [],
            "options": _options(**opt),
            "qpos0": [0.0, 0.0, half, 1.0, 0.0, 0.0, 0.0]}


CHAIN_LINKS = 7
CHAIN_LINK = 0.3
CHAIN_RADIUS = 0.025
CHAIN_HEIGHT = 0.05
CUBE_START = (1.85, 0.25, 0.05)
CUBE_GOAL = (2.0, 0.5, 0.05)


def chain_cube_scene(mu=1.0, **opt):
    """Fixed-base planar arm of 7 z-axis hinges with capsule links (0.3 m, 1 kg,
    joint damping 0.1, torque motors) and a free 0.1 m cube on the plane."""
    bodies, geoms, pairs, acts = [], [], [], []
    for i in range(CHAIN_LINKS):
        parent = i - 1
        pos = (0.0, 0.0, CHAIN_HEIGHT) if i == 0 else (CHAIN_LINK, 0.0, 0.0)
        bodies.append(_hinge_body(parent, pos, (0, 0, 1), 1.0, (CHAIN_LINK / 2, 0, 0),
                                  rod_inertia(1.0, CHAIN_RADIUS, CHAIN_LINK), damping=0.1))
        geoms.append(_geom("capsule", i, [CHAIN_RADIUS, CHAIN_LINK / 2], pos=(CHAIN_LINK / 2, 0, 0)))
        acts.append({"type": "motor", "body": i, "gear": 1.0, "kp": 0.0, "kd": 0.0})
    cube = len(bodies)
    bodies.append(_free_body(1.0, box_inertia(1.0, 0.05, 0.05, 0.05)))
    gcube = len(geoms)
    geoms.append(_geom("box", cube, [0.05, 0.05, 0.05]))
    pairs.append(_pair(gcube, -1, 3, mu))
    for i in range(CHAIN_LINKS):
        pairs.append(_pair(i, gcube, 3, mu))
    for i in range(CHAIN_LINKS):
        pairs.append(_pair(i, -1, 3, mu))
    qpos0 = [0.0] * CHAIN_LINKS + list(CUBE_START) + list(IDQ)
    return {"name": "chain_cube", "bodies": bodies, "geoms": geoms, "pairs": pairs, "actuators": acts,
            "options": _options(**opt), "qpos0": qpos0}


QUAD_TORSO = (0.2, 0.1, 0.05)
QUAD_LINK = 0.2
QUAD_LINK_RADIUS = 0.02
QUAD_FOOT = 0.025
QUAD_HEIGHT = 0.45


def quadruped_scene(mu=0.8, kp=50.0, kd=1.0, **opt):
    """Box torso (0.4 x 0.2 x 0.1 m, 8 kg, free joint) with four legs of three
    hinges (abduction about x, hip and knee about y), 0.2 m capsule links of
    0.5 kg, sphere feet on the plane, PD position servos on all 12 hinges."""
    bodies = [_free_body(8.0, box_inertia(8.0, *QUAD_TORSO))]
    geoms = [_geom("box", 0, list(QUAD_TORSO))]
    pairs, acts = [], []
    # links lie along the body -z axis: transverse moments about x and y
    link_inertia = [0.5 * (3 * QUAD_LINK_RADIUS ** 2 + QUAD_LINK ** 2) / 12.0] * 2 + [0.5 * 0.5 * QUAD_LINK_RADIUS ** 2]
    for sx in (1.0, -1.0):
        for sy in (1.0, -1.0):
            hip = (sx * 0.18, sy * 0.1, 0.0)
            ab = len(bodies)
            bodies.append(_hinge_body(0, hip, (1, 0, 0), 0.5, (0, 0, 0), sphere_inertia(0.5, 0.03)))
            th = len(bodies)
            bodies.append(_hinge_body(ab, (0, 0, 0), (0, 1, 0), 0.5, (0, 0, -QUAD_LINK / 2), link_inertia))
            # capsule along the link: local x of the geom is rotated onto -z
            qdown = (math.cos(math.pi / 4), 0.0, math.sin(math.pi / 4), 0.0)
            geoms.append(_geom("capsule", th, [QUAD_LINK_RADIUS, QUAD_LINK / 2], pos=(0, 0, -QUAD_LINK / 2), quat=qdown))
            sh = len(bodies)
            bodies.append(_hinge_body(th, (0, 0, -QUAD_LINK), (0, 1, 0), 0.5, (0, 0, -QUAD_LINK / 2), link_inertia))
            geoms.append(_geom("capsule", sh, [QUAD_LINK_RADIUS, QUAD_LINK / 2], pos=(0, 0, -QUAD_LINK / 2), quat=qdown))
            foot = len(geoms)
            geoms.append(_geom("sphere", sh, [QUAD_FOOT], pos=(0, 0, -QUAD_LINK)))
            pairs.append(_pair(foot, -1, 3, mu))
            for b in (ab, th, sh):
                acts.append({"type": "position", "body": b, "gear": 1.0, "kp": kp, "kd": kd})
    qpos0 = [0.0, 0.0, QUAD_HEIGHT] + list(IDQ) + [0.0] * 12
    return {"name": "quadruped", "bodies": bodies, "geoms": geoms, "pairs": pairs, "actuators": acts,
            "options": _options(**opt), "qpos0": qpos0}


def scene_dims(scene):
    nq = sum(7 if b["joint"] == "free" else 1 for b in scene["bodies"])
    nv = sum(6 if b["joint"] == "free" else 1 for b in scene["bodies"])
    return nq, nv, len(scene["actuators"])


# --------------------------------------------------------------------------- inputs
def _rng(seed):
    return np.random.Generator(np.random.Philox(seed))


def _yaw_quat(yaw):
    return np.stack([np.cos(yaw / 2), np.zeros_like(yaw), np.zeros_like(yaw), np.sin(yaw / 2)], axis=-1)


def ball_inputs(B=16, seed=1001, T=1.0):
    """Ball drops: centre height 0.1 + U[0.5, 1.5] m, v0 ~ N(0, 0.5^2) per axis,
    identity orientation, zero angular velocity."""
    g = _rng(seed)
    x0 = np.zeros((B, 13))
    x0[:, 0:2] = 0.0
    x0[:, 2] = 0.1 + g.uniform(0.5, 1.5, B)
    x0[:, 3] = 1.0
    x0[:, 7:10] = g.normal(0.0, 0.5, (B, 3))
    return {"x0": x0, "ctrl": None, "T": np.full(B, T), "NI": 1, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3,
            "max_steps": 20000}


def box_push_inputs(B=4096, seed=1002, T=1.0):
    """Box pushes: cube resting on the plane (bottom face at z = 0), yaw ~
    U[-pi, pi], planar push speed ~ U[0, 2] m/s along a direction ~ U[0, 2 pi)."""
    g = _rng(seed)
    x0 = np.zeros((B, 13))
    x0[:, 2] = 0.05
    x0[:, 3:7] = _yaw_quat(g.uniform(-math.pi, math.pi, B))
    speed = g.uniform(0.0, 2.0, B)
    th = g.uniform(0.0, 2 * math.pi, B)
    x0[:, 7] = speed * np.cos(th)
    x0[:, 8] = speed * np.sin(th)
    return {"x0": x0, "ctrl": None, "T": np.full(B, T), "NI": 1, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3,
            "max_steps": 20000}


def chain_inputs(B=16384, seed=1003, T=2.0, NI=50):
    """Arm at rest straight along +x with the cube resting at its start;
    torques u ~ N(0, 1) N m per hinge and control interval."""
    g = _rng(seed)
    scene = chain_cube_scene()
    nq, nv, nu = scene_dims(scene)
    x0 = np.zeros((B, nq + nv))
    x0[:, :nq] = np.asarray(scene["qpos0"])
    ctrl = g.normal(0.0, 1.0, (B, NI, nu))
    return {"x0": x0, "ctrl": ctrl, "T": np.full(B, T), "NI": NI, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3,
            "max_steps": 20000}


def quadruped_inputs(B=8192, seed=1004):
    """Quadruped released at torso height 0.45 m with zero velocity; PD joint
    targets ~ U[-0.3, 0.3] rad held over the horizon T ~ U[0.5, 3] s."""
    g = _rng(seed)
    scene = quadruped_scene()
    nq, nv, nu = scene_dims(scene)
    x0 = np.zeros((B, nq + nv))
    x0[:, :nq] = np.asarray(scene["qpos0"])
    ctrl = g.uniform(-0.3, 0.3, (B, 1, nu))
    T = g.uniform(0.5, 3.0, B)
    return {"x0": x0, "ctrl": ctrl, "T": T, "NI": 1, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3, "max_steps": 20000}


def arm_tilt_scene(tilt=0.015, **opt):
    """The arm + cube with the arm's base (and so every hinge axis) tilted by
    `tilt` rad about the world y axis: the outstretched arm descends towards
    its tip, which starts 6.5 mm into the plane, so the capsule-plane pairs
    (two end slots per link) carry contact forces, with friction against the
    links' sliding, as the arm swings."""
    sc = chain_cube_scene(**opt)
    sc["bodies"][0]["quat"] = [math.cos(tilt / 2), 0.0, math.sin(tilt / 2), 0.0]
    sc["name"] = "arm_tilt"
    return sc


def arm_tilt_inputs(B=64, seed=1009, T=0.5, NI=10):
    """Tilted arm at rest along +x, torques ~ N(0, 1) N m per hinge and interval."""
    g = _rng(seed)
    scene = arm_tilt_scene()
    nq, nv, nu = scene_dims(scene)
    x0 = np.zeros((B, nq + nv))
    x0[:, :nq] = np.asarray(scene["qpos0"])
    ctrl = g.normal(0.0, 1.0, (B, NI, nu))
    return {"x0": x0, "ctrl": ctrl, "T": np.full(B, T), "NI": NI, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3,
            "max_steps": 20000}


def billiard_scene(radius=0.05, mass=0.2, condim=1, mu=0.0, **opt):
    """Two free balls and no gravity, the ball-ball contact only (the billiard
    toy of Sec. 4 and App. C.4 with the table contacts and gravity off)."""
    opt.setdefault("gravity", (0.0, 0.0, 0.0))
    bodies = [_free_body(mass, sphere_inertia(mass, radius)), _free_body(mass, sphere_inertia(mass, radius))]
    geoms = [_geom("sphere", 0, [radius]), _geom("sphere", 1, [radius])]
    return {"name": "billiard", "bodies": bodies, "geoms": geoms, "pairs": [_pair(0, 1, condim, mu)],
            "actuators": [], "options": _options(**opt),
            "qpos0": [0.0, 0.0, 0.0] + list(IDQ) + [0.3, 0.0, 0.0] + list(IDQ)}


def billiard_inputs(B=16, seed=1007, T=0.5):
    """Cue ball at the origin shot along +x at U[0.5, 1.5] m/s towards a ball
    at rest 0.3 m away with a lateral offset U[-0.08, 0.08] m (glancing to
    head-on hits, some misses)."""
    g = _rng(seed)
    x0 = np.zeros((B, 26))
    x0[:, 3] = 1.0
    x0[:, 7] = 0.3
    x0[:, 8] = g.uniform(-0.08, 0.08, B)
    x0[:, 10] = 1.0
    x0[:, 14] = g.uniform(0.5, 1.5, B)
    return {"x0": x0, "ctrl": None, "T": np.full(B, T), "NI": 1, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3,
            "max_steps": 20000}


def capsules_scene(mu=0.5, **opt):
    """A free capsule (radius 0.03, half length 0.1), a free sphere (0.04) and
    a second free capsule, no gravity: capsule-capsule, sphere-capsule and
    sphere-sphere-free pairs with pyramidal friction."""
    opt.setdefault("gravity", (0.0, 0.0, 0.0))
    cap_i = rod_inertia(0.3, 0.03, 0.2)
    bodies = [_free_body(0.3, cap_i), _free_body(0.2, sphere_inertia(0.2, 0.04)), _free_body(0.3, cap_i)]
    geoms = [_geom("capsule", 0, [0.03, 0.1]), _geom("sphere", 1, [0.04]), _geom("capsule", 2, [0.03, 0.1])]
    pairs = [_pair(0, 2, 3, mu), _pair(1, 0, 3, mu), _pair(2, 1, 3, mu)]
    return {"name": "capsules", "bodies": bodies, "geoms": geoms, "pairs": pairs, "actuators": [],
            "options": _options(**opt),
            "qpos0": [0.0, 0.0, 0.0] + list(IDQ) + [0.0, 0.2, 0.0] + list(IDQ) + [0.0, 0.0, 0.2] + list(IDQ)}


def capsules_inputs(B=16, seed=1008, T=0.4):
    """The three bodies thrown together: positions jittered N(0, 0.01) m around
    separated centres, random orientations, velocities towards the centroid
    (0.8 m/s) plus N(0, 0.1), angular velocities N(0, 2)."""
    g = _rng(seed)
    x0 = np.zeros((B, 39))
    centres = np.array([[0.0, 0.0, 0.0], [0.15, 0.2, 0.0], [0.0, 0.05, 0.25]])
    for b in range(3):
        qa, va = 7 * b, 21 + 6 * b
        x0[:, qa:qa + 3] = centres[b] + g.normal(0.0, 0.01, (B, 3))
        qq = g.normal(size=(B, 4))
        x0[:, qa + 3:qa + 7] = qq / np.linalg.norm(qq, axis=1, keepdims=True)
    cen = (x0[:, 0:3] + x0[:, 7:10] + x0[:, 14:17]) / 3
    for b in range(3):
        qa, va = 7 * b, 21 + 6 * b
        d = cen - x0[:, qa:qa + 3]
        d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-9)
        x0[:, va:va + 3] = 0.8 * d + g.normal(0.0, 0.1, (B, 3))
        x0[:, va + 3:va + 6] = g.normal(0.0, 2.0, (B, 3))
    return {"x0": x0, "ctrl": None, "T": np.full(B, T), "NI": 1, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3,
            "max_steps": 20000}


def toss_scene():
    """Cube toss of the integrator comparison (Sec. 3, Fig. 12): the 0.1 m,
    1 kg cube with the toss contact setting solref (0.005 s, 1)."""
    sc = box_scene(solref=(0.005, 1.0))
    sc["name"] = "toss"
    return sc


def toss_inputs(B=2048, seed=1006, T=1.0):
    """Cube tosses as in the paper's integrator comparison (a cube thrown
    onto the plane at v_x = -2 m/s): centre height 0.2 + U[0, 0.05] m, small
    random tilt (quaternion (1, N(0, 0.05)^3), normalised), initial velocity
    (-2 + N(0, 0.05), N(0, 0.05), 0) m/s, no spin.  Loss: the final x position
    (toss distance), gradient w.r.t. the initial velocity."""
    g = _rng(seed)
    x0 = np.zeros((B, 13))
    x0[:, 2] = 0.2 + g.uniform(0.0, 0.05, B)
    qq = np.concatenate([np.ones((B, 1)), g.normal(0.0, 0.05, (B, 3))], axis=1)
    x0[:, 3:7] = qq / np.linalg.norm(qq, axis=1, keepdims=True)
    x0[:, 7] = -2.0 + g.normal(0.0, 0.05, B)
    x0[:, 8] = g.normal(0.0, 0.05, B)
    return {"x0": x0, "ctrl": None, "T": np.full(B, T), "NI": 1, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3,
            "max_steps": 20000}


def chain_goal():
    return np.asarray(CUBE_GOAL)


SCENES = {"ball": ball_scene, "box": box_scene, "chain_cube": chain_cube_scene, "quadruped": quadruped_scene,
          "toss": toss_scene, "billiard": billiard_scene, "capsules": capsules_scene, "arm_tilt": arm_tilt_scene}
INPUTS = {"ball": ball_inputs, "box": box_push_inputs, "chain_cube": chain_inputs, "quadruped": quadruped_inputs,
          "toss": toss_inputs, "billiard": billiard_inputs, "capsules": capsules_inputs, "arm_tilt": arm_tilt_inputs}
