"""Pins of the oracle's constraint solve and right-hand-side derivative:
closed-form single-row solution, brute-force enumeration of active sets,
optimality (KKT) conditions, and central differences of F and F~."""

import itertools

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W


def _quat(ax, th):
    ax = np.asarray(ax, float) / np.linalg.norm(ax)
    return np.concatenate([[np.cos(th / 2)], np.sin(th / 2) * ax])


def test_single_row_closed_form(orc):
    """One frictionless row: f = max(0, a_ref - J a0) / (A + R), A = J M^-1 J^T."""
    sc = W.ball_scene()
    m = orc.OracleModel(sc)
    tc, damp = sc["options"]["solref"]
    dw = sc["options"]["solimp"][1]
    for z, vz in [(0.0998, -1.0), (0.0996, 0.3), (0.0991, 0.0), (0.0999, 2.0)]:
        q = np.array([0.1, 0.2, z, 1, 0, 0, 0])
        v = np.array([0.5, -0.2, vz, 1.0, 2.0, -1.0])
        r = z - 0.1
        d = m.impedance(r)
        A = 1.0                                 # J M^-1 J^T for a unit mass through its COM
        R = A * (1 - d) / d                     # the model's A_hat equals 1/m here
        aref = -2 / (dw * tc) * vz - d / (dw ** 2 * tc ** 2 * damp ** 2) * r
        a0z = -9.81
        f = max(0.0, aref - a0z) / (A + R)
        a = m.rhs(q, v)
        assert abs(a[2] - (a0z + f)) < 1e-12 * max(1.0, abs(f))
        np.testing.assert_allclose(a[[0, 1, 3, 4, 5]], 0.0, atol=1e-12)   # round-off of world-origin lever arms


def _problem(m, q, v, u=None, cfd=False):
    M = m.mass(q)
    rhs0 = m.applied(q, v, u) - m.bias(q, v)
    J, aref, D, _ = m.rows(q, v, cfd)
    return M, rhs0, J, aref, D


def _brute_force(M, rhs0, J, aref, D):
    nr = len(aref)
    sols = []
    for mask in itertools.product([False, True], repeat=nr):
        S = np.array(mask)
        H = M + (J[S].T * D[S]) @ J[S]
        b = rhs0 + J[S].T @ (D[S] * aref[S])
        a = np.linalg.solve(H, b)
        z = J @ a - aref
        if np.all(z[S] < 1e-12 * (1 + np.abs(aref).max())) and np.all(z[~S] >= -1e-12 * (1 + np.abs(aref).max())):
            sols.append(a)
    return sols


@pytest.mark.parametrize("seed", range(6))
def test_multi_row_solve_matches_active_set_enumeration(orc, seed):
    """Tilted box with two or three vertices below the plane (8 or 12 pyramid
    rows): the oracle's Newton result equals the unique self-consistent active
    set found by enumerating all 2^nr candidate sets."""
    m = orc.OracleModel(W.box_scene())
    g = np.random.default_rng(seed)
    for _ in range(50):
        quat = _quat(g.normal(size=3), g.uniform(0.3, 1.2))
        q = np.concatenate([[0, 0, 0.0], quat])
        ct = m.contacts(q)
        r = np.sort(ct[:, 0])
        k = 2 + seed % 2
        q[2] = -(r[k - 1] + r[k]) / 2            # exactly k vertices below the plane
        ct = m.contacts(q)
        if (ct[:, 0] < 0).sum() == k and ct[:, 0][ct[:, 0] < 0].min() > -0.002:
            break
    v = g.normal(scale=0.5, size=6)
    M, rhs0, J, aref, D = _problem(m, q, v)
    assert len(aref) == 4 * k
    sols = _brute_force(M, rhs0, J, aref, D)
    assert len(sols) == 1
    a, info = m.rhs(q, v, detail=True)
    np.testing.assert_allclose(a, sols[0], rtol=0, atol=1e-10 * (1 + np.abs(sols[0]).max()))
    # KKT: zero gradient of the primal cost, forces non-negative and complementary
    a0 = np.linalg.solve(M, rhs0)
    z = J @ a - aref
    grad = M @ (a - a0) + J.T @ (D * np.minimum(z, 0))
    assert np.abs(grad).max() < 1e-9 * (1 + np.abs(rhs0).max())
    f = info["f"]
    assert np.all(f >= 0)
    np.testing.assert_allclose(f, -D * np.minimum(z, 0), atol=1e-9 * (1 + f.max()))


def test_solution_minimises_primal_cost(orc):
    m = orc.OracleModel(W.box_scene())
    g = np.random.default_rng(11)
    q = np.concatenate([[0.1, 0.0, 0.0495], _quat([0.1, 0.2, 1.0], 0.4)])
    v = np.array([0.8, -0.3, -0.2, 0.5, -1.0, 0.3])
    M, rhs0, J, aref, D = _problem(m, q, v)
    a0 = np.linalg.solve(M, rhs0)

    def cost(a):
        z = np.minimum(J @ a - aref, 0)
        return 0.5 * (a - a0) @ M @ (a - a0) + 0.5 * (D * z * z).sum()

    a = m.rhs(q, v)
    c = cost(a)
    for _ in range(200):
        assert cost(a + g.normal(scale=1e-3, size=6)) >= c - 1e-12 * (1 + abs(c))


def _fd_rhs(m, q, v, u, cfd, eps=1e-7):
    nq, nv, nu = m.nq, m.nv, m.nu
    Jq = np.zeros((nv, nq)); Jv = np.zeros((nv, nv)); Ju = np.zeros((nv, nu))
    for i in range(nq):
        e = np.zeros(nq); e[i] = eps
        Jq[:, i] = (m.rhs(q + e, v, u, cfd) - m.rhs(q - e, v, u, cfd)) / (2 * eps)
    for i in range(nv):
        e = np.zeros(nv); e[i] = eps
        Jv[:, i] = (m.rhs(q, v + e, u, cfd) - m.rhs(q, v - e, u, cfd)) / (2 * eps)
    for i in range(nu):
        e = np.zeros(nu); e[i] = eps
        Ju[:, i] = (m.rhs(q, v, u + e, cfd) - m.rhs(q, v, u - e, cfd)) / (2 * eps)
    return Jq, Jv, Ju


CFD_OPT = dict(W.CFD_OPTIONS)


@pytest.mark.parametrize("cfd", [False, True])
@pytest.mark.parametrize("name", ["box", "chain_cube", "quadruped"])
def test_rhs_jacobian_matches_central_differences(orc, name, cfd):
    """Forward-mode derivatives of F (and of F~ with contacts from distance)
    equal central differences at states away from active-set switches."""
    sc = W.SCENES[name](**CFD_OPT)
    m = orc.OracleModel(sc)
    g = np.random.default_rng(12)
    q = np.array(sc["qpos0"], float)
    u = g.normal(size=m.nu) if m.nu else np.zeros(0)
    if name == "box":
        q[2] = 0.0496
        q[3:7] = _quat([0.05, 0.02, 1.0], 0.3)
    elif name == "chain_cube":
        q[:7] = [0.1, -0.2, 0.15, 0.1, -0.1, 0.05, 0.3]
        q[7:10] = [1.5, 0.33, 0.0497]    # cube touching the arm within the CFD width
    else:
        q[2] = 0.42
        q[7:] = g.uniform(-0.2, 0.2, 12)
    v = g.normal(scale=0.2, size=m.nv)
    _, info = m.rhs(q, v, u, cfd, detail=True)
    assert info["nr"] > 0
    Jq, Jv, Ju = m.rhs_jacobian(q, v, u, cfd)
    Fq, Fv, Fu = _fd_rhs(m, q, v, u, cfd)
    scale = 1 + max(np.abs(Fq).max(), np.abs(Fv).max())
    np.testing.assert_allclose(Jq, Fq, atol=2e-5 * scale)
    np.testing.assert_allclose(Jv, Fv, atol=2e-5 * scale)
    if m.nu:
        np.testing.assert_allclose(Ju, Fu, atol=2e-5 * scale)


def test_cfd_rhs_adds_forces_only_at_positive_distance(orc):
    """F~ differs from F only through contacts with 0 <= r < w_c (and the softplus
    position term); far from the plane both are free fall."""
    sc = W.ball_scene(**CFD_OPT)
    m = orc.OracleModel(sc)
    v = np.zeros(6)
    far = np.array([0, 0, 0.2, 1, 0, 0, 0])
    np.testing.assert_allclose(m.rhs(far, v, cfd=True), m.rhs(far, v), atol=0)
    near = np.array([0, 0, 0.12, 1, 0, 0, 0])
    assert m.rhs(near, v)[2] == -9.81
    assert m.rhs(near, v, cfd=True)[2] > -9.81
