"""Pins of the oracle's step-size control: the RMS error norm, the PID
controller of the paper (P = 0.2, I = 0.4, D = 0; App. B, Fig. 12 caption),
its rejection rule, clips and floors, and the contact parameters printed in
the paper (tests/golden/paper_parameters.txt).

The controller is pinned by behaviour, not by retyping its formula:

* on a problem whose error norm depends on the step size alone, a PI
  controller settles where 0.9 err^(-I/5) = 1, i.e. at err = 0.9^(5/I)
  (a swapped exponent or a sign error on the err_prev term moves it);
* a least-squares fit of log(h_n+1 / h_n) on the logs of the last three
  error norms recovers the safety factor and P, I, D of the Soederlind PID
  form h_n+1 = h_n 0.9 err_n^-(P+I+D)/5 err_n-1^(P+2D)/5 err_n-2^(-D/5);
* a retried step after one rejection lands at err = 0.9^5 (the retry factor
  0.9 err^(-1/5) scales an h^5 error by 0.9^5 / err).

The test problem is a torque-free symmetric top in zero gravity with the
absolute tolerance alone: its body-frame angular velocity rotates about the
symmetry axis, every error component is equivariant under that rotation, so
the error norm of a step depends on h only.
"""

import os

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def read_paper_parameters():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out[line[0]] = tuple(float(x) for x in line[1:])
    return out


def _top(orc):
    sc = W.box_scene(gravity=(0.0, 0.0, 0.0))
    sc["bodies"][0]["inertia"] = [0.1, 0.1, 0.3]
    sc["pairs"] = []
    m = orc.OracleModel(sc)
    x0 = np.array([0, 0, 1.0, 1, 0, 0, 0, 0, 0, 0, 1.0, 0.5, 4.0])
    return m, x0


TOL = dict(rtol=0.0, atol=1e-8)


def _accepted_errors(m, x0, hlog):
    """Error norm of each accepted step, recomputed from the replayed states
    (the top is autonomous: one step from the previous state is the replay)."""
    x, errs = x0.copy(), []
    for h in hlog:
        errs.append(m.step_error(x, h, **TOL))
        x, _ = m.replay(x, [h], T=1e3)
    return np.array(errs)


# ----------------------------------------------------------------- error norm
def _norm_case(m):
    """Chain + cube (7 hinges, then a free cube: nq = 14, nv = 13)."""
    q0 = np.full(m.nq, 7.0); q1 = np.full(m.nq, 7.0)
    v0 = np.full(m.nv, 7.0); v1 = np.full(m.nv, 7.0)
    q0[10:14] = q1[10:14] = 0.5          # cube quaternion (0.5, 0.5, 0.5, 0.5)
    return q0, q1, v0, v1


def test_error_norm_absolute_only(orc):
    """atol alone: err = sqrt(sum e^2 / (2 nv))."""
    m = orc.OracleModel(W.chain_cube_scene())
    q0, q1, v0, v1 = _norm_case(m)
    e = np.zeros(2 * m.nv)
    assert m.error_norm(q0, v0, q1, v1, e, rtol=0.0, atol=1.0) == 0.0
    e[:] = 0.3
    assert abs(m.error_norm(q0, v0, q1, v1, e, rtol=0.0, atol=1.0) - 0.3) < 1e-15
    e[:] = 0.0
    e[17] = 2.0
    assert abs(m.error_norm(q0, v0, q1, v1, e, rtol=0.0, atol=1.0) - 2.0 / np.sqrt(26)) < 1e-15


def test_error_norm_relative_scales(orc):
    """rtol alone: each component is scaled by the larger magnitude of the two
    states; the three rotation components of a free joint by 1 (not by a
    quaternion entry); hinges, translations and velocities by their
    coordinate.  Five components at exactly their scale give sqrt(5 / 26)."""
    m = orc.OracleModel(W.chain_cube_scene())
    q0, q1, v0, v1 = _norm_case(m)
    e = np.zeros(2 * m.nv)
    q0[2], q1[2], e[2] = -3.0, 1.0, 3.0           # hinge 2: max(|-3|, |1|)
    q0[8], q1[8], e[8] = 2.0, -4.0, 4.0           # cube y: the end state is larger
    e[11] = 1.0                                   # cube rotation (dof 11): magnitude 1
    v0[4], v1[4], e[13 + 4] = 0.5, -2.0, 2.0      # hinge 4 velocity
    v0[10], v1[10], e[13 + 10] = 3.0, 1.0, 3.0    # cube angular velocity x: the start state is larger
    got = m.error_norm(q0, v0, q1, v1, e, rtol=1.0, atol=0.0)
    assert abs(got - np.sqrt(5.0 / 26.0)) < 1e-15


def test_error_norm_mixed_tolerances_add(orc):
    """scale = atol + rtol max(|y_n|, |y_n+1|) (a sum, not a max of the two)."""
    m = orc.OracleModel(W.chain_cube_scene())
    q0, q1, v0, v1 = _norm_case(m)
    e = np.zeros(2 * m.nv)
    q0[9], q1[9], e[9] = 2.0, 1.0, 1.0            # 0.5 + 0.25 * 2 = 1
    got = m.error_norm(q0, v0, q1, v1, e, rtol=0.25, atol=0.5)
    assert abs(got - np.sqrt(1.0 / 26.0)) < 1e-15


# ----------------------------------------------------------------- controller
def test_error_depends_on_step_size_alone(orc):
    """Premise of the controller pins: the top's step error is a function of h."""
    m, x0 = _top(orc)
    x1 = x0.copy()
    c, s = np.cos(0.7), np.sin(0.7)                   # w_xy rotated about the symmetry axis
    x1[10:12] = [c * x0[10] - s * x0[11], s * x0[10] + c * x0[11]]
    x1[3:7] = [np.cos(0.3), np.sin(0.3) * 0.6, 0.0, np.sin(0.3) * 0.8]   # another orientation
    for h in (1e-2, 1.3e-2):                           # near the operating point (err ~ 0.1 .. 0.4)
        e0, e1 = m.step_error(x0, h, **TOL), m.step_error(x1, h, **TOL)
        assert abs(e0 - e1) <= 1e-7 * e0                # rounding of the embedded difference


def test_pi_controller_fixed_point(orc):
    """Accepted error norms settle at 0.9^(5/I) with the paper's I = 0.4."""
    I = read_paper_parameters()["pid"][1]
    m, x0 = _top(orc)
    r = m.rollout(x0, T=1.0, h0=5e-3, **TOL)
    assert r["status"] == 0 and r["nrej"] == 0
    errs = _accepted_errors(m, x0, r["hlog"][:-1])           # the last step is clamped to T
    np.testing.assert_allclose(errs[-10:], 0.9 ** (5.0 / I), rtol=1e-7)
    assert abs(0.9 ** (5.0 / I) - 0.2679361841) < 1e-9


def test_pid_gains_recovered_from_the_transient(orc):
    """Fit log(h_n+1 / h_n) = log(s) + c1 log err_n + c2 log err_n-1 + c3 log err_n-2
    over the transient from h0 = 5 ms: the fit is exact and gives the safety
    factor 0.9 and the paper's P, I, D."""
    P, I, D = read_paper_parameters()["pid"]
    m, x0 = _top(orc)
    r = m.rollout(x0, T=1.0, h0=5e-3, **TOL)
    hl = r["hlog"]
    le = np.log(_accepted_errors(m, x0, hl[:30]))
    lh = np.log(hl[:31])
    n = np.arange(2, 29)
    X = np.stack([np.ones(n.size), le[n], le[n - 1], le[n - 2]], axis=1)
    y = lh[n + 1] - lh[n]
    c, res, rank, _ = np.linalg.lstsq(X, y, rcond=None)
    assert rank == 4
    assert np.abs(X @ c - y).max() < 1e-9
    Dg = -5.0 * c[3]
    Pg = 5.0 * c[2] - 2.0 * Dg
    Ig = -5.0 * c[1] - Pg - Dg
    assert abs(np.exp(c[0]) - 0.9) < 1e-8
    assert abs(Pg - P) < 1e-8 and abs(Ig - I) < 1e-8 and abs(Dg - D) < 1e-8


def test_rejected_step_retry_lands_at_0_9_to_the_5th(orc):
    """One rejection: the retry factor 0.9 err^(-1/5) puts the retried step at
    err = 0.9^5 (h^5 law; 0.2 % for these step sizes)."""
    m, x0 = _top(orc)
    for h0 in (0.02, 0.03):
        assert 1.0 < m.step_error(x0, h0, **TOL) < (0.9 / 0.2) ** 5
        r = m.rollout(x0, T=1.0, h0=h0, **TOL)
        assert r["nrej"] == 1
        assert abs(m.step_error(x0, r["hlog"][0], **TOL) - 0.9 ** 5) < 2e-3


def test_rejection_factor_is_clipped_at_0_2(orc):
    """Above err = (0.9 / 0.2)^5 the retry factor is 0.2: from h0 = 0.1 s
    (err ~ 9e3) the first retry is 0.02 s, rejected again, and the run
    continues as one started at 0.02 s."""
    m, x0 = _top(orc)
    assert m.step_error(x0, 0.1, **TOL) > (0.9 / 0.2) ** 5
    r = m.rollout(x0, T=1.0, h0=0.1, **TOL)
    r2 = m.rollout(x0, T=1.0, h0=0.02, **TOL)
    assert r["nrej"] == 2 and r2["nrej"] == 1
    np.testing.assert_allclose(r["hlog"][:20], r2["hlog"][:20], rtol=1e-8)   # 0.1 * 0.2 != 0.02 by one ulp


def test_growth_clip_and_error_floor(orc):
    """From h0 = 1 us the first error norm (~1e-14) is below the 1e-10 floor:
    the factor 0.9 (1e-10)^-0.12 = 14.3 is clipped to 10; the second step has
    both its error and the previous one at the floor: 0.9 (1e-10)^(-0.12 + 0.04)."""
    m, x0 = _top(orc)
    r = m.rollout(x0, T=1.0, h0=1e-6, **TOL)
    hl = r["hlog"]
    errs = _accepted_errors(m, x0, hl[:2])
    assert errs.max() < 1e-10
    assert hl[1] == 10.0 * hl[0]
    assert abs(hl[2] / hl[1] - 0.9 * 1e-10 ** (-0.08)) < 1e-12


# ----------------------------------------------------------------- printed parameters
def test_workload_parameters_are_the_papers():
    """The contact parameters the workloads use are the ones the paper prints.
    solref (0.002 s, 1) is the workload specification's stiff setting, not a
    paper value; the CFD taper width w_c is 0.05 m for the 0.1 m cubes of the
    test scenes (the paper's MPC scene uses 1 m) and is not compared."""
    p = read_paper_parameters()
    assert tuple(W.SOLIMP) == p["solimp_toss"]
    assert tuple(W.CFD_SOLIMP) == p["solimp_mpc_cfd"]
    cfd = p["solimp_cfd_mpc"]
    assert (W.CFD_SOLIMP_CFD[0], W.CFD_SOLIMP_CFD[1], W.CFD_SOLIMP_CFD[3], W.CFD_SOLIMP_CFD[4]) == \
        (cfd[0], cfd[1], cfd[3], cfd[4])
    # continuity at r = 0: the CFD spline starts at the contact impedance d_o
    assert W.CFD_SOLIMP_CFD[1] == W.CFD_SOLIMP[0]
    assert W.SOLIMP_CFD[1] == W.SOLIMP[0]
    assert p["solref_toss"][1] == W.SOLREF[1]


def test_oracle_impedance_uses_the_printed_solimp(orc):
    """The oracle's impedance at |r| >= width is d_w and at r = 0 is d_o, for the
    printed solimp tuples (toss and MPC-with-CFD)."""
    p = read_paper_parameters()
    for key in ("solimp_toss", "solimp_mpc_cfd"):
        d_o, d_w, width = p[key][:3]
        m = orc.OracleModel(W.ball_scene(solimp=p[key]))
        assert abs(m.impedance(-2 * width) - d_w) < 1e-15
        assert abs(m.impedance(0.0) - d_o) < 1e-15
