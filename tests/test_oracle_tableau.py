"""Pins of the oracle's Dormand-Prince 5(4) tableau (App. C.2 cites the method):
published coefficients, consistency, and the Runge-Kutta order conditions
(order 5 for the propagated weights b, order 4 for the embedded bhat)."""

import os
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    a = np.zeros((7, 7)); b = np.zeros(7); bh = np.zeros(7); c = np.zeros(7)
    for line in open(os.path.join(HERE, "golden", "dopri5_tableau.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "a":
            a[int(line[1]), int(line[2])] = float(Fraction(int(line[3]), int(line[4])))
        else:
            arr = {"b": b, "bhat": bh, "c": c}[line[0]]
            arr[int(line[1])] = float(Fraction(int(line[2]), int(line[3])))
    return a, b, bh, c


def _conditions(A, b, c):
    """Order conditions of explicit RK methods, rooted trees up to order 5."""
    Ac = A @ c
    Ac2 = A @ c ** 2
    AAc = A @ Ac
    return [
        (b.sum(), 1.0),
        (b @ c, 1 / 2),
        (b @ c ** 2, 1 / 3), (b @ Ac, 1 / 6),
        (b @ c ** 3, 1 / 4), (b @ (c * Ac), 1 / 8), (b @ Ac2, 1 / 12), (b @ AAc, 1 / 24),
        (b @ c ** 4, 1 / 5), (b @ (c ** 2 * Ac), 1 / 10), (b @ (c * Ac2), 1 / 15), (b @ (c * AAc), 1 / 30),
        (b @ Ac ** 2, 1 / 20), (b @ (A @ c ** 3), 1 / 20), (b @ (A @ (c * Ac)), 1 / 40), (b @ (A @ Ac2), 1 / 60),
        (b @ (A @ AAc), 1 / 120),
    ]


def test_tableau_matches_published_coefficients(orc):
    a, b, bh, c = orc.tableau()
    ga, gb, gbh, gc = _golden()
    np.testing.assert_allclose(a, ga, rtol=0, atol=1e-15)
    np.testing.assert_allclose(b, gb, rtol=0, atol=1e-15)
    np.testing.assert_allclose(bh, gbh, rtol=0, atol=1e-15)
    np.testing.assert_allclose(c, gc, rtol=0, atol=1e-15)


def test_row_sums_and_fsal(orc):
    a, b, bh, c = orc.tableau()
    np.testing.assert_allclose(a.sum(axis=1), c, atol=1e-14)
    np.testing.assert_allclose(a[6, :6], b[:6], atol=0)       # first same as last
    assert b[6] == 0.0
    assert np.all(np.triu(a) == 0.0)                          # explicit


def test_order_conditions(orc):
    a, b, bh, c = orc.tableau()
    for got, want in _conditions(a, b, c):
        assert abs(got - want) < 1e-14
    conds = _conditions(a, bh, c)
    for got, want in conds[:8]:                               # embedded method: order 4
        assert abs(got - want) < 1e-14
    assert max(abs(g - w) for g, w in conds[8:]) > 1e-6       # ... but not order 5


# ------------------------------------------------------------------ Tsitouras 5(4), semi-implicit Euler
def _golden_tsit5():
    a = np.zeros((7, 7)); e = np.zeros(7); c = np.zeros(7)
    for line in open(os.path.join(HERE, "golden", "tsit5_tableau.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "a":
            a[int(line[1]), int(line[2])] = float(line[3])
        else:
            {"e": e, "c": c}[line[0]][int(line[1])] = float(line[2])
    b = np.zeros(7); b[:6] = a[6, :6]
    return a, b, b - e, c


def test_tsit5_matches_published_coefficients(orc):
    t = orc.tableau_full("tsit5")
    ga, gb, gbh, gc = _golden_tsit5()
    assert t["S"] == 7
    np.testing.assert_array_equal(t["av"], ga)
    np.testing.assert_array_equal(t["aq"], ga)
    np.testing.assert_allclose(t["b"], gb, rtol=0, atol=1e-17)
    np.testing.assert_allclose(t["bhat"], gbh, rtol=0, atol=1e-17)
    np.testing.assert_array_equal(t["c"], gc)


def test_tsit5_order_conditions():
    """The published decimals satisfy every order-5 condition of b and every
    order-4 condition of bhat to rounding (and bhat is not of order 5)."""
    a, b, bh, c = _golden_tsit5()
    np.testing.assert_allclose(a.sum(axis=1), c, atol=1e-15)
    assert np.all(np.triu(a) == 0.0) and b[6] == 0.0
    for got, want in _conditions(a, b, c):
        assert abs(got - want) < 1e-14
    conds = _conditions(a, bh, c)
    for got, want in conds[:8]:
        assert abs(got - want) < 1e-14
    assert max(abs(g - w) for g, w in conds[8:]) > 1e-6


def test_semi_implicit_euler_coefficients(orc):
    """Semi-implicit Euler as a two-stage partitioned scheme: the velocity takes
    the stage-0 derivative, the position takes the NEW velocity (diagonal
    position coefficient), no error estimate."""
    t = orc.tableau_full("euler")
    assert t["S"] == 2
    assert t["av"][1, 0] == 1.0 and t["av"][1, 1] == 0.0
    assert t["aq"][1, 1] == 1.0 and t["aq"][1, 0] == 0.0
    np.testing.assert_array_equal(t["b"], t["bhat"])           # no embedded difference
