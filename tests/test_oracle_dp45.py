"""Pins of the oracle's Dormand-Prince tableau and stepper: the Butcher order
conditions (exact rational arithmetic), consistency c_i = sum_j a_ij,
|m| = 1 after every accepted step, and the adaptive controller keeping every
accepted error below the tolerance while landing exactly on the end time."""
from fractions import Fraction as Fr

import numpy as np

from inputs import config_small
from oracle import dp45
from oracle.dp45 import Oracle, State


def _order_conditions(b, A, c, order):
    s = len(b)
    a = [[A[i][j] if j < len(A[i]) else Fr(0) for j in range(s)] for i in range(s)]

    def ac(v):
        return [sum(a[i][j] * v[j] for j in range(s)) for i in range(s)]

    def dot(u, v):
        return sum(x * y for x, y in zip(u, v))

    def mul(u, v):
        return [x * y for x, y in zip(u, v)]

    one = [Fr(1)] * s
    c2 = mul(c, c)
    c3 = mul(c2, c)
    conds = [(dot(b, one), Fr(1)), (dot(b, c), Fr(1, 2)),
             (dot(b, c2), Fr(1, 3)), (dot(b, ac(c)), Fr(1, 6)),
             (dot(b, c3), Fr(1, 4)), (dot(b, mul(c, ac(c))), Fr(1, 8)),
             (dot(b, ac(c2)), Fr(1, 12)), (dot(b, ac(ac(c))), Fr(1, 24))]
    if order >= 5:
        conds += [(dot(b, mul(c3, c)), Fr(1, 5)), (dot(b, mul(c2, ac(c))), Fr(1, 10)),
                  (dot(b, mul(ac(c), ac(c))), Fr(1, 20)), (dot(b, mul(c, ac(c2))), Fr(1, 15)),
                  (dot(b, mul(c, ac(ac(c)))), Fr(1, 30)), (dot(b, ac(c3)), Fr(1, 20)),
                  (dot(b, ac(mul(c, ac(c)))), Fr(1, 40)), (dot(b, ac(ac(c2))), Fr(1, 60)),
                  (dot(b, ac(ac(ac(c)))), Fr(1, 120))]
    return conds


def test_row_sums_equal_nodes():
    for i, row in enumerate(dp45.A):
        assert sum(row, Fr(0)) == dp45.C[i]


def test_fifth_order_solution_satisfies_all_17_conditions():
    for got, want in _order_conditions(dp45.B5, dp45.A, dp45.C, 5):
        assert got == want


def test_embedded_solution_is_fourth_but_not_fifth_order():
    conds = _order_conditions(dp45.B4, dp45.A, dp45.C, 5)
    assert all(g == w for g, w in conds[:8])
    assert any(g != w for g, w in conds[8:])


def test_fsal_last_row_is_b5():
    assert list(dp45.A[6]) + [Fr(0)] == list(dp45.B5)


def test_unit_length_after_steps():
    w = config_small((6, 5, 2), (2e-9, 2e-9, 2e-9), 4)
    o = Oracle(w.problem)
    st = o.run_fixed(State(w.m0), 5e-14, 10)
    assert np.abs(np.sqrt((st.ms[0] ** 2).sum(axis=0)) - 1).max() < 4e-16


def test_adaptive_controller():
    w = config_small((6, 5, 2), (2e-9, 2e-9, 2e-9), 9)
    o = Oracle(w.problem)
    tol = 1e-5
    errs = []
    orig = o.attempt

    def spy(st, k1, dt):
        new, k7, err = orig(st, k1, dt)
        errs.append(err)
        return new, k7, err

    o.attempt = spy
    st, stats = o.run_adaptive(State(w.m0), 1e-15, tol, 3e-12)
    assert stats["t"] == 3e-12
    assert stats["accepted"] > 3
    assert sum(e <= tol for e in errs) >= stats["accepted"]
    assert stats["evals"] == 1 + 6 * (stats["accepted"] + stats["rejected"])
