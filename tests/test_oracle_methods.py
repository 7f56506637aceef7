"""Pins of the oracle's five embedded Runge-Kutta methods against the
convergence and error-estimate orders the paper's table of solvers prints
(Methods): Heun (2, 1), Bogacki-Shampine (3, 2), Cash-Karp (5, 4), Fehlberg
(5, 4), Dormand-Prince (5, 4).

* the Butcher order conditions (exact rationals): the propagated weights b
  satisfy every condition through the convergence order, the embedded b*
  through the error order but not the next;
* the observed global order on the macrospin closed form;
* the order of the error estimate: err ~ dt^(q+1)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from inputs import GAMMA, Problem
from oracle.dp45 import METHODS, Oracle, State

ORDERS = {"HEUN": (2, 1), "BS23": (3, 2), "CASHKARP": (5, 4), "RKF45": (5, 4), "DP45": (5, 4)}


def _conditions_by_order(b, a):
    """[[(value, required), ...] for order 1, 2, ...] up to order 5."""
    s = len(b)
    A = [[a[i][j] if j < len(a[i]) else Fr(0) for j in range(s)] for i in range(s)]
    c = [sum(A[i], Fr(0)) for i in range(s)]

    def ac(v):
        return [sum(A[i][j] * v[j] for j in range(s)) for i in range(s)]

    def dot(u, v):
        return sum(x * y for x, y in zip(u, v))

    def mul(u, v):
        return [x * y for x, y in zip(u, v)]

    one = [Fr(1)] * s
    c2, c3 = mul(c, c), mul(mul(c, c), c)
    return [
        [(dot(b, one), Fr(1))],
        [(dot(b, c), Fr(1, 2))],
        [(dot(b, c2), Fr(1, 3)), (dot(b, ac(c)), Fr(1, 6))],
        [(dot(b, c3), Fr(1, 4)), (dot(b, mul(c, ac(c))), Fr(1, 8)), (dot(b, ac(c2)), Fr(1, 12)),
         (dot(b, ac(ac(c))), Fr(1, 24))],
        [(dot(b, mul(c3, c)), Fr(1, 5)), (dot(b, mul(c2, ac(c))), Fr(1, 10)),
         (dot(b, mul(ac(c), ac(c))), Fr(1, 20)), (dot(b, mul(c, ac(c2))), Fr(1, 15)),
         (dot(b, mul(c, ac(ac(c)))), Fr(1, 30)), (dot(b, ac(c3)), Fr(1, 20)),
         (dot(b, ac(mul(c, ac(c)))), Fr(1, 40)), (dot(b, ac(ac(c2))), Fr(1, 60)),
         (dot(b, ac(ac(ac(c)))), Fr(1, 120))],
    ]


def _stage_rows(m):
    """The s x s stage matrix of a method (rows 0..s-1) from its A rows."""
    s = len(m["b"])
    return [list(r) for r in m["A"][:s]] + [[]] * max(0, s - len(m["A"]))


def _order_of(weights, rows):
    conds = _conditions_by_order(weights, rows)
    q = 0
    for group in conds:
        if all(v == r for v, r in group):
            q += 1
        else:
            break
    return q


@pytest.mark.parametrize("name", sorted(ORDERS))
def test_butcher_orders_match_the_printed_table(name):
    m = METHODS[name]
    p, q = ORDERS[name]
    rows = _stage_rows(m)
    assert _order_of(m["b"], rows) == p
    assert _order_of(m["bstar"], rows) == q


@pytest.mark.parametrize("name", sorted(ORDERS))
def test_solution_row_and_error_weights(name):
    m = METHODS[name]
    S, b = m["S"], list(m["b"])
    row = list(m["A"][S])                     # the solution row: b (without an FSAL stage's zero)
    assert row + [Fr(0)] * (len(b) - len(row)) == b
    assert sum(m["E"], Fr(0)) == 0            # both weight sets sum to 1
    assert m["exponent"] == 1.0 / (ORDERS[name][1] + 1)


def _macrospin(method, dt, nsteps, alpha=0.1, B=1.0, th0=0.5):
    p = Problem((1, 1, 1), (1e-9,) * 3, 1, frozenset({"ZEEMAN"}))
    p.set("MS", 8e5).set("ALPHA", alpha).set("B_EXT", (0.0, 0.0, B))
    m0 = np.array([np.sin(th0), 0.0, np.cos(th0)]).reshape(3, 1, 1, 1)
    return Oracle(p, method=method).run_fixed(State([m0]), dt, nsteps).ms[0].ravel()


def _exact(t, alpha=0.1, B=1.0, th0=0.5):
    g = GAMMA / (1 + alpha ** 2)
    th = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-alpha * g * B * t))
    ph = g * B * t
    return np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])


@pytest.mark.parametrize("name", sorted(ORDERS))
def test_observed_convergence_order(name):
    p, _ = ORDERS[name]
    T = 40e-12
    ns = (40, 80, 160) if p >= 5 else (160, 320, 640)
    errs = [np.abs(_macrospin(name, T / n, n) - _exact(T)).max() for n in ns]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - p) < 0.6), (errs, slopes)


@pytest.mark.parametrize("name", sorted(ORDERS))
def test_error_estimate_order(name):
    """One step's estimate scales as dt^(q+1) for small dt."""
    _, q = ORDERS[name]
    p = Problem((1, 1, 1), (1e-9,) * 3, 1, frozenset({"ZEEMAN"}))
    p.set("MS", 8e5).set("ALPHA", 0.1).set("B_EXT", (0.0, 0.0, 1.0))
    m0 = np.array([np.sin(0.5), 0.0, np.cos(0.5)]).reshape(3, 1, 1, 1)
    o = Oracle(p, method=name)
    st = State([m0])
    k1 = o.rhs(st)
    errs = [o.attempt(st, k1, dt)[2] for dt in (4e-13, 2e-13, 1e-13)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - (q + 1)) < 0.35), (errs, slopes)
