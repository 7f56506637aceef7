"""Embedded Runge-Kutta time integration of the magnetisation (and, when the
elastic term is on, of u and v), oracle version.

Test infrastructure only (see oracle/__init__.py).

The paper lists five embedded Runge-Kutta solvers with optional adaptive
steps, each with its convergence order and the order of its error estimate
(Methods, table of solvers; dynamic equation dm/dt = tau): Heun (2, 1),
Bogacki-Shampine (3, 2), Cash-Karp (5, 4), Fehlberg (5, 4) and
Dormand-Prince (5, 4).  The tableaux are the published ones (Heun's
method with the Euler estimate; Bogacki and Shampine, Appl. Math. Lett. 2,
321 (1989); Cash and Karp, ACM TOMS 16, 201 (1990); Fehlberg, NASA TR
R-315 (1969); Dormand and Prince, J. Comput. Appl. Math. 6, 19 (1980)),
used with local extrapolation: the higher-order solution is propagated.

Every method is run the same way: stages 2..s, then one evaluation at the
new (renormalised) solution, which is the first stage of the next step.
For the FSAL methods (Bogacki-Shampine, Dormand-Prince) that evaluation is
their last stage; for the others it is the extra evaluation every step
needs anyway.  So a step costs S field evaluations after the first (S = 6
for Dormand-Prince), and the error estimate sum_j (b_j - b*_j) k_j runs over
k_1 .. k_S+1 (the solution evaluation has weight b*_s only for FSAL
methods).

Readings of what the paper leaves open (shared with the CUDA path):
  * m is renormalised to unit length after every accepted step; the seventh
    stage (FSAL) is evaluated at the renormalised state;
  * err = dt * max over cells, components and sublattices of
    |sum_i (b_i - b*_i) k_i|, on the magnetisation only;
  * accept when err <= tol; dt <- dt * clamp(0.9 (tol/err)^(1/5), 0.2, 5),
    limited to [dt_min, dt_max]; a step at dt_min is always accepted;
  * a run of fixed duration shortens its last step to end on time.
"""
from fractions import Fraction as Fr

import numpy as np

from . import fields as _fields
from . import elastic as _elastic


def _method(a_rows, b, bstar, fsal, q):
    """Stage rows A[1..S] (row S = the solution weights b), the error weights
    E over k_1..k_S+1 and the controller exponent 1/(q+1) of an embedded
    tableau with s stages (FSAL: its last stage is evaluated at b)."""
    s = len(b)
    A = [[]] + [list(r) for r in a_rows]
    if fsal:
        assert list(A[-1]) == list(b[:-1]) and b[-1] == 0
        A = A[:s]
        S = s - 1
        E = [bj - bsj for bj, bsj in zip(b, bstar)]
    else:
        A = A[:s] + [list(b)]
        S = s
        E = [bj - bsj for bj, bsj in zip(b, bstar)] + [Fr(0)]
    return {"A": A, "b": list(b), "bstar": list(bstar), "S": S, "E": E, "exponent": 1.0 / (q + 1)}


METHODS = {
    "HEUN": _method([[Fr(1)]], [Fr(1, 2), Fr(1, 2)], [Fr(1), Fr(0)], False, 1),
    "BS23": _method([[Fr(1, 2)], [Fr(0), Fr(3, 4)], [Fr(2, 9), Fr(1, 3), Fr(4, 9)]],
                    [Fr(2, 9), Fr(1, 3), Fr(4, 9), Fr(0)], [Fr(7, 24), Fr(1, 4), Fr(1, 3), Fr(1, 8)], True, 2),
    "CASHKARP": _method([[Fr(1, 5)], [Fr(3, 40), Fr(9, 40)], [Fr(3, 10), Fr(-9, 10), Fr(6, 5)],
                         [Fr(-11, 54), Fr(5, 2), Fr(-70, 27), Fr(35, 27)],
                         [Fr(1631, 55296), Fr(175, 512), Fr(575, 13824), Fr(44275, 110592), Fr(253, 4096)]],
                        [Fr(37, 378), Fr(0), Fr(250, 621), Fr(125, 594), Fr(0), Fr(512, 1771)],
                        [Fr(2825, 27648), Fr(0), Fr(18575, 48384), Fr(13525, 55296), Fr(277, 14336), Fr(1, 4)],
                        False, 4),
    "RKF45": _method([[Fr(1, 4)], [Fr(3, 32), Fr(9, 32)], [Fr(1932, 2197), Fr(-7200, 2197), Fr(7296, 2197)],
                      [Fr(439, 216), Fr(-8), Fr(3680, 513), Fr(-845, 4104)],
                      [Fr(-8, 27), Fr(2), Fr(-3544, 2565), Fr(1859, 4104), Fr(-11, 40)]],
                     [Fr(16, 135), Fr(0), Fr(6656, 12825), Fr(28561, 56430), Fr(-9, 50), Fr(2, 55)],
                     [Fr(25, 216), Fr(0), Fr(1408, 2565), Fr(2197, 4104), Fr(-1, 5), Fr(0)], False, 4),
    "DP45": _method([[Fr(1, 5)], [Fr(3, 40), Fr(9, 40)], [Fr(44, 45), Fr(-56, 15), Fr(32, 9)],
                     [Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)],
                     [Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)],
                     [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)]],
                    [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84), Fr(0)],
                    [Fr(5179, 57600), Fr(0), Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200),
                     Fr(187, 2100), Fr(1, 40)], True, 4),
}

# Dormand-Prince, by name (the default method)
A = METHODS["DP45"]["A"]
C = [Fr(0), Fr(1, 5), Fr(3, 10), Fr(4, 5), Fr(8, 9), Fr(1), Fr(1)]
B5 = METHODS["DP45"]["b"]
B4 = METHODS["DP45"]["bstar"]
E = METHODS["DP45"]["E"]

SAFETY, GROW_MIN, GROW_MAX, EXPONENT = 0.9, 0.2, 5.0, 0.2   # EXPONENT: Dormand-Prince's 1/5


class State:
    """RK state: list of sublattice magnetisations, optional u and v."""

    def __init__(self, ms, u=None, v=None):
        self.ms = [np.asarray(m, dtype=np.float64) for m in ms]
        self.u = None if u is None else np.asarray(u, dtype=np.float64)
        self.v = None if v is None else np.asarray(v, dtype=np.float64)

    def parts(self):
        out = list(self.ms)
        if self.u is not None:
            out += [self.u, self.v]
        return out

    @classmethod
    def from_parts(cls, parts, n_sub, elastic):
        if elastic:
            return cls(parts[:n_sub], parts[n_sub], parts[n_sub + 1])
        return cls(parts[:n_sub])


def normalise(m):
    n = np.sqrt((m * m).sum(axis=0))
    return np.where(n > 0, m / np.where(n > 0, n, 1.0), 0.0)


class Oracle:
    """Right-hand side and embedded Runge-Kutta stepping for one problem
    (method: a key of METHODS, Dormand-Prince by default)."""

    def __init__(self, problem, noct=None, method="DP45"):
        self.p = problem
        self.m = METHODS[method]
        self.P = _fields.cell_params(problem)
        self.elastic = "ELASTIC" in problem.terms
        if "DEMAG" in problem.terms and noct is None:
            from .demag import tensor_octant
            noct = tensor_octant(problem.shape, problem.cell)
        self.noct = noct
        self.evals = 0

    def fields(self, st):
        return _fields.effective_fields(self.p, st.ms, st.u, self.noct, P=self.P)

    def rhs(self, st):
        """d/dt of every part of the state."""
        self.evals += 1
        Bs = self.fields(st)
        ks = _fields.torques(self.p, st.ms, Bs, self.P)
        if self.elastic:
            f = _elastic.total_force(self.p, self.P, st.ms, st.u, st.v)
            ks += [st.v.copy(), f / self.p.glob["RHO"]]
        return ks

    def _combine(self, y, ks, coefs, dt):
        out = []
        for i, base in enumerate(y):
            acc = base.copy()
            for c, k in zip(coefs, ks):
                if c != 0:
                    acc = acc + (dt * float(c)) * k[i]
            out.append(acc)
        return out

    def attempt(self, st, k1, dt):
        """One attempt from state `st` with first stage k1: the stages, the
        renormalised solution and its evaluation.  Returns (new state, the
        first stage of the next step, err)."""
        y = st.parts()
        ks = [k1]
        n_sub = self.p.n_sub
        A, E, S = self.m["A"], self.m["E"], self.m["S"]
        for i in range(1, S + 1):
            yi = self._combine(y, ks, A[i], dt)
            if i == S:
                for s in range(n_sub):
                    yi[s] = normalise(yi[s])
            ks.append(self.rhs(State.from_parts(yi, n_sub, self.elastic)))
        err = 0.0
        for s in range(n_sub):
            e = sum(float(E[j]) * ks[j][s] for j in range(S + 1) if E[j] != 0)
            mask = self.P["MS"][s] > 0
            if mask.any():
                err = max(err, float(np.abs(e)[:, mask].max()))
        err *= dt
        return State.from_parts(yi, n_sub, self.elastic), ks[S], err

    def run_fixed(self, st, dt, nsteps, callback=None):
        k1 = self.rhs(st)
        for n in range(nsteps):
            st, k1, _ = self.attempt(st, k1, dt)
            if callback is not None:
                callback(n + 1, st)
        return st

    def run_adaptive(self, st, dt, tol, duration, dt_min=1e-18, dt_max=1e-11,
                     max_attempts=10 ** 7):
        """Adaptive DP45 until t = duration.  Returns (state, stats)."""
        t = 0.0
        k1 = self.rhs(st)
        accepted = rejected = 0
        while t < duration and accepted + rejected < max_attempts:
            h = min(dt, duration - t)
            new, k7, err = self.attempt(st, k1, h)
            ok = err <= tol or h <= dt_min
            fac = GROW_MAX if err == 0 else SAFETY * (tol / err) ** self.m["exponent"]
            fac = min(max(fac, GROW_MIN), GROW_MAX)
            if ok:
                st, k1, t = new, k7, t + h
                accepted += 1
            else:
                rejected += 1
            dt = min(max(h * fac, dt_min), dt_max)
        return st, dict(t=t, dt=dt, accepted=accepted, rejected=rejected, evals=self.evals)
