"""Dormand-Prince RK45 time integration of the magnetisation (and, when the
elastic term is on, of u and v), oracle version.

Test infrastructure only (see oracle/__init__.py).

The paper lists Dormand-Prince (RK45, order 5 with an order-4 error
estimate) among its embedded Runge-Kutta solvers with optional adaptive
steps (Methods, table of solvers; dynamic equation dm/dt = tau).  The
tableau is the published one of Dormand and Prince, J. Comput. Appl. Math.
6, 19 (1980), used with local extrapolation (the order-5 solution is
propagated) and FSAL (the last stage is the first of the next step).

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

A = [
    [],
    [Fr(1, 5)],
    [Fr(3, 40), Fr(9, 40)],
    [Fr(44, 45), Fr(-56, 15), Fr(32, 9)],
    [Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)],
    [Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)],
    [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)],
]
C = [Fr(0), Fr(1, 5), Fr(3, 10), Fr(4, 5), Fr(8, 9), Fr(1), Fr(1)]
B5 = [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84), Fr(0)]
B4 = [Fr(5179, 57600), Fr(0), Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200),
      Fr(187, 2100), Fr(1, 40)]
E = [b5 - b4 for b5, b4 in zip(B5, B4)]

SAFETY, GROW_MIN, GROW_MAX, EXPONENT = 0.9, 0.2, 5.0, 0.2


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
    """Right-hand side and DP45 stepping for one problem."""

    def __init__(self, problem, noct=None):
        self.p = problem
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
        """One DP45 attempt from state `st` with first stage k1.
        Returns (new state, k7, err)."""
        y = st.parts()
        ks = [k1]
        n_sub = self.p.n_sub
        for i in range(1, 7):
            yi = self._combine(y, ks, A[i], dt)
            if i == 6:
                for s in range(n_sub):
                    yi[s] = normalise(yi[s])
            ks.append(self.rhs(State.from_parts(yi, n_sub, self.elastic)))
        err = 0.0
        for s in range(n_sub):
            e = sum(float(E[j]) * ks[j][s] for j in range(7) if E[j] != 0)
            mask = self.P["MS"][s] > 0
            if mask.any():
                err = max(err, float(np.abs(e)[:, mask].max()))
        err *= dt
        return State.from_parts(yi, n_sub, self.elastic), ks[6], err

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
            fac = GROW_MAX if err == 0 else SAFETY * (tol / err) ** EXPONENT
            fac = min(max(fac, GROW_MIN), GROW_MAX)
            if ok:
                st, k1, t = new, k7, t + h
                accepted += 1
            else:
                rejected += 1
            dt = min(max(h * fac, dt_min), dt_max)
        return st, dict(t=t, dt=dt, accepted=accepted, rejected=rejected, evals=self.evals)
