"""Pins of the oracle's elastodynamics and magnetoelastic coupling: the exact
dispersion of the 4th-order stencils in the bulk, exactness on linear fields
(uniform strain gives the closed-form magnetoelastic field at every cell),
the magnetoelastic force as the divergence of the magnetoelastic stress,
the divergence as the negative transpose of the gradient, the absence of
growing modes of the discrete elastic operator, and energy conservation
without viscosity."""
import numpy as np
import pytest

from inputs import Problem
from oracle import elastic, fields


def _problem(shape, h=2e-9, terms=("ELASTIC",), n_sub=1):
    p = Problem(shape, (h, h, h), n_sub, frozenset(terms))
    p.set("MS", 4e5).set("B1", -1e7).set("B2", -0.6e7)
    p.glob.update(C11=2.5e11, C12=1.5e11, C44=1e11, RHO=7e3, ETA=0.0)
    return p


def _symbol(k, h):
    """The 4th-order first-derivative stencil acting on exp(ikx) multiplies it
    by i s(k), s = (8 sin kh - sin 2kh) / (6h)."""
    return (8 * np.sin(k * h) - np.sin(2 * k * h)) / (6 * h)


@pytest.mark.parametrize("axis", [0, 1])
def test_bulk_plane_wave_dispersion(axis):
    n, h = 48, 2e-9
    shape = [1, 1, 1]
    shape[axis] = n
    p = _problem(tuple(shape), h)
    k = 2 * np.pi * 5 / (n * h)
    x = np.arange(n) * h
    g = p.glob
    s2 = _symbol(k, h) ** 2
    for comp, c in ((axis, g["C11"]), ((axis + 1) % 3, g["C44"])):
        u = np.zeros((3, n))
        u[comp] = 1e-11 * np.sin(k * x)
        u = u.reshape((3,) + tuple(shape[::-1]))
        f = elastic.elastic_force(u, np.zeros_like(u), p).reshape(3, n)
        ref = -c * s2 * u.reshape(3, n)[comp]
        sl = slice(4, n - 4)
        assert np.abs(f[comp, sl] - ref[sl]).max() <= 1e-10 * np.abs(ref).max()


def test_uniform_strain_gives_closed_form_mel_field():
    shape = (7, 6, 5)
    p = _problem(shape, terms=("MEL",))
    h = p.cell[0]
    E = np.array([[1e-3, 2e-4, -3e-4], [2e-4, -5e-4, 1e-4], [-3e-4, 1e-4, 7e-4]])
    z, y, x = np.meshgrid(*(np.arange(n) * h for n in shape[::-1]), indexing="ij")
    r = np.stack([x, y, z])
    u = np.einsum("ij,jzyx->izyx", E, r)          # u_i = E_ij x_j, strain = sym(E)
    eps = elastic.strain(u, p.cell)
    S = 0.5 * (E + E.T)
    want = [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]
    for a, w in zip(eps, want):
        assert np.abs(a - w).max() < 1e-15
    rng = np.random.default_rng(5)
    m = rng.normal(size=(3,) + shape[::-1])
    m /= np.linalg.norm(m, axis=0)
    P = fields.cell_params(p)
    B = fields.mel_field(p, P, 0, m, eps)
    B1, B2, Ms = -1e7, -0.6e7, 4e5
    ref = -(2 / Ms) * np.stack([
        B1 * S[0, 0] * m[0] + B2 * (S[0, 1] * m[1] + S[0, 2] * m[2]),
        B1 * S[1, 1] * m[1] + B2 * (S[0, 1] * m[0] + S[1, 2] * m[2]),
        B1 * S[2, 2] * m[2] + B2 * (S[0, 2] * m[0] + S[1, 2] * m[1])])
    assert np.abs(B - ref).max() < 1e-9 * np.abs(ref).max()


def test_mel_force_is_divergence_of_mel_stress():
    """For m linear in x the finite differences are exact, and the force of
    the paper's formula must equal d_x of sigma_mel (B1 m_x^2, B2 m_x m_y,
    B2 m_x m_z) computed by hand: (2 B1 m_x b_x, B2 (b_x m_y + m_x b_y),
    B2 (b_x m_z + m_x b_z))."""
    n, h, B1, B2 = 9, 2e-9, -1e7, -0.6e7
    x = np.arange(n) * h
    a = np.array([0.3, -0.2, 0.5])
    b = np.array([1.1e7, 2.3e7, -0.7e7])
    m = (a[:, None] + b[:, None] * x[None, :]).reshape(3, 1, 1, n)
    f = elastic.mel_force(m, B1, B2, (h, h, h)).reshape(3, n)
    mm = m.reshape(3, n)
    ref = np.stack([2 * B1 * mm[0] * b[0],
                    B2 * (b[0] * mm[1] + mm[0] * b[1]),
                    B2 * (b[0] * mm[2] + mm[0] * b[2])])
    assert np.abs(f - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 13])
def test_divergence_is_minus_transpose_of_gradient(n):
    """sum_j a_j (div S)_j = -sum_i (grad a)_i S_i for any a, S."""
    rng = np.random.default_rng(n)
    a = rng.normal(size=(1, 1, n))
    S = rng.normal(size=(1, 1, n))
    lhs = (a * elastic.div1(S, -1, 0.7)).sum()
    rhs = -(elastic.d1(a, -1, 0.7) * S).sum()
    assert abs(lhs - rhs) < 1e-13 * (np.abs(a).sum() * np.abs(S).sum() + 1)


def test_traction_free_natural_condition():
    """A uniform stress that violates sigma.n = 0 pushes only the cells within
    reach of the edge closure (the outer four layers)."""
    S = np.full((1, 1, 10), 3.0)
    f = elastic.div1(S, -1, 1.0).ravel()
    assert np.all(np.abs(f[4:-4]) < 1e-15)
    assert f[0] > 0 and f[-1] < 0


@pytest.mark.parametrize("shape", [(6, 5, 1), (9, 4, 1), (5, 4, 3)])
def test_no_growing_modes(shape):
    """u'' = F u / rho is stable only if every eigenvalue of F is real and
    non-positive; checked on the assembled operator."""
    p = _problem(shape)
    n = 3 * np.prod(shape)
    F = np.empty((n, n))
    z = np.zeros((3,) + shape[::-1])
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        F[:, j] = elastic.elastic_force(e.reshape(z.shape), z, p).ravel()
    ev = np.linalg.eigvals(F)
    scale = np.abs(ev).max()
    assert ev.real.max() < 1e-9 * scale
    assert np.abs(ev.imag).max() < 1e-6 * scale


def test_energy_conserved_without_viscosity():
    from oracle.dp45 import Oracle, State
    shape = (24, 20, 1)
    p = _problem(shape)
    z = np.zeros((3,) + shape[::-1])
    yy, xx = np.meshgrid(np.arange(20), np.arange(24), indexing="ij")
    bump = np.exp(-((xx - 12) ** 2 + (yy - 10) ** 2) / 8.0)
    u = z.copy()
    u[0, 0] = 1e-11 * bump
    u[1, 0] = -0.5e-11 * bump
    m = np.zeros_like(z)
    m[2] = 1.0
    o = Oracle(p)
    st = State([m], u, z.copy())
    E0 = sum(elastic.elastic_energy(p, st.u, st.v))
    st = o.run_fixed(st, 2e-14, 100)
    E1 = sum(elastic.elastic_energy(p, st.u, st.v))
    assert abs(E1 / E0 - 1) < 1e-9


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 9, 17])
def test_gradient_rows_exact_on_polynomials(n):
    """Every row of the gradient scheme is a consistent derivative of the
    order its stencil has, which fixes its coefficients: all rows (one-sided
    edges, second-order central next to them, fourth-order bulk) differentiate
    linear fields exactly, every row but those of n = 2 quadratics, and the
    bulk rows quartics too (n >= 5).  A wrong coefficient or a dropped term in
    any row fails one of these."""
    h = 1.5
    x = np.arange(n, dtype=np.float64) * h + 0.7

    def d(f):
        return elastic.d1(f[None, None, :], -1, h)[0, 0]
    assert np.allclose(d(3.0 - 2.0 * x), -2.0, rtol=0, atol=1e-12)
    if n >= 3:
        assert np.allclose(d(1.0 + 0.5 * x - 0.25 * x ** 2), 0.5 - 0.5 * x, rtol=0, atol=1e-11)
    if n >= 5:
        bulk = slice(2, n - 2)
        for p in (3, 4):
            f, df = x ** p, p * x ** (p - 1)
            assert np.allclose(d(f)[bulk], df[bulk], rtol=1e-12, atol=1e-9), p
        # and the bulk rows are not exact at degree 5 (the stencil is 4th order, not higher)
        f5 = x ** 5
        assert np.abs(d(f5)[bulk] - 5 * x[bulk] ** 4).max() > 1e-6
