"""Pins of the oracle's demag tensor and demag field against results that do
not come from the oracle's own formulas: the exact self factor of a cube,
trace identities, parity, the point-dipole limit, the additivity of the
tensor over a block of cells, an independent surface-charge integral for a
prism's self factor, an independent Gauss-Legendre integral of the dipole
kernel, and the direct O(N^2) sum of the definition."""
from math import pi

import numpy as np
import pytest
from scipy import integrate

from inputs import MU0
from oracle import demag


def _tensor(offset, cell):
    X, Y, Z = (np.array([float(o)]) for o in offset)
    return demag.cell_tensor(X, Y, Z, cell)[:, 0]


def _full(N6):
    xx, yy, zz, xy, xz, yz = N6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


# -- self terms ------------------------------------------------------------
def test_cube_self_factor_is_one_third():
    N = _tensor((0, 0, 0), (1e-9, 1e-9, 1e-9))
    assert np.allclose(N[:3], 1.0 / 3.0, rtol=0, atol=1e-14)
    assert np.allclose(N[3:], 0.0, atol=1e-15)


@pytest.mark.parametrize("cell", [(2e-9, 2e-9, 1e-9), (1e-9, 3e-9, 0.5e-9), (4e-9, 1e-9, 7e-9)])
def test_self_trace_is_one(cell):
    N = _tensor((0, 0, 0), cell)
    assert abs(N[:3].sum() - 1.0) < 1e-13


def _surface_charge_nzz(a, b, c):
    """Self factor N_zz of an a x b x c prism from the energy of its two
    charged faces: N_zz = (I(0) - I(c)) / (2 pi a b c) with
    I(h) = 4 int_0^a (a-u) [b asinh(b/s) - sqrt(b^2+s^2) + s] du,
    s = sqrt(u^2 + h^2) (the face-face Coulomb integral, inner integral done
    in closed form)."""
    def I(h):
        def f(u):
            s = np.hypot(u, h)
            return (a - u) * (b * np.arcsinh(b / s) - np.hypot(b, s) + s)
        val, _ = integrate.quad(f, 0.0, a, limit=400, epsabs=0, epsrel=1e-13)
        return 4.0 * val
    return (I(0.0) - I(c)) / (2.0 * pi * a * b * c)


@pytest.mark.parametrize("dims", [(1.0, 1.0, 1.0), (2.0, 2.0, 1.0), (3.0, 1.0, 0.5),
                                  (10.0, 10.0, 1.0), (1.0, 2.0, 5.0)])
def test_self_factor_matches_surface_charge_integral(dims):
    a, b, c = dims
    N = _tensor((0, 0, 0), dims)
    ref = _surface_charge_nzz(a, b, c)
    assert abs(N[2] - ref) < 1e-10, (N[2], ref)


# -- identities off the diagonal -------------------------------------------
OFFSETS = [(1, 0, 0), (1, 1, 0), (1, 1, 1), (2, -1, 3), (-3, 4, -2), (7, 2, 1),
           (9, 5, 3), (12, 1, 0), (-15, 10, 4), (30, -2, 7), (80, 40, 3)]


@pytest.mark.parametrize("cell", [(1.0, 1.0, 1.0), (2.0, 2.0, 1.0), (1.0, 3.0, 2.0)])
def test_trace_zero_off_self(cell):
    for o in OFFSETS:
        r = tuple(oi * ci for oi, ci in zip(o, cell))
        N = _tensor(r, cell)
        scale = np.abs(N).max()
        assert abs(N[:3].sum()) <= 2e-9 * scale, (o, N)


def test_parity():
    cell = (2.0, 1.5, 1.0)
    for o in OFFSETS:
        r = np.array([oi * ci for oi, ci in zip(o, cell)])
        N = _tensor(r, cell)
        for flip in ((-1, 1, 1), (1, -1, 1), (1, 1, -1)):
            Nf = _tensor(r * np.array(flip), cell)
            for comp, odd in enumerate(demag.ODD):
                sign = np.prod([f for f, od in zip(flip, odd) if od]) if any(odd) else 1
                assert abs(Nf[comp] - sign * N[comp]) <= 3e-9 * np.abs(N).max()


@pytest.mark.parametrize("cell,ratio", [((1.0, 1.0, 1.0), 16.0), ((2.0, 1.0, 1.0), 4.0)])
def test_point_dipole_limit(cell, ratio):
    """N(r) -> -(V/4 pi)(3 rr - I)/r^3.  The first correction is
    (1/2) sum_i E[s_i^2] d_i^2 of the dipole kernel; for a cube it is a
    Laplacian of a harmonic function and vanishes, so the error falls as
    (D/r)^4 for a cube and as (D/r)^2 otherwise."""
    errs = []
    V = cell[0] * cell[1] * cell[2]
    for scale in (10.0, 20.0, 40.0, 80.0):
        r = np.array([0.8, 0.5, 0.3]) * scale
        N = _full(_tensor(r, cell))
        rn = np.linalg.norm(r)
        rh = r / rn
        dip = -(V / (4 * pi)) * (3 * np.outer(rh, rh) - np.eye(3)) / rn ** 3
        errs.append(np.abs(N - dip).max() / np.abs(dip).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios / ratio - 1) < 0.1), errs


def _gl_tensor(r, cell, n=12):
    """N(r) = V E_s[-d_a d_b 1/(4 pi |r+s|)], s triangular per axis, by
    Gauss-Legendre quadrature on each half of [-D, D] (independent of the
    Newell formula and of the expansion)."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    pts, wts = [], []
    for D in cell:
        p = np.concatenate([-D / 2 + xg * D / 2, D / 2 + xg * D / 2])
        w = np.concatenate([wg * D / 2, wg * D / 2]) * (1 - np.abs(p) / D) / D
        pts.append(p)
        wts.append(w)
    sx, sy, sz = np.meshgrid(*pts, indexing="ij")
    W = np.einsum("i,j,k->ijk", *wts)
    x = r[0] + sx
    y = r[1] + sy
    z = r[2] + sz
    R2 = x * x + y * y + z * z
    R5 = R2 ** 2.5
    comp = {0: x, 1: y, 2: z}
    V = cell[0] * cell[1] * cell[2]
    out = []
    for a, b in demag.PAIRS:
        K = -(3 * comp[a] * comp[b] - (R2 if a == b else 0.0)) / (4 * pi * R5)
        out.append(V * (W * K).sum())
    return np.array(out)


@pytest.mark.parametrize("cell", [(1.0, 1.0, 1.0), (2.0, 2.0, 1.0)])
def test_tensor_matches_independent_quadrature(cell):
    for o in [(3, 0, 0), (4, 2, 1), (6, 5, 0), (5, 4, 3), (9, 3, 2), (10, 1, 1),
              (12, 3, 1), (15, 10, 4), (30, 0, 0), (25, 25, 5)]:
        r = np.array([oi * ci for oi, ci in zip(o, cell)], dtype=float)
        N = _tensor(r, cell)
        ref = _gl_tensor(r, cell)
        err = np.abs(N - ref).max() / np.abs(ref).max()
        assert err < 3e-9, (o, err)


def test_cutoff_agreement_newell_vs_asymptotic():
    """On the cutoff shell the two formulas agree to a few 1e-9 relative."""
    worst = 0.0
    for cell in [(1.0, 1.0, 1.0), (2.0, 2.0, 1.0), (2.0, 1.0, 1.5)]:
        L = max(cell)
        for d in [(1, 0, 0), (0.8, 0.6, 0), (0.6, 0.6, 0.53), (0.3, 0.4, 0.866)]:
            r = np.array(d) / np.linalg.norm(d) * demag.RC * L
            X, Y, Z = (np.array([v]) for v in r)
            Nn = demag.newell_tensor(X, Y, Z, cell)[:, 0]
            Na = demag.asymptotic_tensor(X, Y, Z, cell)[:, 0]
            worst = max(worst, np.abs(Nn - Na).max() / np.abs(Nn).max())
    assert worst < 5e-9, worst


@pytest.mark.parametrize("block,cell", [((2, 2, 2), (1.0, 1.0, 1.0)),
                                        ((3, 2, 1), (2.0, 2.0, 1.0)),
                                        ((4, 1, 3), (1.0, 2.0, 1.5)),
                                        ((14, 13, 2), (1.0, 1.0, 1.0))])
def test_prism_additivity(block, cell):
    """(1/n) sum_{c,c'} N(r_c - r_c') equals the self tensor of the whole
    block (the tensor integral is additive).  The 14x13x2 block reaches
    offsets beyond the cutoff, so both formulas and their junction count."""
    k, l, m = block
    oi, oj, ok = np.meshgrid(np.arange(-k + 1, k), np.arange(-l + 1, l), np.arange(-m + 1, m),
                             indexing="ij")
    count = (k - np.abs(oi)) * (l - np.abs(oj)) * (m - np.abs(ok))
    N = demag.cell_tensor(oi * cell[0], oj * cell[1], ok * cell[2], cell)
    avg = (N * count).sum(axis=(1, 2, 3)) / (k * l * m)
    big = _tensor((0, 0, 0), (k * cell[0], l * cell[1], m * cell[2]))
    assert np.abs(avg - big).max() < 2e-11, (avg, big)


# -- the field -----------------------------------------------------------------
@pytest.mark.parametrize("shape,cell", [((5, 4, 3), (2e-9, 3e-9, 1.5e-9)),
                                        ((3, 6, 2), (1e-9, 1e-9, 1e-9)),
                                        ((6, 3, 1), (4e-9, 4e-9, 2e-9)),
                                        ((1, 1, 7), (1e-9, 2e-9, 1e-9)),
                                        ((8, 8, 2), (2e-9, 2e-9, 1e-9))])
def test_fft_convolution_equals_direct_sum(shape, cell):
    rng = np.random.default_rng(7)
    M = rng.normal(size=(3,) + shape[::-1]) * 8e5
    Bd = demag.demag_direct(shape, cell, M)
    Bf = demag.demag_fft(shape, cell, M)
    assert np.abs(Bd - Bf).max() <= 1e-12 * np.abs(Bd).max()


def test_single_cube_field():
    Ms = 1e6
    M = np.zeros((3, 1, 1, 1))
    M[2] = Ms
    B = demag.demag_fft((1, 1, 1), (3e-9,) * 3, M)
    assert abs(B[2, 0, 0, 0] + MU0 * Ms / 3) < 1e-14


def test_uniform_block_average_field_is_prism_factor():
    """Uniformly magnetised block of 24x16x2 cells: the cell-averaged field
    is -mu0 N_prism M with N_prism the self factor of the whole block."""
    shape, cell = (24, 16, 2), (1e-9, 1e-9, 1e-9)
    M = np.zeros((3, 2, 16, 24))
    M[0], M[2] = 3e5, 8e5
    B = demag.demag_fft(shape, cell, M)
    Np = _full(_tensor((0, 0, 0), (24e-9, 16e-9, 2e-9)))
    ref = -MU0 * Np @ np.array([3e5, 0.0, 8e5])
    assert np.abs(B.reshape(3, -1).mean(axis=1) - ref).max() < 1e-11 * np.abs(ref).max()


def test_thin_film_centre_field_tends_to_minus_mu0_ms():
    Ms = 8e5
    prev = 0.0
    for n in (16, 64, 256):
        M = np.zeros((3, 1, n, n))
        M[2] = Ms
        B = demag.demag_fft((n, n, 1), (1e-9, 1e-9, 1e-9), M)
        ratio = -B[2, 0, n // 2, n // 2] / (MU0 * Ms)
        assert prev < ratio < 1.0
        prev = ratio
    assert prev > 0.99
