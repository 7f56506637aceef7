"""Demagnetising (magnetostatic) field, oracle version.

Test infrastructure only (see oracle/__init__.py).

Follows the paper's Methods section "Magnetostatic field": the cell-to-cell
demag tensor is the analytical result of Newell, Williams and Dunlop (J.
Geophys. Res. 98, 9551 (1993)) below a cutoff radius and an asymptotic
result above it; for an antiferromagnet the sublattice magnetisations of a
cell are summed before the field is evaluated.  The field is
    B_demag(r_c) = -mu0 * sum_{c'} N(r_c - r_c') M(c').

N is the "demagnetising factor" tensor: a uniformly magnetised isolated cube
has N = I/3, so B = -mu0 M / 3 at its centre.

Asymptotic expansion (our statement of the multipole method the paper
cites): the tensor between two identical cuboids at centre offset r equals
    N(r) = V * E_s[ -d_a d_b (1 / (4 pi |r + s|)) ],
where s = u2 - u1 is the difference of two points uniform in the cell, whose
components are independent and triangular on [-D_i, D_i].  Expanding in s,
    N_ab(r) = -V/(4 pi) sum_{alpha even} E[s^alpha]/alpha! d^(alpha+e_a+e_b) (1/r)
with E[s_i^(2k)] = 2 D_i^(2k) / ((2k+1)(2k+2)).  Terms up to |alpha| = 2p
leave an error of relative order (D/r)^(2p+2).  Derivatives of 1/r come from
the McMurchie-Davidson recurrence (J. Comput. Phys. 26, 218 (1978)).

Cutoff and order (the paper gives neither): Newell for |r| < RC * max(D),
asymptotic with p = ORDER beyond.  At the cutoff the two agree to ~1e-9
relative in FP64 (checked in tests/test_oracle_demag.py).
"""
from math import factorial, pi

import numpy as np

from inputs import MU0

RC = 10.0      # cutoff radius in units of the largest cell dimension
ORDER = 4      # asymptotic expansion through E[s^8] terms

# component order used everywhere: xx, yy, zz, xy, xz, yz
PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
# parity of each component along (x, y, z): 1 = odd (sign flip on reflection)
ODD = ((0, 0, 0), (0, 0, 0), (0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1))


# --------------------------------------------------------------------------
# Newell f and g functions (even in all arguments / odd in x and y)
# --------------------------------------------------------------------------
def newell_f(x, y, z):
    """Newell's f(x, y, z); N_xx is its 27-point second difference."""
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = (2.0 * x2 - y2 - z2) * R / 6.0
    with np.errstate(divide="ignore", invalid="ignore"):
        rxz = np.sqrt(x2 + z2)
        rxy = np.sqrt(x2 + y2)
        out = out + np.where(rxz > 0, 0.5 * y * (z2 - x2) * np.arcsinh(y / rxz), 0.0)
        out = out + np.where(rxy > 0, 0.5 * z * (y2 - x2) * np.arcsinh(z / rxy), 0.0)
        out = out - np.where(x > 0, x * y * z * np.arctan(y * z / (x * R)), 0.0)
    return out


def newell_g(x, y, z):
    """Newell's g(x, y, z); N_xy is its 27-point second difference."""
    sgn = np.sign(x) * np.sign(y)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = -x * y * R / 3.0
    with np.errstate(divide="ignore", invalid="ignore"):
        rxy = np.sqrt(x2 + y2)
        ryz = np.sqrt(y2 + z2)
        rxz = np.sqrt(x2 + z2)
        out = out + np.where(rxy > 0, x * y * z * np.arcsinh(z / rxy), 0.0)
        out = out + np.where(ryz > 0, y / 6.0 * (3.0 * z2 - y2) * np.arcsinh(x / ryz), 0.0)
        out = out + np.where(rxz > 0, x / 6.0 * (3.0 * z2 - x2) * np.arcsinh(y / rxz), 0.0)
        out = out - np.where(z > 0, z ** 3 / 6.0 * np.arctan(x * y / (z * R)), 0.0)
        out = out - np.where(y > 0, z * y2 / 2.0 * np.arctan(x * z / (y * R)), 0.0)
        out = out - np.where(x > 0, z * x2 / 2.0 * np.arctan(y * z / (x * R)), 0.0)
    return sgn * out


_W = {-1: -1.0, 0: 2.0, 1: -1.0}


def _second_difference(fun, X, Y, Z, a, b, c):
    """sum_{i,j,k in -1,0,1} w_i w_j w_k fun(X + i a, Y + j b, Z + k c),
    w_0 = 2, w_{+-1} = -1, divided by 4 pi a b c."""
    acc = 0.0
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                acc = acc + _W[i] * _W[j] * _W[k] * fun(X + i * a, Y + j * b, Z + k * c)
    return acc / (4.0 * pi * a * b * c)


def newell_tensor(X, Y, Z, cell):
    """Six components (xx, yy, zz, xy, xz, yz) of the Newell cell tensor at
    centre offsets (X, Y, Z), arrays in metres."""
    L = max(cell)
    X, Y, Z = (np.asarray(v, dtype=np.float64) / L for v in (X, Y, Z))
    dx, dy, dz = (c / L for c in cell)
    return np.stack([
        _second_difference(newell_f, X, Y, Z, dx, dy, dz),
        _second_difference(newell_f, Y, X, Z, dy, dx, dz),
        _second_difference(newell_f, Z, Y, X, dz, dy, dx),
        _second_difference(newell_g, X, Y, Z, dx, dy, dz),
        _second_difference(newell_g, X, Z, Y, dx, dz, dy),
        _second_difference(newell_g, Y, Z, X, dy, dz, dx),
    ])


# --------------------------------------------------------------------------
# Asymptotic expansion
# --------------------------------------------------------------------------
def _double_factorial(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def inv_r_derivatives(X, Y, Z, nmax):
    """All partial derivatives d^t_x d^u_y d^v_z (1/r), t+u+v <= nmax, by the
    McMurchie-Davidson recurrence
        R^n_000 = (-1)^n (2n-1)!! / r^(2n+1),
        R^n_{t,u,v} = (t-1) R^{n+1}_{t-2,u,v} + X R^{n+1}_{t-1,u,v}  (t > 0),
    and the same along y and z; the derivative is R^0_{t,u,v}."""
    r2 = X * X + Y * Y + Z * Z
    inv_r = 1.0 / np.sqrt(r2)
    inv_r2 = 1.0 / r2
    R = {}
    for n in range(nmax + 1):
        R[(n, 0, 0, 0)] = (-1) ** n * _double_factorial(2 * n - 1) * inv_r * inv_r2 ** n
    for tot in range(1, nmax + 1):
        for t in range(tot + 1):
            for u in range(tot - t + 1):
                v = tot - t - u
                for n in range(nmax - tot + 1):
                    if t > 0:
                        val = X * R[(n + 1, t - 1, u, v)]
                        if t > 1:
                            val = val + (t - 1) * R[(n + 1, t - 2, u, v)]
                    elif u > 0:
                        val = Y * R[(n + 1, t, u - 1, v)]
                        if u > 1:
                            val = val + (u - 1) * R[(n + 1, t, u - 2, v)]
                    else:
                        val = Z * R[(n + 1, t, u, v - 1)]
                        if v > 1:
                            val = val + (v - 1) * R[(n + 1, t, u, v - 2)]
                    R[(n, t, u, v)] = val
    return {k[1:]: val for k, val in R.items() if k[0] == 0}


def _moment(d, k):
    """E[s^(2k)] for s triangular on [-d, d]."""
    return 1.0 if k == 0 else 2.0 * d ** (2 * k) / ((2 * k + 1) * (2 * k + 2))


def asymptotic_tensor(X, Y, Z, cell, order=ORDER, chunk=16384):
    """Asymptotic cell tensor (six components) at centre offsets X, Y, Z."""
    L = max(cell)
    X, Y, Z = (np.atleast_1d(np.asarray(v, dtype=np.float64) / L).ravel() for v in (X, Y, Z))
    dx, dy, dz = (c / L for c in cell)
    V = dx * dy * dz
    out = np.empty((6, X.size))
    terms = []
    for i in range(order + 1):
        for j in range(order + 1 - i):
            for k in range(order + 1 - i - j):
                coef = (_moment(dx, i) * _moment(dy, j) * _moment(dz, k)
                        / (factorial(2 * i) * factorial(2 * j) * factorial(2 * k)))
                terms.append((coef, (2 * i, 2 * j, 2 * k)))
    for s in range(0, X.size, chunk):
        sl = slice(s, s + chunk)
        D = inv_r_derivatives(X[sl], Y[sl], Z[sl], 2 * order + 2)
        for comp, (a, b) in enumerate(PAIRS):
            acc = 0.0
            for coef, base in terms:
                idx = list(base)
                idx[a] += 1
                idx[b] += 1
                acc = acc + coef * D[tuple(idx)]
            out[comp, sl] = -V / (4.0 * pi) * acc
    return out


def cell_tensor(X, Y, Z, cell, rc=RC, order=ORDER):
    """Cell tensor at offsets (X, Y, Z): Newell below rc*max(cell), the
    asymptotic expansion at and above it.  Returns shape (6,) + X.shape."""
    X, Y, Z = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (X, Y, Z)))
    shape = X.shape
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    far = np.sqrt(X * X + Y * Y + Z * Z) >= rc * max(cell)
    out = np.empty((6, X.size))
    if (~far).any():
        out[:, ~far] = newell_tensor(X[~far], Y[~far], Z[~far], cell)
    if far.any():
        out[:, far] = asymptotic_tensor(X[far], Y[far], Z[far], cell, order)
    return out.reshape((6,) + shape)


def tensor_octant(shape, cell):
    """N at offsets (i dx, j dy, k dz), 0 <= i < nx etc.: float64 [6][nz][ny][nx]."""
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return cell_tensor(i * cell[0], j * cell[1], k * cell[2], cell)


def tensor_at(noct, ix, iy, iz):
    """N at integer offsets (ix, iy, iz) (any signs) from the octant table,
    using the parity of each component."""
    out = []
    for comp in range(6):
        v = noct[comp, np.abs(iz), np.abs(iy), np.abs(ix)]
        ox, oy, oz = ODD[comp]
        if ox:
            v = v * np.sign(ix)
        if oy:
            v = v * np.sign(iy)
        if oz:
            v = v * np.sign(iz)
        out.append(v)
    return np.stack(out)


def _apply(Nc, M):
    """H = N M for a symmetric tensor given by its 6 components."""
    xx, yy, zz, xy, xz, yz = Nc
    return np.stack([xx * M[0] + xy * M[1] + xz * M[2],
                     xy * M[0] + yy * M[1] + yz * M[2],
                     xz * M[0] + yz * M[1] + zz * M[2]])


# --------------------------------------------------------------------------
# Field: definition (direct sum) and zero-padded FFT convolution
# --------------------------------------------------------------------------
def demag_direct(shape, cell, M, noct=None, cells=None):
    """B_demag by the O(N^2) sum of the definition.  M: [3][nz][ny][nx] in
    A/m.  `cells` optionally restricts the targets to a list of flat cell
    indices; then the result has shape [3][len(cells)]."""
    nx, ny, nz = shape
    if noct is None:
        noct = tensor_octant(shape, cell)
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    src = M.reshape(3, -1)
    kx, ky, kz = kx.ravel(), ky.ravel(), kz.ravel()
    targets = range(nx * ny * nz) if cells is None else cells
    out = np.empty((3, len(targets)))
    for n, c in enumerate(targets):
        Nc = tensor_at(noct, kx[c] - kx, ky[c] - ky, kz[c] - kz)
        out[:, n] = -MU0 * _apply(Nc, src).sum(axis=1)
    if cells is None:
        return out.reshape(3, nz, ny, nx)
    return out


def padded_sizes(shape):
    """Linear (non-circular) zero padding: 2n on axes with n > 1."""
    return tuple(2 * n if n > 1 else 1 for n in shape)


def demag_fft(shape, cell, M, noct=None):
    """B_demag by the zero-padded FFT convolution of M with N."""
    nx, ny, nz = shape
    Px, Py, Pz = padded_sizes(shape)
    if noct is None:
        noct = tensor_octant(shape, cell)

    def fold(n, P):
        pos = np.arange(P)
        off = np.where(pos < n, pos, pos - P)
        valid = np.abs(off) < n
        return np.where(valid, np.abs(off), 0), np.sign(off), valid

    ixs, sx, vx = fold(nx, Px)
    iys, sy, vy = fold(ny, Py)
    izs, sz, vz = fold(nz, Pz)
    mask = vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
    Khat = []
    for comp in range(6):
        K = noct[comp][np.ix_(izs, iys, ixs)] * mask
        ox, oy, oz = ODD[comp]
        if ox:
            K = K * sx[None, None, :]
        if oy:
            K = K * sy[None, :, None]
        if oz:
            K = K * sz[:, None, None]
        Khat.append(np.fft.rfftn(K, axes=(0, 1, 2)))
    Mp = np.zeros((3, Pz, Py, Px))
    Mp[:, :nz, :ny, :nx] = M
    Mhat = np.fft.rfftn(Mp, axes=(1, 2, 3))
    Hhat = _apply(Khat, Mhat)
    H = np.fft.irfftn(Hhat, s=(Pz, Py, Px), axes=(1, 2, 3))
    return -MU0 * H[:, :nz, :ny, :nx]
