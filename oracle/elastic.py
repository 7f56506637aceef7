"""Elastodynamics and magnetoelastic force, oracle version.

Test infrastructure only (see oracle/__init__.py).

Follows the paper's Methods sections "Elasticity" and "Magnetoelasticity":
  * rho d^2u/dt^2 = f_tot (Eq. elasticity), written as du/dt = v,
    dv/dt = f_tot / rho.
  * The strain is the numeric gradient of u and the elastic force the numeric
    divergence of the stress, both 4th-order central differences in the
    bulk and lower order near and at the boundaries.  The lower-order
    schemes are our reading of a passage the paper leaves open:
      gradient   - 2nd-order central one cell from an edge, 2nd-order
                   one-sided at an edge cell, (f1 - f0)/h when n = 2;
      divergence - the negative transpose of that gradient operator
                   (-G^T).  In the bulk it is the same 4th-order central
                   stencil; near the edges it is the closure that makes the
                   elastic force minus the gradient of the discrete strain
                   energy, so the semi-discrete system conserves energy, has
                   no growing modes, and has the traction-free condition
                   sigma.n = 0 as its natural boundary condition.  (A
                   face-traction half-cell closure was rejected: with the
                   shear coupling of 2-D grids it has complex eigenvalues,
                   i.e. growing modes.)
    An axis with a single cell has zero derivatives along it.
  * Cubic stiffness: sigma_ii = c11 eps_ii + c12 (eps_jj + eps_kk),
    sigma_ij = 2 c44 eps_ij, plus the viscous term eta C:eps_dot.
  * Magnetoelastic force, Eq. (magnetoelastic-force), with each derivative of
    m taken with the gradient scheme above; for an antiferromagnet each
    sublattice adds its own force (shared u, v, C, eps).
"""
import numpy as np


def d1(F, axis, h):
    """Gradient scheme along `axis` of F (last three axes are z, y, x)."""
    n = F.shape[axis]
    out = np.zeros_like(F)
    if n == 1:
        return out

    def sl(i):
        s = [slice(None)] * F.ndim
        s[axis] = i
        return tuple(s)

    if n == 2:
        g = (F[sl(1)] - F[sl(0)]) / h
        out[sl(0)] = g
        out[sl(1)] = g
        return out
    out[sl(0)] = (-3.0 * F[sl(0)] + 4.0 * F[sl(1)] - F[sl(2)]) / (2.0 * h)
    out[sl(n - 1)] = (3.0 * F[sl(n - 1)] - 4.0 * F[sl(n - 2)] + F[sl(n - 3)]) / (2.0 * h)
    for i in (1, n - 2):
        if 0 < i < n - 1:
            out[sl(i)] = (F[sl(i + 1)] - F[sl(i - 1)]) / (2.0 * h)
    for i in range(2, n - 2):
        out[sl(i)] = (-F[sl(i + 2)] + 8.0 * F[sl(i + 1)]
                      - 8.0 * F[sl(i - 1)] + F[sl(i - 2)]) / (12.0 * h)
    return out


def _rows(n, h):
    """Rows of the 1-D gradient operator G as {i: [(j, G_ij), ...]}."""
    if n == 1:
        return {}
    if n == 2:
        return {0: [(0, -1.0 / h), (1, 1.0 / h)], 1: [(0, -1.0 / h), (1, 1.0 / h)]}
    rows = {0: [(0, -1.5 / h), (1, 2.0 / h), (2, -0.5 / h)],
            n - 1: [(n - 3, 0.5 / h), (n - 2, -2.0 / h), (n - 1, 1.5 / h)]}
    for i in {1, n - 2}:
        if 0 < i < n - 1:
            rows[i] = [(i - 1, -0.5 / h), (i + 1, 0.5 / h)]
    for i in range(2, n - 2):
        rows[i] = [(i - 2, 1.0 / (12 * h)), (i - 1, -8.0 / (12 * h)),
                   (i + 1, 8.0 / (12 * h)), (i + 2, -1.0 / (12 * h))]
    return rows


def div1(S, axis, h):
    """Divergence scheme along `axis`: -G^T S with G the gradient operator of
    `d1`, i.e. (div S)_j = -sum_i G_ij S_i."""
    n = S.shape[axis]
    out = np.zeros_like(S)

    def sl(i):
        s = [slice(None)] * S.ndim
        s[axis] = i
        return tuple(s)

    for i, row in _rows(n, h).items():
        for j, g in row:
            out[sl(j)] -= g * S[sl(i)]
    return out


_AX = (-1, -2, -3)   # array axis of x, y, z


def grad(u, cell):
    """du_j/dx_i as G[i][j] (arrays [nz][ny][nx])."""
    return [[d1(u[j], _AX[i], cell[i]) for j in range(3)] for i in range(3)]


def strain(u, cell):
    """Tensor strain eps_ij = (d_i u_j + d_j u_i) / 2 as (xx, yy, zz, xy, xz, yz)."""
    G = grad(u, cell)
    return np.stack([G[0][0], G[1][1], G[2][2],
                     0.5 * (G[0][1] + G[1][0]),
                     0.5 * (G[0][2] + G[2][0]),
                     0.5 * (G[1][2] + G[2][1])])


def stress(eps, c11, c12, c44):
    exx, eyy, ezz, exy, exz, eyz = eps
    return np.stack([c11 * exx + c12 * (eyy + ezz),
                     c11 * eyy + c12 * (exx + ezz),
                     c11 * ezz + c12 * (exx + eyy),
                     2.0 * c44 * exy, 2.0 * c44 * exz, 2.0 * c44 * eyz])


def _full(sig):
    xx, yy, zz, xy, xz, yz = sig
    return [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]


def elastic_force(u, v, p):
    """f_el = div(sigma), sigma = C:eps(u) + eta C:eps(v)."""
    g = p.glob
    sig = stress(strain(u, p.cell), g["C11"], g["C12"], g["C44"])
    if g.get("ETA", 0.0) != 0.0:
        sig = sig + g["ETA"] * stress(strain(v, p.cell), g["C11"], g["C12"], g["C44"])
    S = _full(sig)
    return np.stack([sum(div1(S[i][j], _AX[i], p.cell[i]) for i in range(3))
                     for j in range(3)])


def mel_force(m, B1, B2, cell):
    """Eq. (magnetoelastic-force) for one sublattice."""
    G = grad(m, cell)             # G[i][j] = d_i m_j
    mx, my, mz = m
    fx = 2 * B1 * mx * G[0][0] + B2 * (mx * (G[1][1] + G[2][2]) + my * G[1][0] + mz * G[2][0])
    fy = 2 * B1 * my * G[1][1] + B2 * (my * (G[0][0] + G[2][2]) + mx * G[0][1] + mz * G[2][1])
    fz = 2 * B1 * mz * G[2][2] + B2 * (mz * (G[0][0] + G[1][1]) + mx * G[0][2] + my * G[1][2])
    return np.stack([fx, fy, fz])


def total_force(p, P, ms, u, v):
    f = elastic_force(u, v, p)
    if "MEL" in p.terms:
        for s in range(p.n_sub):
            f = f + mel_force(ms[s], P["B1"][s], P["B2"][s], p.cell)
    return f


def elastic_energy(p, u, v):
    """Strain energy 1/2 sigma:eps and kinetic energy 1/2 rho v^2 (J)."""
    g = p.glob
    dV = p.cell[0] * p.cell[1] * p.cell[2]
    eps = strain(u, p.cell)
    sig = stress(eps, g["C11"], g["C12"], g["C44"])
    w = (sig[:3] * eps[:3]).sum(axis=0) + 2.0 * (sig[3:] * eps[3:]).sum(axis=0)
    return 0.5 * dV * w.sum(), 0.5 * g["RHO"] * dV * (v * v).sum()
