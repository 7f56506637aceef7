"""Effective field terms and LLG torque, oracle version.

Test infrastructure only (see oracle/__init__.py).

Arrays are float64, SoA [3][nz][ny][nx] per sublattice.  Cell index
c = x + nx (y + ny z).  A cell with Ms = 0 is empty: it has no
magnetisation, its field and torque are zero, and its neighbours see it as
a boundary.

Passages followed (arXiv 2411.18194, Methods):
  * LLG torque, Eq. (LLG_torque):
        tau = -gamma/(1+alpha^2) [m x B + alpha m x (m x B)].
  * Exchange, Eq. (AFM_exchange_field): the ferromagnetic term
    (2 A11 / Ms) lap(m) on the 6-neighbour stencil; across a region
    interface A is the harmonic mean 2 A1 A2 / (A1 + A2) (the mumax3
    convention the paper defers to).  For two sublattices also
    (A12 / Ms) lap(m') + (4 A0 / (Ms a^2)) m'.
  * Interfacial DMI, Eq. (dmi) with D_xzx = D_yzy = D, D_xxz = D_yyz = -D,
    i.e. energy density D [m_z div m - (m . grad) m_z] and field
    (2D/Ms)(d_x m_z, d_y m_z, -d_x m_x - d_y m_y) with central differences.
    Across an interface D is the arithmetic mean.
  * Neumann boundary condition, Eq. (AFM_Neumann_BC) with A12 = 0 and the
    interfacial tensor: d_n m = -(D / 2A) (z x n) x m; a missing neighbour
    takes the ghost value m + Delta_n d_n m in the exchange and DMI stencils.
    For two sublattices without DMI the condition reduces to d_n m = 0.
  * Open boundary (the alternative the same passage names, Problem.open_bc):
    a missing neighbour drops out of the exchange and DMI sums, so the field
    is the exact negative gradient of the pair energy (energies()).  Without
    DMI this equals the Neumann field (the ghost is m).
  * Uniaxial anisotropy "as in mumax3":
        B = (2 Ku1/Ms)(m.u) u + (4 Ku2/Ms)(m.u)^3 u,
    plus a second uniaxial term (2 Kb1/Ms)(m.ub) ub (used for the biaxial
    antiferromagnet workload).
  * Zeeman: B_ext.
  * Magnetoelastic field, Eq. (magnetoelastic-field):
        B_mel = -(2/Ms)(B1 eps_ii m_i + B2 sum_{j != i} eps_ij m_j),
    eps the tensor (not engineering) strain of the shared displacement.
"""
import numpy as np

from inputs import GAMMA, MU0, PARAM_SCALARS, PARAM_VECTORS
from . import demag as _demag
from . import elastic as _elastic

AXES = ((-1, 0), (-2, 1), (-3, 2))   # (array axis, spatial index) for x, y, z


def cell_params(p):
    """Expand the per-region tables to per-cell arrays.
    Scalars: [n_sub][nz][ny][nx]; vectors: [n_sub][3][nz][ny][nx]."""
    reg = p.regions
    P = {k: p.scal[k][:, reg] for k in PARAM_SCALARS}
    for k in PARAM_VECTORS:
        v = np.moveaxis(p.vec[k][:, reg], -1, 1)
        if k in ("ANIS_U", "ANIS_UB", "ANIS_C1"):
            v = _unit(v)
        P[k] = v
    # cubic axes: c2 made orthogonal to c1 (Gram-Schmidt), c3 = c1 x c2
    c1 = P["ANIS_C1"]
    P["ANIS_C2"] = _unit(P["ANIS_C2"] - (P["ANIS_C2"] * c1).sum(axis=1, keepdims=True) * c1)
    P["ANIS_C3"] = np.cross(c1, P["ANIS_C2"], axis=1)
    return P


def _unit(v):
    nrm = np.sqrt((v * v).sum(axis=1, keepdims=True))
    return np.where(nrm > 0, v / np.where(nrm > 0, nrm, 1.0), 0.0)


def shift(a, axis, d):
    """Value at c + d (d = +-1) along `axis`; zero beyond the edge.
    Returns (shifted array, inside-grid mask over the last three axes)."""
    out = np.zeros_like(a)
    n = a.shape[axis]
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if d > 0:
        src[axis], dst[axis] = slice(1, n), slice(0, n - 1)
    else:
        src[axis], dst[axis] = slice(0, n - 1), slice(1, n)
    out[tuple(dst)] = a[tuple(src)]
    inside = np.zeros(a.shape[-3:], dtype=bool)
    di = [slice(None)] * 3
    di[axis] = dst[axis]
    inside[tuple(di)] = True
    return out, inside


def _harmonic(a, b):
    s = a + b
    return np.where(s != 0, 2.0 * a * b / np.where(s != 0, s, 1.0), 0.0)


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def _dot(a, b):
    return (a * b).sum(axis=0)


def ghost_derivative(m, A, D, spatial, d):
    """d_n m at a boundary with outward normal n = d * e_spatial:
    -(D / 2A) (z x n) x m (zero when A = 0 and across z-faces)."""
    if spatial == 2:
        return np.zeros_like(m)
    n = np.zeros(3)
    n[spatial] = d
    zxn = np.cross([0.0, 0.0, 1.0], n)
    v = np.stack([zxn[1] * m[2] - zxn[2] * m[1],
                  zxn[2] * m[0] - zxn[0] * m[2],
                  zxn[0] * m[1] - zxn[1] * m[0]])
    coef = np.where(A > 0, -D / (2.0 * np.where(A > 0, A, 1.0)), 0.0)
    return coef * v


def neighbour(p, P, s, m, axis, spatial, d):
    """Neighbour value of sublattice s along (axis, d): the real neighbour if it
    exists and is magnetic, else the boundary ghost (Neumann) or, for an open
    boundary, the cell's own value with D_pair = 0.  Returns
    (value, present mask, A_pair, D_pair)."""
    Ms, A, D = P["MS"][s], P["AEX"][s], P["DIND"][s]
    h = p.cell[spatial]
    m_nb, inside = shift(m, axis, d)
    Ms_nb, _ = shift(Ms, axis, d)
    A_nb, _ = shift(A, axis, d)
    D_nb, _ = shift(D, axis, d)
    present = inside & (Ms_nb > 0)
    use_dmi = "DMI" in p.terms
    if getattr(p, "open_bc", False):
        # open: no ghost; the missing pair contributes m - m = 0 to the
        # exchange sum and carries D = 0 in the DMI sum
        value = np.where(present, m_nb, m)
        D_pair = np.where(present, 0.5 * (D + D_nb), 0.0)
    else:
        Dg = D if use_dmi else np.zeros_like(D)
        ghost = m + h * ghost_derivative(m, A, Dg, spatial, d)
        value = np.where(present, m_nb, ghost)
        D_pair = np.where(present, 0.5 * (D + D_nb), D)
    A_pair = np.where(present, _harmonic(A, A_nb), A)
    return value, present, A_pair, D_pair


def exchange_field(p, P, s, m):
    """(2 A / Ms) sum_d (m_d - m) / Delta_d^2 (ferromagnetic exchange)."""
    Ms = P["MS"][s]
    B = np.zeros_like(m)
    for axis, spatial in AXES:
        h = p.cell[spatial]
        for d in (-1, 1):
            val, present, A_pair, _ = neighbour(p, P, s, m, axis, spatial, d)
            B += 2.0 * A_pair * (val - m) / (h * h)
    return np.where(Ms > 0, B / np.where(Ms > 0, Ms, 1.0), 0.0)


def dmi_field(p, P, s, m):
    """Interfacial DMI: (1/Ms) sum_{d=+-x} sgn(d) D m_z(c+d)/dx on B_x, the
    same with y on B_y, and -(1/Ms) sum sgn(d) D m_{x|y}(c+d)/h on B_z
    (central differences of (2D/Ms)(d_x m_z, d_y m_z, -d_x m_x - d_y m_y))."""
    Ms = P["MS"][s]
    B = np.zeros_like(m)
    for axis, spatial in AXES[:2]:
        h = p.cell[spatial]
        for d in (-1, 1):
            val, present, _, D_pair = neighbour(p, P, s, m, axis, spatial, d)
            B[spatial] += d * D_pair * val[2] / h
            B[2] -= d * D_pair * val[spatial] / h
    return np.where(Ms > 0, B / np.where(Ms > 0, Ms, 1.0), 0.0)


def anisotropy_field(p, P, s, m):
    Ms = P["MS"][s]
    inv = np.where(Ms > 0, 1.0 / np.where(Ms > 0, Ms, 1.0), 0.0)
    u, ub = P["ANIS_U"][s], P["ANIS_UB"][s]
    mu, mub = _dot(m, u), _dot(m, ub)
    return inv * ((2.0 * P["KU1"][s] * mu + 4.0 * P["KU2"][s] * mu ** 3) * u
                  + 2.0 * P["KB1"][s] * mub * ub)


def cubic_anisotropy_field(p, P, s, m):
    """Cubic anisotropy (the paper's field terms: uniaxial or cubic, done as in
    mumax3): energy density Kc1 (a^2 b^2 + a^2 c^2 + b^2 c^2) with a, b, c the
    components of m along the cubic axes c1, c2, c3; field -(1/Ms) dE/dm."""
    Ms = P["MS"][s]
    inv = np.where(Ms > 0, 1.0 / np.where(Ms > 0, Ms, 1.0), 0.0)
    c1, c2, c3 = P["ANIS_C1"][s], P["ANIS_C2"][s], P["ANIS_C3"][s]
    a, b, c = _dot(m, c1), _dot(m, c2), _dot(m, c3)
    K = P["KC1"][s]
    return -2.0 * K * inv * (a * (b * b + c * c) * c1 + b * (a * a + c * c) * c2 + c * (a * a + b * b) * c3)


def afm_field(p, P, s, ms):
    """Intersublattice exchange for sublattice s: (A12/Ms) lap(m') with
    zero-Neumann ghosts + (4 A0 / (Ms a^2)) m'."""
    o = 1 - s
    Ms, Ms_o = P["MS"][s], P["MS"][o]
    mo = np.where(Ms_o > 0, ms[o], 0.0)
    A12, A0, a = p.glob["A12"], p.glob["A0"], p.glob["LATTICE_A"]
    lap = np.zeros_like(mo)
    for axis, spatial in AXES:
        h = p.cell[spatial]
        for d in (-1, 1):
            mo_nb, inside = shift(mo, axis, d)
            Ms_nb, _ = shift(Ms_o, axis, d)
            present = inside & (Ms_nb > 0)
            lap += np.where(present, mo_nb - mo, 0.0) / (h * h)
    inv = np.where(Ms > 0, 1.0 / np.where(Ms > 0, Ms, 1.0), 0.0)
    return inv * (A12 * lap + 4.0 * A0 / (a * a) * mo)


def mel_field(p, P, s, m, eps):
    """Eq. (magnetoelastic-field); eps = (xx, yy, zz, xy, xz, yz)."""
    Ms = P["MS"][s]
    inv = np.where(Ms > 0, 1.0 / np.where(Ms > 0, Ms, 1.0), 0.0)
    B1, B2 = P["B1"][s], P["B2"][s]
    exx, eyy, ezz, exy, exz, eyz = eps
    return -2.0 * inv * np.stack([
        B1 * exx * m[0] + B2 * (exy * m[1] + exz * m[2]),
        B1 * eyy * m[1] + B2 * (exy * m[0] + eyz * m[2]),
        B1 * ezz * m[2] + B2 * (exz * m[0] + eyz * m[1]),
    ])


def demag_source(p, P, ms):
    """M = sum_s Ms^(s) m^(s) (A/m)."""
    return sum(P["MS"][s] * ms[s] for s in range(p.n_sub))


def effective_fields(p, ms, u=None, noct=None, demag="fft", P=None, parts=False):
    """B_eff for every sublattice.  ms: list of float64 [3][nz][ny][nx].
    With parts=True also returns a dict of the individual terms."""
    P = cell_params(p) if P is None else P
    terms = p.terms
    out, detail = [], []
    Bd = None
    if "DEMAG" in terms:
        M = demag_source(p, P, ms)
        if demag == "fft":
            Bd = _demag.demag_fft(p.shape, p.cell, M, noct)
        else:
            Bd = _demag.demag_direct(p.shape, p.cell, M, noct)
    eps = None
    if "MEL" in terms:
        eps = _elastic.strain(u, p.cell)
    for s in range(p.n_sub):
        m = ms[s]
        d = {}
        if Bd is not None:
            d["demag"] = Bd
        if "EXCH" in terms:
            d["exch"] = exchange_field(p, P, s, m)
        if "DMI" in terms:
            d["dmi"] = dmi_field(p, P, s, m)
        if "ANIS" in terms:
            d["anis"] = anisotropy_field(p, P, s, m)
        if "CUBIC" in terms:
            d["cubic"] = cubic_anisotropy_field(p, P, s, m)
        if "ZEEMAN" in terms:
            d["zeeman"] = P["B_EXT"][s] * np.ones_like(m)
        if "AFM" in terms and p.n_sub == 2:
            d["afm"] = afm_field(p, P, s, ms)
        if "MEL" in terms:
            d["mel"] = mel_field(p, P, s, m, eps)
        B = sum(d.values()) if d else np.zeros_like(m)
        B = np.where(P["MS"][s] > 0, B, 0.0)
        out.append(B)
        detail.append(d)
    return (out, detail) if parts else out


def llg_torque(m, B, alpha):
    """Eq. (LLG_torque)."""
    mxB = _cross(m, B)
    return -GAMMA / (1.0 + alpha * alpha) * (mxB + alpha * _cross(m, mxB))


def torques(p, ms, Bs, P=None):
    P = cell_params(p) if P is None else P
    return [np.where(P["MS"][s] > 0, llg_torque(ms[s], Bs[s], P["ALPHA"][s]), 0.0)
            for s in range(p.n_sub)]


# --------------------------------------------------------------------------
# Energies (J) whose negative gradient is the discrete field:
# B = -(1 / (Ms dV)) dE/dm in the interior.
# --------------------------------------------------------------------------
def energies(p, ms, u=None, noct=None, P=None):
    P = cell_params(p) if P is None else P
    dV = p.cell[0] * p.cell[1] * p.cell[2]
    E = {}
    terms = p.terms
    if "DEMAG" in terms:
        M = demag_source(p, P, ms)
        Bd = _demag.demag_fft(p.shape, p.cell, M, noct)
        E["demag"] = -0.5 * dV * (M * Bd).sum()
    for s in range(p.n_sub):
        m, Ms = ms[s], P["MS"][s]
        if "EXCH" in terms or "DMI" in terms:
            for axis, spatial in AXES:
                h = p.cell[spatial]
                val, present, A_pair, D_pair = neighbour(p, P, s, m, axis, spatial, 1)
                keep = present & (Ms > 0)
                if "EXCH" in terms:
                    E["exch"] = E.get("exch", 0.0) + dV * (np.where(
                        keep, A_pair * ((val - m) ** 2).sum(axis=0), 0.0)).sum() / (h * h)
                if "DMI" in terms and spatial < 2:
                    pair = m[2] * val[spatial] - m[spatial] * val[2]
                    E["dmi"] = E.get("dmi", 0.0) + dV * np.where(keep, D_pair * pair, 0.0).sum() / h
        if "ANIS" in terms:
            mu, mub = _dot(m, P["ANIS_U"][s]), _dot(m, P["ANIS_UB"][s])
            e = -P["KU1"][s] * mu ** 2 - P["KU2"][s] * mu ** 4 - P["KB1"][s] * mub ** 2
            E["anis"] = E.get("anis", 0.0) + dV * np.where(Ms > 0, e, 0.0).sum()
        if "CUBIC" in terms:
            a, b, c = (_dot(m, P[k][s]) for k in ("ANIS_C1", "ANIS_C2", "ANIS_C3"))
            e = P["KC1"][s] * (a * a * b * b + a * a * c * c + b * b * c * c)
            E["cubic"] = E.get("cubic", 0.0) + dV * np.where(Ms > 0, e, 0.0).sum()
        if "ZEEMAN" in terms:
            E["zeeman"] = E.get("zeeman", 0.0) - dV * (Ms * _dot(m, P["B_EXT"][s])).sum()
        if "MEL" in terms:
            eps = _elastic.strain(u, p.cell)
            exx, eyy, ezz, exy, exz, eyz = eps
            B1, B2 = P["B1"][s], P["B2"][s]
            e = (B1 * (exx * m[0] ** 2 + eyy * m[1] ** 2 + ezz * m[2] ** 2)
                 + 2.0 * B2 * (exy * m[0] * m[1] + exz * m[0] * m[2] + eyz * m[1] * m[2]))
            E["mel"] = E.get("mel", 0.0) + dV * np.where(Ms > 0, e, 0.0).sum()
    if "AFM" in terms and p.n_sub == 2:
        m1, m2 = ms
        Ms1, Ms2 = P["MS"][0], P["MS"][1]
        both = (Ms1 > 0) & (Ms2 > 0)
        A12, A0, a = p.glob["A12"], p.glob["A0"], p.glob["LATTICE_A"]
        e = 0.0
        for axis, spatial in AXES:
            h = p.cell[spatial]
            n1, inside = shift(m1, axis, 1)
            n2, _ = shift(m2, axis, 1)
            b_nb, _ = shift(both.astype(float), axis, 1)
            keep = inside & both & (b_nb > 0)
            e += np.where(keep, ((n1 - m1) * (n2 - m2)).sum(axis=0), 0.0).sum() * A12 / (h * h)
        e -= (4.0 * A0 / (a * a)) * np.where(both, _dot(m1, m2), 0.0).sum()
        E["afm"] = dV * e
    return E
