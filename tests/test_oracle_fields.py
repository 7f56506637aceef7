"""Pins of the oracle's field terms and LLG torque: discrete closed forms
(plane-wave exchange eigenvalue, exact discrete DMI cycloid), the energy
whose gradient each conservative term must be, the boundary condition
against the continuum cycloid, the macrospin LLG solution, and the Kittel
and antiferromagnetic resonance frequencies."""
import numpy as np
import pytest

from inputs import GAMMA, MU0, Problem, config_small
from oracle import demag, fields
from oracle.dp45 import Oracle, State


def _wire(n, axis, D=3e-3, A=1.5e-11, Ms=8e5, h=1e-9, terms=("EXCH", "DMI")):
    shape = [1, 1, 1]
    shape[axis] = n
    p = Problem(tuple(shape), (h, h, h), 1, frozenset(terms))
    p.set("MS", Ms).set("AEX", A).set("DIND", D).set("ALPHA", 0.1)
    return p


def test_uniform_state_has_zero_exchange_field_and_energy():
    w = config_small((6, 5, 4), (2e-9, 3e-9, 1e-9), 3, terms=("EXCH",))
    p = w.problem
    m = np.zeros((3, 4, 5, 6))
    m[0], m[2] = 0.6, 0.8
    B = fields.exchange_field(p, fields.cell_params(p), 0, m)
    assert np.abs(B).max() == 0.0
    assert fields.energies(p, [m])["exch"] == 0.0


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_plane_wave_exchange_eigenvalue(axis):
    n, h, A, Ms = 40, 2e-9, 1.3e-11, 8e5
    p = _wire(n, axis, D=0.0, A=A, Ms=Ms, h=h, terms=("EXCH",))
    k = 2 * np.pi * 5 / (n * h)
    x = np.arange(n) * h
    m = np.zeros((3, n))
    m[0], m[1] = np.cos(k * x), np.sin(k * x)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    m = m.reshape((3,) + tuple(shape))
    B = fields.exchange_field(p, fields.cell_params(p), 0, m).reshape(3, n)
    lam = -(2 * A / Ms) * (2 - 2 * np.cos(k * h)) / h ** 2
    ref = lam * m.reshape(3, n)
    assert np.abs(B[:, 1:-1] - ref[:, 1:-1]).max() <= 1e-12 * abs(lam)


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_discrete_cycloid_field_closed_form(axis, sign):
    """Exchange + interfacial DMI on the cycloid m = (sin qx, 0, cos qx)
    (x along `axis`), interior of a film: the discrete field is B = lam m with
        lam = -(4A/(Ms h^2))(1 - cos qh) - (2D/(Ms h)) sin qh,
    so the energy per cell 2A(1 - cos qh)/h^2 + D sin(qh)/h is lowest at
    tan(qh) = -Dh/(2A) (q -> -D/2A).  Checks the DMI sign and magnitude."""
    n, w, h, A, D, Ms = 24, 5, 1e-9, 1.5e-11, 3e-3, 8e5
    shape = [w, w, 1]
    shape[axis] = n
    p = Problem(tuple(shape), (h, h, h), 1, frozenset({"EXCH", "DMI"}))
    p.set("MS", Ms).set("AEX", A).set("DIND", D)
    q = sign * 0.37 / h
    grid = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]),
                       indexing="ij")
    x = grid[2 - axis] * h
    m = np.zeros((3,) + x.shape)
    m[axis], m[2] = np.sin(q * x), np.cos(q * x)
    B = fields.effective_fields(p, [m])[0]
    lam = -(4 * A / (Ms * h * h)) * (1 - np.cos(q * h)) - (2 * D / (Ms * h)) * np.sin(q * h)
    interior = [slice(None), slice(None), slice(1, -1), slice(1, -1)]
    err = np.abs(B - lam * m)[tuple(interior)].max()
    assert err < 1e-12 * abs(lam), (err, lam)


def test_boundary_condition_matches_continuum_cycloid():
    """d_n m = -(D/2A)(z x n) x m is satisfied by the continuum cycloid
    m = (sin qx, 0, cos qx), q = -D/(2A), at both ends of a wire along x
    and by its y analogue."""
    A, D = 1.5e-11, 3e-3
    q = -D / (2 * A)
    for spatial in (0, 1):
        for x in (0.3e-9, 7.1e-9):
            m = np.zeros(3)
            m[spatial], m[2] = np.sin(q * x), np.cos(q * x)
            dm = np.zeros(3)
            dm[spatial], dm[2] = q * np.cos(q * x), -q * np.sin(q * x)
            for d in (-1, 1):
                g = fields.ghost_derivative(m.reshape(3, 1), np.array([A]), np.array([D]),
                                            spatial, d)[:, 0]
                assert np.allclose(g, d * dm, rtol=1e-14, atol=1e-6)


def _fd_field(energy_fn, ms, s, cell_idx, Ms, dV, h=1e-5):
    """-(1/(Ms dV)) dE/dm by central differences of the energy."""
    out = np.zeros(3)
    for c in range(3):
        plus = [m.copy() for m in ms]
        minus = [m.copy() for m in ms]
        plus[s][(c,) + cell_idx] += h
        minus[s][(c,) + cell_idx] -= h
        out[c] = -(energy_fn(plus) - energy_fn(minus)) / (2 * h) / (Ms * dV)
    return out


@pytest.mark.parametrize("term", ["demag", "exch", "dmi", "anis", "zeeman", "cubic"])
def test_field_is_energy_gradient_ferromagnet(term):
    name = {"demag": "DEMAG", "exch": "EXCH", "dmi": "DMI", "anis": "ANIS",
            "zeeman": "ZEEMAN", "cubic": "CUBIC"}[term]
    terms = (name, "EXCH") if term == "dmi" else (name,)
    w = config_small((7, 6, 3), (2e-9, 2.5e-9, 1e-9), 11, terms=terms, n_regions=2)
    p = w.problem
    P = fields.cell_params(p)
    ms = [w.m0[0].astype(np.float64)]
    noct = demag.tensor_octant(p.shape, p.cell)
    _, parts = fields.effective_fields(p, ms, noct=noct, P=P, parts=True)
    dV = np.prod(p.cell)

    def E(mm):
        return fields.energies(p, mm, noct=noct, P=P)[term]

    for idx in [(0, 1, 1), (1, 3, 4), (2, 4, 5), (1, 2, 2)]:
        ref = _fd_field(E, ms, 0, idx, P["MS"][0][idx], dV)
        got = parts[0][term][(slice(None),) + idx]
        assert np.abs(got - ref).max() <= 1e-6 * max(np.abs(ref).max(), 1e-3), (idx, got, ref)


@pytest.mark.parametrize("term", ["afm", "exch", "mel"])
def test_field_is_energy_gradient_antiferromagnet(term):
    terms = {"afm": ("AFM",), "exch": ("EXCH",), "mel": ("MEL",)}[term]
    w = config_small((7, 6, 2), (2e-9, 2e-9, 2e-9), 5, terms=terms, n_sub=2)
    p = w.problem
    p.set("DIND", 0.0)
    P = fields.cell_params(p)
    ms = [w.m0[s].astype(np.float64) for s in range(2)]
    rng = np.random.default_rng(3)
    u = rng.normal(size=(3, 2, 6, 7)) * 1e-11
    _, parts = fields.effective_fields(p, ms, u=u, P=P, parts=True)
    dV = np.prod(p.cell)

    def E(mm):
        return fields.energies(p, mm, u=u, P=P)[term]

    for s in range(2):
        for idx in [(0, 1, 1), (1, 3, 4), (0, 4, 5)]:
            ref = _fd_field(E, ms, s, idx, P["MS"][s][idx], dV)
            got = parts[s][term][(slice(None),) + idx]
            assert np.abs(got - ref).max() <= 1e-6 * max(np.abs(ref).max(), 1e-3), (s, idx, got, ref)


def test_anisotropy_along_axis():
    p = Problem((1, 1, 1), (1e-9,) * 3, 1, frozenset({"ANIS"}))
    p.set("MS", 1e6).set("KU1", 5e5).set("KU2", 1e5).set("ANIS_U", (0.0, 0.6, 0.8))
    m = np.array([0.0, 0.6, 0.8]).reshape(3, 1, 1, 1)
    B = fields.effective_fields(p, [m])[0].ravel()
    assert np.allclose(B, (2 * 5e5 + 4 * 1e5) / 1e6 * np.array([0.0, 0.6, 0.8]), rtol=1e-15)


def test_torque_perpendicular_and_gyromagnetic():
    rng = np.random.default_rng(1)
    m = rng.normal(size=(3, 50))
    m /= np.linalg.norm(m, axis=0)
    B = rng.normal(size=(3, 50))
    for alpha in (0.0, 0.3):
        t = fields.llg_torque(m, B, alpha)
        assert np.abs((m * t).sum(axis=0)).max() < 1e-15 * GAMMA * np.abs(B).max()
    t0 = fields.llg_torque(m, B, 0.0)
    assert np.allclose(t0, -GAMMA * np.cross(m.T, B.T).T, rtol=1e-14)


def _macrospin(alpha, B, theta0, dt, nsteps):
    p = Problem((1, 1, 1), (1e-9,) * 3, 1, frozenset({"ZEEMAN"}))
    p.set("MS", 8e5).set("ALPHA", alpha).set("B_EXT", (0.0, 0.0, B))
    m0 = np.array([np.sin(theta0), 0.0, np.cos(theta0)]).reshape(3, 1, 1, 1)
    o = Oracle(p)
    st = o.run_fixed(State([m0]), dt, nsteps)
    return st.ms[0].ravel()


def _macrospin_exact(alpha, B, theta0, t):
    g = GAMMA / (1 + alpha ** 2)
    th = 2 * np.arctan(np.tan(theta0 / 2) * np.exp(-alpha * g * B * t))
    ph = g * B * t
    return np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])


def test_macrospin_closed_form_and_fifth_order():
    alpha, B, th0, T = 0.1, 1.0, 0.5, 40e-12
    errs = []
    for n in (40, 80, 160):
        m = _macrospin(alpha, B, th0, T / n, n)
        errs.append(np.abs(m - _macrospin_exact(alpha, B, th0, T)).max())
    assert errs[-1] < 1e-9
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - 5) < 0.6), (errs, slopes)


def _precession_frequency(ms_t, dt):
    ph = np.unwrap(np.arctan2(ms_t[:, 1], ms_t[:, 0]))
    t = np.arange(len(ph)) * dt
    return np.polyfit(t, ph, 1)[0] / (2 * np.pi)


@pytest.mark.parametrize("cell,Bz", [((2e-9, 2e-9, 2e-9), 0.1), ((10e-9, 10e-9, 1e-9), 1.5)])
def test_kittel_frequency(cell, Bz):
    """Uniform mode of one cell in B along z: f = (gamma/2pi)(B - mu0 Ms (Nzz - Nxx))
    with N the cell's self factors (N_xx = N_yy)."""
    Ms, alpha = 8e5, 1e-4
    p = Problem((1, 1, 1), cell, 1, frozenset({"ZEEMAN", "DEMAG"}))
    p.set("MS", Ms).set("ALPHA", alpha).set("B_EXT", (0.0, 0.0, Bz))
    N = demag.cell_tensor(np.zeros(1), np.zeros(1), np.zeros(1), cell)[:, 0]
    f_ref = GAMMA / (2 * np.pi) * (Bz - MU0 * Ms * (N[2] - N[0]))
    dt = 1.0 / f_ref / 200
    o = Oracle(p)
    th = np.deg2rad(1.0)
    st = State([np.array([np.sin(th), 0, np.cos(th)]).reshape(3, 1, 1, 1)])
    traj = []
    st_k = o.rhs(st)
    for n in range(1000):
        st, st_k, _ = o.attempt(st, st_k, dt)
        traj.append(st.ms[0].ravel())
    f = _precession_frequency(np.array(traj), dt)
    assert abs(f / f_ref - 1) < 1e-3, (f, f_ref)


def test_antiferromagnetic_resonance_frequency():
    """Uniform antiparallel state, easy axis z, homogeneous AFM exchange only:
    f = (gamma/2pi) sqrt(B_K (2 B_E + B_K)), B_E = 4|A0|/(Ms a^2), B_K = 2K/Ms."""
    Ms, K, A0, a = 4e5, 1e5, -4e-11, 0.42e-9
    p = Problem((1, 1, 1), (2e-9,) * 3, 2, frozenset({"ANIS", "AFM"}))
    p.set("MS", Ms).set("ALPHA", 0.0).set("KU1", K).set("ANIS_U", (0.0, 0.0, 1.0))
    p.glob.update(A0=A0, A12=-1e-12, LATTICE_A=a)
    BE, BK = 4 * abs(A0) / (Ms * a * a), 2 * K / Ms
    f_ref = GAMMA / (2 * np.pi) * np.sqrt(BK * (2 * BE + BK))
    th = np.deg2rad(0.5)
    m1 = np.array([np.sin(th), 0, np.cos(th)]).reshape(3, 1, 1, 1)
    m2 = -m1
    o = Oracle(p)
    dt = 1.0 / (GAMMA * BE / (2 * np.pi)) / 60
    st = State([m1, m2])
    k = o.rhs(st)
    lx, times = [], []
    nsteps = int(6.0 / f_ref / dt)
    for n in range(nsteps):
        st, k, _ = o.attempt(st, k, dt)
        lx.append((st.ms[0] - st.ms[1]).ravel()[0])
    lx = np.array(lx)
    t = (np.arange(nsteps) + 1) * dt
    idx = np.where((lx[:-1] < 0) & (lx[1:] >= 0))[0]
    tc = t[idx] - lx[idx] * dt / (lx[idx + 1] - lx[idx])
    f = (len(tc) - 1) / (tc[-1] - tc[0])
    assert abs(f / f_ref - 1) < 1e-3, (f, f_ref)


def test_energy_decreases_with_damping():
    w = config_small((12, 10, 1), (3e-9, 3e-9, 3e-9), 21,
                     terms=("DEMAG", "EXCH", "ZEEMAN", "ANIS"))
    p = w.problem
    p.set("ALPHA", 0.5).set("DIND", 0.0)
    o = Oracle(p)
    st = State(w.m0)
    k = o.rhs(st)
    E = []
    for n in range(40):
        st, k, _ = o.attempt(st, k, 2e-14)
        E.append(sum(fields.energies(p, st.ms, noct=o.noct).values()))
    assert np.all(np.diff(E) < 0), np.diff(E)


def test_cubic_anisotropy_closed_forms():
    """Cubic anisotropy: no field along a cubic axis, and along the body
    diagonal (c1 + c2 + c3)/sqrt(3) the field -(4 Kc1 / (3 Ms)) m, for rotated
    axes."""
    p = Problem((2, 1, 1), (1e-9,) * 3, 1, frozenset({"CUBIC"}))
    Ms, K = 8e5, 3e4
    rot = np.array([[0.36, 0.48, -0.8], [-0.8, 0.6, 0.0], [0.48, 0.64, 0.6]])   # orthogonal
    c1, c2, c3 = rot
    p.set("MS", Ms).set("KC1", K).set("ANIS_C1", tuple(c1)).set("ANIS_C2", tuple(c2))
    P = fields.cell_params(p)
    assert np.allclose(P["ANIS_C3"][0][:, 0, 0, 0], np.cross(c1, c2))
    diag = (c1 + c2 + c3) / np.sqrt(3.0)
    m = np.stack([c2, diag], axis=1).reshape(3, 1, 1, 2)
    B = fields.cubic_anisotropy_field(p, P, 0, m)
    assert np.abs(B[:, 0, 0, 0]).max() < 1e-12
    assert np.allclose(B[:, 0, 0, 1], -(4.0 * K / (3.0 * Ms)) * diag, rtol=1e-12, atol=0)


def _open_problem(seed, terms=("EXCH", "DMI"), empty=0.2):
    w = config_small((5, 4, 2), (2e-9, 2.5e-9, 1e-9), seed, terms=terms, n_regions=2, empty_fraction=empty)
    w.problem.open_bc = True
    return w


@pytest.mark.parametrize("term", ["exch", "dmi"])
def test_open_boundary_field_is_energy_gradient_everywhere(term):
    """With the open boundary a missing neighbour drops out of the pair sums,
    so at every magnetic cell -- corners, edges and faces towards empty cells
    included -- the field is the negative gradient of the pair energy."""
    w = _open_problem(31)
    p = w.problem
    P = fields.cell_params(p)
    ms = [w.m0[0].astype(np.float64)]
    _, parts = fields.effective_fields(p, ms, P=P, parts=True)
    dV = np.prod(p.cell)

    def E(mm):
        return fields.energies(p, mm, P=P)[term]

    nx, ny, nz = p.shape
    checked = 0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                idx = (z, y, x)
                if P["MS"][0][idx] == 0:
                    continue
                ref = _fd_field(E, ms, 0, idx, P["MS"][0][idx], dV)
                got = parts[0][term][(slice(None),) + idx]
                assert np.abs(got - ref).max() <= 1e-6 * max(np.abs(ref).max(), 1e-3), (idx, got, ref)
                checked += 1
    assert checked >= 25


def test_open_boundary_two_cell_wire_closed_form():
    """Two cells along x (or y), open ends: each cell sees only the other,
    B_exch = (2A/Ms)(m' - m)/h^2 and B_dmi = (D/(Ms h)) s (m'_z e_a - m'_a e_z)
    with s = +1 for the neighbour at +h, -1 at -h."""
    A, D, Ms, h = 1.5e-11, 3e-3, 8e5, 1e-9
    for axis in (0, 1):
        p = _wire(2, axis, D=D, A=A, Ms=Ms, h=h)
        p.open_bc = True
        rng = np.random.default_rng(7 + axis)
        m = rng.normal(size=(3, 2))
        m /= np.linalg.norm(m, axis=0)
        shape = [1, 1, 1]
        shape[axis] = 2
        ms = [m.reshape((3,) + tuple(shape[::-1]))]
        _, parts = fields.effective_fields(p, ms, parts=True)
        ex = parts[0]["exch"].reshape(3, 2)
        dm = parts[0]["dmi"].reshape(3, 2)
        for c, s in ((0, 1), (1, -1)):
            o = 1 - c
            assert np.allclose(ex[:, c], 2 * A / Ms * (m[:, o] - m[:, c]) / h ** 2, rtol=1e-13)
            want = np.zeros(3)
            want[axis] = s * D * m[2, o] / (Ms * h)
            want[2] = -s * D * m[axis, o] / (Ms * h)
            assert np.allclose(dm[:, c], want, rtol=1e-13, atol=1e-12)


def test_open_and_neumann_boundaries():
    """Without DMI the two conditions give the same field everywhere; with
    DMI they agree away from the boundary and differ at x/y boundary cells."""
    for terms, same in ((("EXCH",), True), (("EXCH", "DMI"), False)):
        w = config_small((6, 5, 2), (2e-9, 2e-9, 1e-9), 41, terms=terms)
        p = w.problem
        ms = [w.m0[0].astype(np.float64)]
        Bn = fields.effective_fields(p, ms)[0]
        p.open_bc = True
        Bo = fields.effective_fields(p, ms)[0]
        if same:
            assert np.array_equal(Bn, Bo)
        else:
            inner = (slice(None), slice(None), slice(1, -1), slice(1, -1))
            assert np.allclose(Bn[inner], Bo[inner], rtol=1e-14, atol=0)
            edge = np.abs(Bn - Bo).max(axis=0)
            assert edge[:, 0, :].min() > 0 and edge[:, :, 0].min() > 0
