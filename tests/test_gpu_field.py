"""Parity of one field + torque evaluation of the CUDA path (through the
C-ABI) with the FP64 oracle, element by element, on seeded inputs.

Sizes span several x/y tiles with ragged tails, padded lengths 2^k and
3*2^k up to the largest supported (4096 along x and along y), the pass-B
cluster split of large ky planes (R = 2, 4), the fixed and generic z
transforms (nz = 1, 2, 4, 8, and 3 and 16), axes of one cell, several regions
with empty cells, and the two-sublattice magnetoelastic path."""
import numpy as np
import pytest

from inputs import MU0, config_small, random_unit_vectors
from gpu_util import field_tolerance, torque_tolerance, make_magnet, gpu_eval, oracle_eval

pytestmark = pytest.mark.gpu

FM = ("DEMAG", "EXCH", "ANIS", "DMI", "ZEEMAN")

CASES = [
    # shape, cell, seed, terms, regions, empty fraction
    ((5, 4, 3), (2e-9, 3e-9, 1.5e-9), 1, FM, 1, 0.0),
    ((17, 9, 1), (2e-9, 2e-9, 2e-9), 2, FM, 1, 0.0),
    ((24, 20, 2), (3e-9, 2e-9, 1e-9), 3, FM, 3, 0.1),
    ((64, 64, 1), (4e-9, 4e-9, 4e-9), 4, ("DEMAG", "EXCH", "ZEEMAN"), 1, 0.0),
    ((33, 19, 8), (2e-9, 2e-9, 1e-9), 5, FM, 1, 0.0),
    ((16, 300, 8), (2e-9, 2e-9, 1e-9), 6, FM, 1, 0.0),      # ky split R = 2
    ((8, 600, 4), (2e-9, 2e-9, 1e-9), 7, FM, 2, 0.0),       # R = 2, Py = 1536
    ((4, 1100, 4), (2e-9, 2e-9, 2e-9), 8, FM, 1, 0.0),      # R = 4, Py = 3072
    ((10, 6, 3), (2e-9, 2e-9, 1e-9), 9, FM, 1, 0.0),        # generic nz
    ((1, 1, 1), (3e-9, 3e-9, 3e-9), 10, FM, 1, 0.0),
    ((1, 7, 1), (2e-9, 2e-9, 2e-9), 11, FM, 1, 0.0),
    ((9, 1, 2), (2e-9, 2e-9, 2e-9), 12, FM, 1, 0.0),
    ((40, 12, 1), (2e-9, 2e-9, 2e-9), 13, ("EXCH", "DMI", "ANIS"), 4, 0.15),   # no demag
    ((2048, 3, 2), (2e-9, 2e-9, 1e-9), 14, FM, 1, 0.0),     # largest padded x length, 4096
    ((3, 2048, 2), (2e-9, 2e-9, 1e-9), 15, FM, 1, 0.0),     # largest padded y length, 4096
    ((6, 5, 16), (2e-9, 2e-9, 1e-9), 16, FM, 2, 0.05),      # largest nz with demag (generic z DFT, Pz = 32)
]


@pytest.mark.parametrize("shape,cell,seed,terms,nreg,empty", CASES,
                         ids=["x".join(map(str, c[0])) + "-%d" % c[2] for c in CASES])
def test_field_and_torque_parity(shape, cell, seed, terms, nreg, empty):
    w = config_small(shape, cell, seed, terms=terms, n_regions=nreg, empty_fraction=empty)
    p = w.problem
    mag = make_magnet(p, w.m0)
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0)
    tolB = field_tolerance(p, Bo[0])
    assert np.all(np.abs(Bg[0] - Bo[0]) <= tolB), np.abs(Bg[0] - Bo[0]).max()
    tolT = torque_tolerance(p, Bo[0], tolB)
    assert np.all(np.abs(Tg[0] - To[0]) <= tolT), np.abs(Tg[0] - To[0]).max()
    mag.close()


# Grids whose pass B runs on the warp-level transforms (folded y length
# Py / R of 256, 512 or 1024, nz of 1, 2, 4 or 8): shape, cell, seed, terms,
# regions, empty fraction, expected R of the default shape.
WARP_CASES = [
    ((5, 120, 2), (2e-9, 2e-9, 1e-9), 51, FM, 1, 0.0, 1),      # Py = 256, one CTA per plane
    ((6, 200, 1), (2e-9, 2e-9, 2e-9), 52, FM, 2, 0.05, 1),     # Py = 512, nz = 1, regions and empty cells
    ((4, 400, 4), (2e-9, 2e-9, 1e-9), 53, FM, 1, 0.0, 1),      # Py = 1024, nz = 4
    ((3, 1000, 8), (2e-9, 2e-9, 1e-9), 54, FM, 1, 0.0, 2),     # Py = 2048: a two-CTA cluster per plane, ragged ny
    ((2, 777, 2), (2e-9, 2e-9, 1e-9), 55, FM, 3, 0.1, 2),      # odd ny (8-byte copies), three regions
]


@pytest.mark.parametrize("shape,cell,seed,terms,nreg,empty,R", WARP_CASES,
                         ids=["x".join(map(str, c[0])) + "-%d" % c[2] for c in WARP_CASES])
def test_warp_pass_b_parity(shape, cell, seed, terms, nreg, empty, R):
    """The warp-level pass B (one warp per y column, in-register DFTs, one
    shared-memory transpose; z transform + kernel multiply per ky in
    registers) is the default where it applies; field and torque against
    the oracle, element by element."""
    w = config_small(shape, cell, seed, terms=terms, n_regions=nreg, empty_fraction=empty)
    p = w.problem
    mag = make_magnet(p, w.m0)
    sh = mag.get_shape()
    assert sh["engine"] == 1 and sh["R"] == R, sh
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0)
    tolB = field_tolerance(p, Bo[0])
    assert np.all(np.abs(Bg[0] - Bo[0]) <= tolB), np.abs(Bg[0] - Bo[0]).max()
    assert np.all(np.abs(Tg[0] - To[0]) <= torque_tolerance(p, Bo[0], tolB)), np.abs(Tg[0] - To[0]).max()
    mag.close()


# Grids whose passes A and C run on the warp-level x transforms (Px = 2048,
# nx of 769 .. 1024): shape, cell, seed, terms, regions, empty fraction.
WARPX_CASES = [
    ((1000, 6, 2), (2e-9, 2e-9, 1e-9), 61, FM, 1, 0.0),      # 16-byte stage loads (nx % 4 == 0)
    ((999, 5, 1), (2e-9, 2e-9, 2e-9), 62, FM, 2, 0.05),     # odd nx (one cell per load), odd ny (last pair of one row)
    ((1024, 7, 3), (2e-9, 2e-9, 1e-9), 63, FM, 3, 0.1),     # nx = N exactly, generic z, regions and empty cells
    ((800, 120, 2), (2e-9, 2e-9, 1e-9), 64, FM, 1, 0.0),    # with the warp pass B as well
]


@pytest.mark.parametrize("shape,cell,seed,terms,nreg,empty", WARPX_CASES,
                         ids=["x".join(map(str, c[0])) + "-%d" % c[2] for c in WARPX_CASES])
def test_warp_x_passes_parity(shape, cell, seed, terms, nreg, empty):
    """Passes A and C on the warp-level x transforms (tiles of one row pair:
    the even and odd halves of the padded transform, one warp each per
    component) are the default for Px = 2048; field and torque against the
    oracle, element by element."""
    w = config_small(shape, cell, seed, terms=terms, n_regions=nreg, empty_fraction=empty)
    p = w.problem
    mag = make_magnet(p, w.m0)
    assert mag.get_shape()["engine"] & 2
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0)
    tolB = field_tolerance(p, Bo[0])
    assert np.all(np.abs(Bg[0] - Bo[0]) <= tolB), np.abs(Bg[0] - Bo[0]).max()
    assert np.all(np.abs(Tg[0] - To[0]) <= torque_tolerance(p, Bo[0], tolB)), np.abs(Tg[0] - To[0]).max()
    mag.close()


# Pass C's four-cell stencil (one sublattice, uniform material, nx a
# multiple of 4, tile rows of m staged in shared memory): shape, cell, seed,
# terms, open boundary.  The DMI ghosts at every x and y edge, the open
# boundary, a last tile of one row (odd ny), nx = N exactly (the last item
# has no right neighbour), cubic anisotropy and the magnetoelastic field.
STENCIL4_CASES = [
    ((1000, 5, 3), (2e-9, 2e-9, 1e-9), 71, FM, False),
    ((1000, 6, 2), (3e-9, 2e-9, 1e-9), 72, FM, True),
    ((1024, 4, 2), (2e-9, 2e-9, 1e-9), 73, ("DEMAG", "EXCH", "CUBIC", "ZEEMAN"), False),
    ((1024, 3, 1), (2e-9, 3e-9, 2e-9), 74, ("DEMAG", "EXCH", "ANIS", "DMI", "MEL", "ELASTIC"), False),
]


@pytest.mark.parametrize("shape,cell,seed,terms,open_bc", STENCIL4_CASES,
                         ids=["x".join(map(str, c[0])) + "-%d" % c[2] for c in STENCIL4_CASES])
def test_warp_x_four_cell_stencil_parity(shape, cell, seed, terms, open_bc):
    w = config_small(shape, cell, seed, terms=terms)
    p = w.problem
    p.open_bc = open_bc
    u = None
    if "ELASTIC" in terms:
        nx, ny, nz = shape
        u = (np.random.default_rng(seed).normal(size=(3, nz, ny, nx)) * 2e-12).astype(np.float32)
    mag = make_magnet(p, w.m0, u, None if u is None else np.zeros_like(u))
    assert mag.get_shape()["engine"] & 2
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0, u)
    tolB = field_tolerance(p, Bo[0])
    assert np.all(np.abs(Bg[0] - Bo[0]) <= tolB), np.abs(Bg[0] - Bo[0]).max()
    assert np.all(np.abs(Tg[0] - To[0]) <= torque_tolerance(p, Bo[0], tolB)), np.abs(Tg[0] - To[0]).max()
    mag.close()


def test_warp_x_two_sublattice_magnetoelastic_parity():
    """The two-sublattice magnetoelastic path on the warp x passes (summed M
    in pass A, both sublattices' local fields in pass C)."""
    w = config_small((1024, 4, 1), (2e-9, 2e-9, 2e-9), 65, n_sub=2,
                     terms=("DEMAG", "EXCH", "ANIS", "AFM", "MEL", "ELASTIC", "ZEEMAN"))
    p = w.problem
    p.set("DIND", 0.0)
    rng = np.random.default_rng(6)
    u = (rng.normal(size=(3, 1, 4, 1024)) * 2e-12).astype(np.float32)
    mag = make_magnet(p, w.m0, u, np.zeros_like(u))
    assert mag.get_shape()["engine"] & 2
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0, u)
    for s in range(2):
        tolB = field_tolerance(p, Bo[s], s)
        assert np.all(np.abs(Bg[s] - Bo[s]) <= tolB), (s, np.abs(Bg[s] - Bo[s]).max())
        assert np.all(np.abs(Tg[s] - To[s]) <= torque_tolerance(p, Bo[s], tolB)), s
    mag.close()


def test_warp_x_trajectory_matches_oracle_and_block_engine():
    """Stage assembly (including the renormalised last stage) runs in the
    warp pass A: 20 fixed Dormand-Prince steps against the oracle, and the
    same steps on the block engine agree to FP32 rounding."""
    import torch
    from oracle.dp45 import Oracle, State
    w = config_small((1000, 6, 2), (2e-9, 2e-9, 1e-9), 66, terms=FM)
    p = w.problem
    dt = 2e-14
    out = []
    for engine in (2, 0):
        mag = make_magnet(p, w.m0)
        if engine != 2:
            mag.set_shape(engine=engine)
        assert mag.get_shape()["engine"] == engine
        mag.set_solver(adaptive=False, dt=dt)
        mag.step(20)
        m = torch.empty((3,) + p.shape[::-1], dtype=torch.float32, device="cuda")
        mag.get_m(0, m)
        out.append(m.cpu().numpy().astype(np.float64))
        mag.close()
    st = Oracle(p).run_fixed(State([m.astype(np.float64) for m in w.m0]), dt, 20)
    assert np.abs(out[0] - st.ms[0]).max() <= 1e-4
    assert np.abs(out[0] - out[1]).max() <= 1e-5


def test_two_sublattice_magnetoelastic_parity():
    w = config_small((23, 18, 1), (2e-9, 2e-9, 2e-9), 31, n_sub=2,
                     terms=("DEMAG", "EXCH", "ANIS", "AFM", "MEL", "ELASTIC", "ZEEMAN"))
    p = w.problem
    p.set("DIND", 0.0)
    rng = np.random.default_rng(5)
    u = (rng.normal(size=(3, 1, 18, 23)) * 2e-12).astype(np.float32)
    v = np.zeros_like(u)
    mag = make_magnet(p, w.m0, u, v)
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0, u)
    for s in range(2):
        tolB = field_tolerance(p, Bo[s], s)
        assert np.all(np.abs(Bg[s] - Bo[s]) <= tolB), (s, np.abs(Bg[s] - Bo[s]).max())
        tolT = torque_tolerance(p, Bo[s], tolB)
        assert np.all(np.abs(Tg[s] - To[s]) <= tolT), (s, np.abs(Tg[s] - To[s]).max())
    mag.close()


def test_large_random_exchange_field_within_bar():
    """Random m on 2x2x1 nm cells with A = 1.6e-11 gives |B_exch| up to
    ~1.7e2 T; the double-float exchange sum keeps the error under the
    1e-5 mu0 Ms bar (which is below one FP32 ulp of such fields)."""
    w = config_small((40, 36, 8), (2e-9, 2e-9, 1e-9), 41, terms=("EXCH", "DMI", "ANIS", "DEMAG"))
    p = w.problem
    p.set("MS", 1.1e6).set("AEX", 1.6e-11).set("DIND", 3e-3).set("KU1", 8e5).set("KU2", 0.0)
    p.set("KB1", 0.0).set("ANIS_U", (0.0, 0.0, 1.0))
    mag = make_magnet(p, w.m0)
    Bg, _ = gpu_eval(mag, p)
    Bo, _ = oracle_eval(p, w.m0)
    from inputs import MU0
    bar = 1e-5 * MU0 * 1.1e6
    assert np.abs(Bo[0]).max() > 100.0
    assert np.abs(Bg[0] - Bo[0]).max() <= bar
    mag.close()


def test_radix3_x_length_at_full_tile_capacity():
    """nx = 1025 pads to Px = 3072 = 3 * 2^10, so every x transform ends with
    a radix-3 pass, which holds a third fewer values per thread than the
    power-of-two passes (pass A: 15 instead of 16).  With ny = 152, nz = 16
    the tiles hold 4 rows (pass A's capacity rules out 8), so pass A
    transforms 2 row pairs of 3072 points: 6144 values, more than 15 per
    thread of the 384-thread block a 16-value sizing would give.  Sampled
    cells against the oracle's direct sum of the demag definition plus its
    local terms."""
    from oracle import demag, fields
    from inputs import Problem
    p = Problem((1025, 152, 16), (3e-9, 3e-9, 2e-9), 1, frozenset({"DEMAG", "EXCH"}))
    p.set("MS", 8e5).set("AEX", 1.3e-11)
    m0 = random_unit_vectors(515, p.shape)
    mag = make_magnet(p, [m0])
    assert mag.get_shape()["ty"] == 4      # pass A capacity: 4 row pairs of 3072 exceed 15 x 512
    Bg, _ = gpu_eval(mag, p)
    mag.close()
    nx, ny, nz = p.shape
    m = m0.astype(np.float64)
    noct = demag.tensor_octant(p.shape, p.cell)
    P = fields.cell_params(p)
    local = sum(fields.effective_fields(
        Problem(p.shape, p.cell, 1, frozenset({"EXCH"}), p.regions, p.scal, p.vec, p.glob), [m], P=P))
    picks = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (1024, 3, 8), (513, 76, 15), (700, 151, 0), (2, 100, 7)]
    cells = [x + nx * (y + ny * z) for x, y, z in picks]
    Bd = demag.demag_direct(p.shape, p.cell, P["MS"][0] * m, noct=noct, cells=cells)
    bar = 1e-5 * MU0 * 8e5
    for (x, y, z), bd in zip(picks, Bd.T):
        ref = bd + local[:, z, y, x]
        assert np.abs(Bg[0][:, z, y, x] - ref).max() <= bar, ((x, y, z), Bg[0][:, z, y, x], ref)


def test_ferrimagnet_unequal_sublattices():
    """A ferrimagnet (the paper's two-sublattice formalism with unequal
    sublattices, Methods): Ms, A and damping differ per sublattice; demag
    acts on the summed M.  Field parity for both sublattices and a 20-step
    fixed-dt trajectory against the oracle."""
    import torch
    from oracle.dp45 import Oracle, State
    w = config_small((24, 20, 2), (2e-9, 2e-9, 1e-9), 123,
                     terms=("DEMAG", "EXCH", "ANIS", "AFM", "ZEEMAN"), n_sub=2)
    p = w.problem
    p.set("MS", 6e5, 0).set("MS", 3.5e5, 1)
    ms = p.scal["MS"][:, 0]
    assert ms[0] / ms[1] > 1.5
    mag = make_magnet(p, w.m0)
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, [m.astype(np.float64) for m in w.m0])
    for s in range(2):
        assert np.all(np.abs(Bg[s] - Bo[s]) <= field_tolerance(p, Bo[s], s)), s
    dt = 2e-15
    mag.set_solver(adaptive=False, dt=dt)
    mag.step(20)
    st = Oracle(p).run_fixed(State(w.m0), dt, 20)
    for s in range(2):
        out = torch.empty((3,) + p.shape[::-1], dtype=torch.float32, device="cuda")
        mag.get_m(s, out)
        assert np.abs(out.cpu().numpy() - st.ms[s]).max() <= 1e-4, s
    mag.close()


def test_cubic_anisotropy_parity():
    """Cubic anisotropy (non-orthogonal input axes, made orthonormal by both
    codes), two regions with their own axes and constants, with demag,
    exchange and Zeeman: field and torque against the oracle."""
    w = config_small((24, 20, 3), (2e-9, 2e-9, 1e-9), 131, terms=("DEMAG", "EXCH", "CUBIC", "ZEEMAN"),
                     n_regions=2)
    p = w.problem
    assert np.abs(p.scal["KC1"][0, :2]).min() > 0
    mag = make_magnet(p, w.m0)
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, [w.m0[0].astype(np.float64)])
    tol = field_tolerance(p, Bo[0])
    assert np.all(np.abs(Bg[0] - Bo[0]) <= tol), np.abs(Bg[0] - Bo[0]).max()
    assert np.all(np.abs(Tg[0] - To[0]) <= torque_tolerance(p, Bo[0], tol))
    mag.close()


def test_every_launch_shape_matches_oracle():
    """Every valid launch shape (pass-B engine, residue classes R, kernel
    staging, y plan; pass A/C tile rows) gives the same field within the
    bar: the shape changes only the FP32 rounding order."""
    import itertools
    from paper_2411_18194_gb300 import MmpError
    w = config_small((24, 256, 8), (2e-9, 2e-9, 1e-9), 21, terms=FM)
    p = w.problem
    mag = make_magnet(p, w.m0)
    Bo, To = oracle_eval(p, w.m0)
    tolB = field_tolerance(p, Bo[0])
    tolT = torque_tolerance(p, Bo[0], tolB)
    seen = []
    for eng, R, st, ry, (ty, tyc) in itertools.product((0, 1), (1, 2, 4, 8), (0, 1), (0, 1),
                                                       ((8, 0), (2, 4), (4, 8))):
        try:
            mag.set_shape(engine=eng, R=R, stage_kernel=st, radix_y=ry, ty=ty, tyc=tyc)
        except MmpError:
            continue
        seen.append((eng, R))
        Bg, Tg = gpu_eval(mag, p)
        assert np.all(np.abs(Bg[0] - Bo[0]) <= tolB), (eng, R, st, ry, ty, tyc, np.abs(Bg[0] - Bo[0]).max())
        assert np.all(np.abs(Tg[0] - To[0]) <= tolT), (eng, R, st, ry, ty, tyc)
    assert set(seen) == {(0, 1), (0, 2), (0, 4), (0, 8), (1, 1), (1, 2)}
    mag.close()


def test_open_boundary_parity():
    """Open boundary (missing neighbours drop out of the exchange and DMI
    sums) with DMI, several regions and empty cells; the Neumann field of
    the same state differs at the boundary, so the switch is live."""
    w = config_small((24, 20, 2), (3e-9, 2e-9, 1e-9), 23, terms=FM, n_regions=3, empty_fraction=0.1)
    p = w.problem
    p.open_bc = True
    mag = make_magnet(p, w.m0)
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0)
    tolB = field_tolerance(p, Bo[0])
    assert np.all(np.abs(Bg[0] - Bo[0]) <= tolB), np.abs(Bg[0] - Bo[0]).max()
    tolT = torque_tolerance(p, Bo[0], tolB)
    assert np.all(np.abs(Tg[0] - To[0]) <= tolT), np.abs(Tg[0] - To[0]).max()
    mag.set_boundary("neumann")
    Bn, _ = gpu_eval(mag, p)
    assert np.abs(Bn[0] - Bg[0]).max() > 100 * tolB.max()
    mag.close()


def test_all_cells_empty():
    """Degenerate magnet with no magnetic cell: zero field and torque, and
    fixed steps leave the state unchanged (to FP32 renormalisation)."""
    import torch
    w = config_small((12, 9, 2), (2e-9, 2e-9, 1e-9), 61, terms=FM, empty_fraction=1.0)
    p = w.problem
    assert np.all(p.scal["MS"][0][p.regions] == 0)
    mag = make_magnet(p, w.m0)
    Bg, Tg = gpu_eval(mag, p)
    assert np.all(Bg[0] == 0) and np.all(Tg[0] == 0)
    mag.set_solver(adaptive=False, dt=1e-13)
    mag.step(3)
    out = torch.empty((3,) + p.shape[::-1], dtype=torch.float32, device="cuda")
    mag.get_m(0, out)
    m = out.cpu().numpy()
    assert np.all(np.isfinite(m)) and np.allclose(m, w.m0[0], rtol=0, atol=1e-6)
    mag.close()


@pytest.mark.parametrize("open_bc", [False, True])
def test_single_magnetic_cell(open_bc):
    """One magnetic cell inside an empty grid: all six neighbours missing,
    so exchange and DMI see only the boundary condition and the demag field
    is the cell's self term."""
    w = config_small((9, 7, 3), (2e-9, 3e-9, 1e-9), 62, terms=FM)
    p = w.problem
    p.regions[...] = 255
    p.regions[1, 3, 4] = 0
    p.set("MS", 0.0, None, 255)
    p.open_bc = open_bc
    mag = make_magnet(p, w.m0)
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0)
    tolB = field_tolerance(p, Bo[0])
    assert np.all(np.abs(Bg[0] - Bo[0]) <= tolB), np.abs(Bg[0] - Bo[0]).max()
    assert np.all(np.abs(Tg[0] - To[0]) <= torque_tolerance(p, Bo[0], tolB))
    assert np.count_nonzero(np.abs(Bo[0]).sum(axis=0)) == 1
    mag.close()
