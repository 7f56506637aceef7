"""Problem description and the named synthetic workloads.

A `Problem` is the statement the paper gives for one magnet: a regular grid
and cell size, one or two sublattices, material parameters per region (a
uint8 region map selects the row of a 256-entry table), global
antiferromagnetic and elastic constants, and the set of field terms.  It
holds parameter values only; each consumer (the oracle, the C-ABI binding)
expands them itself.
"""
from dataclasses import dataclass, field
import numpy as np

from .rng import random_unit_vectors, noisy_axis_vectors, uniform01, splitmix64

# Constants shared by both implementations (SI units).
GAMMA = 1.7595e11          # gyromagnetic ratio, rad s^-1 T^-1
MU0 = 4e-7 * np.pi         # vacuum permeability, T m / A

N_REGIONS = 256

# Per-sublattice, per-region scalar and vector parameters.
PARAM_SCALARS = ("MS", "AEX", "ALPHA", "KU1", "KU2", "KB1", "DIND", "B1", "B2", "KC1")
PARAM_VECTORS = ("ANIS_U", "ANIS_UB", "B_EXT", "ANIS_C1", "ANIS_C2")
GLOBALS = ("A0", "A12", "LATTICE_A", "C11", "C12", "C44", "RHO", "ETA")
TERMS = ("DEMAG", "EXCH", "ANIS", "DMI", "ZEEMAN", "AFM", "MEL", "ELASTIC", "CUBIC")


@dataclass
class Problem:
    shape: tuple                      # (nx, ny, nz)
    cell: tuple                       # (dx, dy, dz) in metres
    n_sub: int = 1
    terms: frozenset = frozenset()
    regions: np.ndarray = None        # uint8 [nz][ny][nx]; None means all region 0
    scal: dict = field(default_factory=dict)   # name -> float64 [n_sub][256]
    vec: dict = field(default_factory=dict)    # name -> float64 [n_sub][256][3]
    glob: dict = field(default_factory=dict)   # name -> float
    open_bc: bool = False             # open boundary (missing neighbours drop out) instead of Neumann

    def __post_init__(self):
        for k in PARAM_SCALARS:
            self.scal.setdefault(k, np.zeros((self.n_sub, N_REGIONS)))
        for k in PARAM_VECTORS:
            v = np.zeros((self.n_sub, N_REGIONS, 3))
            if k == "ANIS_U":
                v[..., 2] = 1.0
            if k in ("ANIS_UB", "ANIS_C1"):
                v[..., 0] = 1.0
            if k == "ANIS_C2":
                v[..., 1] = 1.0
            self.vec.setdefault(k, v)
        for k in GLOBALS:
            self.glob.setdefault(k, 0.0)
        if self.regions is None:
            nx, ny, nz = self.shape
            self.regions = np.zeros((nz, ny, nx), dtype=np.uint8)
        self.terms = frozenset(self.terms)

    # convenience setters -------------------------------------------------
    def set(self, name, value, sub=None, region=None):
        subs = range(self.n_sub) if sub is None else [sub]
        regs = slice(None) if region is None else region
        for s in subs:
            if name in self.scal:
                self.scal[name][s, regs] = value
            else:
                self.vec[name][s, regs] = np.asarray(value, dtype=np.float64)
        return self

    @property
    def n_cells(self):
        nx, ny, nz = self.shape
        return nx * ny * nz


@dataclass
class Workload:
    """A problem plus its initial state and solver settings."""
    name: str
    problem: Problem
    m0: list                          # per sublattice float32 [3][nz][ny][nx]
    u0: np.ndarray = None             # float32 [3][nz][ny][nx] or None
    v0: np.ndarray = None
    adaptive: bool = False
    dt: float = 1e-13
    tol: float = 1e-5
    steps: int = 0
    duration: float = 0.0
    dt_min: float = 1e-18
    dt_max: float = 1e-11
    seed: int = 0


BASE_SEED = 20241127


def config_c1():
    """Plain ferromagnet 64x64x1, 4 nm cubes; demag + exchange + Zeeman;
    2000 fixed DP45 steps at dt = 1e-13 s."""
    p = Problem((64, 64, 1), (4e-9, 4e-9, 4e-9), 1,
                frozenset({"DEMAG", "EXCH", "ZEEMAN"}))
    p.set("MS", 8e5).set("AEX", 1.3e-11).set("ALPHA", 0.02)
    p.set("B_EXT", (0.0, 0.0, 0.01))
    seed = BASE_SEED + 0
    return Workload("ferromagnet 64x64x1 (4 nm cells), demag+exchange+Zeeman, "
                    "2000 fixed DP45 steps", p,
                    [random_unit_vectors(seed, p.shape)], adaptive=False,
                    dt=1e-13, steps=2000, seed=seed)


def config_c2():
    """Large ferromagnet 1024x1024x8, 2x2x1 nm cells; demag + exchange +
    uniaxial anisotropy along z + interfacial DMI; adaptive DP45 to 200 ps."""
    p = Problem((1024, 1024, 8), (2e-9, 2e-9, 1e-9), 1,
                frozenset({"DEMAG", "EXCH", "ANIS", "DMI"}))
    p.set("MS", 1.1e6).set("AEX", 1.6e-11).set("ALPHA", 0.1)
    p.set("KU1", 8e5).set("ANIS_U", (0.0, 0.0, 1.0)).set("DIND", 3e-3)
    seed = BASE_SEED + 1
    return Workload("ferromagnet 1024x1024x8 (2x2x1 nm cells), demag+exchange+"
                    "anisotropy+iDMI, adaptive DP45 (tol 1e-5) for 200 ps", p,
                    [random_unit_vectors(seed, p.shape)], adaptive=True,
                    dt=1e-14, tol=1e-5, duration=200e-12, seed=seed)


def config_c3():
    """Two-sublattice antiferromagnet 1024x256x1, 2 nm cubes, with
    magnetoelastic coupling and elastodynamics; fixed dt 5e-15 s for 100 ps.

    Values the workload statement leaves open are fixed here: biaxial
    anisotropy = easy x (K = 8.57e4 J/m^3) + hard z (K = -8.57e5 J/m^3),
    lattice constant a = 0.42 nm, alpha = 0.01, B_ext = 0, eta = 0.
    """
    shape = (1024, 256, 1)
    p = Problem(shape, (2e-9, 2e-9, 2e-9), 2,
                frozenset({"DEMAG", "EXCH", "ANIS", "AFM", "MEL", "ELASTIC"}))
    p.set("MS", 4e5).set("AEX", 1e-11).set("ALPHA", 0.01)
    p.set("KU1", 8.57e4).set("ANIS_U", (1.0, 0.0, 0.0))
    p.set("KB1", -8.57e5).set("ANIS_UB", (0.0, 0.0, 1.0))
    p.set("B1", -1e7).set("B2", -1e7)
    p.glob.update(A0=-4e-11, A12=-1e-12, LATTICE_A=0.42e-9, C11=2.5e11,
                  C12=1.5e11, C44=1e11, RHO=7e3, ETA=0.0)
    seed = BASE_SEED + 2
    m0 = [noisy_axis_vectors(seed, shape, (1.0, 0.0, 0.0), 1.0, sub=0),
          noisy_axis_vectors(seed, shape, (-1.0, 0.0, 0.0), 1.0, sub=1)]
    z = np.zeros((3, 1, 256, 1024), dtype=np.float32)
    return Workload("antiferromagnet 1024x256x1 (2 nm cells), 2 sublattices, "
                    "magnetoelastic + elastic, 20000 fixed DP45 steps", p, m0,
                    u0=z.copy(), v0=z.copy(), adaptive=False, dt=5e-15,
                    steps=20000, seed=seed)


def _rand_params(seed, n):
    return uniform01(seed, np.arange(n, dtype=np.uint64))


def config_small(shape, cell, seed, terms=("DEMAG", "EXCH", "ANIS", "DMI", "ZEEMAN"),
                 n_sub=1, n_regions=1, empty_fraction=0.0):
    """A small random problem for parity tests: seeded material values,
    optional several regions and optional empty (Ms = 0) cells."""
    nx, ny, nz = shape
    p = Problem(shape, cell, n_sub, frozenset(terms))
    r = _rand_params(seed, 64)
    if n_regions > 1:
        rc = splitmix64(seed + 7, np.arange(nx * ny * nz, dtype=np.uint64))
        p.regions = (rc % np.uint64(n_regions)).astype(np.uint8).reshape(nz, ny, nx)
    if empty_fraction > 0:
        ru = uniform01(seed + 11, np.arange(nx * ny * nz, dtype=np.uint64)).reshape(nz, ny, nx)
        p.regions[ru < empty_fraction] = 255
    k = 0
    for reg in range(n_regions):
        for s in range(n_sub):
            p.set("MS", 4e5 + 8e5 * r[k % 64], s, reg); k += 1
            p.set("AEX", 5e-12 + 1.5e-11 * r[k % 64], s, reg); k += 1
            p.set("ALPHA", 0.01 + 0.3 * r[k % 64], s, reg); k += 1
            p.set("KU1", 1e5 + 5e5 * r[k % 64], s, reg); k += 1
            p.set("KU2", 2e4 * r[k % 64], s, reg); k += 1
            p.set("KB1", -2e5 * r[k % 64], s, reg); k += 1
            p.set("DIND", 3e-3 * (r[k % 64] - 0.3), s, reg); k += 1
            ax = np.array([r[k % 64] - 0.5, r[(k + 1) % 64] - 0.5, 0.8]); k += 2
            p.set("ANIS_U", ax / np.linalg.norm(ax), s, reg)
            p.set("ANIS_UB", (1.0, 0.0, 0.0), s, reg)
            p.set("B_EXT", (0.02 * r[k % 64], -0.01, 0.05), s, reg); k += 1
            p.set("B1", -1e7 * r[k % 64], s, reg); k += 1
            p.set("B2", -5e6 * r[k % 64], s, reg); k += 1
    # cubic anisotropy parameters from their own stream (the draws above keep
    # their values); the axes are not orthogonal on purpose
    r2 = _rand_params(seed + 101, 8 * n_regions * n_sub + 8)
    k2 = 0
    for reg in range(n_regions):
        for s in range(n_sub):
            p.set("KC1", 5e4 * (r2[k2] - 0.3), s, reg)
            p.set("ANIS_C1", (1.0, r2[k2 + 1] - 0.5, r2[k2 + 2] - 0.5), s, reg)
            p.set("ANIS_C2", (r2[k2 + 3] - 0.5, 1.0, r2[k2 + 4] - 0.5), s, reg)
            k2 += 5
    if n_regions > 1 or empty_fraction > 0:
        p.set("MS", 0.0, None, 255)
    p.glob.update(A0=-4e-11, A12=-1e-12, LATTICE_A=0.42e-9, C11=2.5e11,
                  C12=1.5e11, C44=1e11, RHO=7e3, ETA=0.0)
    m0 = [random_unit_vectors(seed, shape, sub=s) for s in range(n_sub)]
    return Workload("small random %dx%dx%d" % shape, p, m0, seed=seed)


# Sizes for the batched and served workloads (powers of two and 3*2^k).
BATCH_SIZES = (32, 64, 96, 128, 192, 256, 384, 512)


def stable_dt(p, courant=0.25):
    """A fixed DP45 step for an explicit run of problem p: `courant` over the
    fastest precession rate gamma * B_max, with B_max the largest exchange
    field of a discrete Laplacian (2A/Ms * 4/h^2 per axis with more than one
    cell) plus mu0 Ms.  A workload parameter, not part of the method."""
    ms = float(p.scal["MS"][0].max())
    a = float(p.scal["AEX"][0].max())
    lap = sum(4.0 / h ** 2 for h, n in zip(p.cell, p.shape) if n > 1)
    bmax = 2.0 * a / ms * lap + MU0 * ms
    return courant / (GAMMA * bmax)


def batch_instances(count=256, seed=BASE_SEED + 3):
    """Independent ferromagnets with seeded uneven sizes and materials
    (demag + exchange, 2 nm cubes, random initial state), each with its own
    fixed step (stable_dt)."""
    out = []
    r = uniform01(seed, np.arange(8 * count, dtype=np.uint64)).reshape(count, 8)
    for i in range(count):
        nx = BATCH_SIZES[int(r[i, 0] * len(BATCH_SIZES))]
        ny = BATCH_SIZES[int(r[i, 1] * len(BATCH_SIZES))]
        nz = (1, 2, 4)[int(r[i, 2] * 3)]
        p = Problem((nx, ny, nz), (2e-9, 2e-9, 2e-9), 1, frozenset({"DEMAG", "EXCH"}))
        p.set("MS", 4e5 + 1e6 * r[i, 3]).set("AEX", 5e-12 + 1.5e-11 * r[i, 4])
        p.set("ALPHA", 0.01 + 0.49 * r[i, 5])
        s = seed * 1000 + i
        out.append(Workload("instance %d" % i, p, [random_unit_vectors(s, p.shape)], seed=s, dt=stable_dt(p)))
    return out


def serve_requests(count, seed=BASE_SEED + 4, rate_hz=200.0):
    """Poisson arrivals of relax-to-equilibrium solves on grids from 64^2x1 to
    1024^2x4 with applied fields |B| <= 50 mT.  Returns (arrival_s, Workload)."""
    r = uniform01(seed, np.arange(8 * count, dtype=np.uint64)).reshape(count, 8)
    t = np.cumsum(-np.log1p(-r[:, 0]) / rate_hz)
    sizes = (64, 128, 256, 512, 1024)
    out = []
    for i in range(count):
        n = sizes[min(int(r[i, 1] ** 2 * len(sizes)), len(sizes) - 1)]
        nz = (1, 2, 4)[int(r[i, 2] * 3)] if n <= 256 else 1 + 3 * int(r[i, 2] > 0.8)
        p = Problem((n, n, nz), (4e-9, 4e-9, 2e-9), 1,
                    frozenset({"DEMAG", "EXCH", "ZEEMAN"}))
        p.set("MS", 8e5).set("AEX", 1.3e-11).set("ALPHA", 0.5)
        bz = 0.05 * r[i, 3]
        bx = 0.05 * np.sqrt(max(0.0, 1 - r[i, 3] ** 2)) * (r[i, 4] - 0.5)
        p.set("B_EXT", (bx, 0.0, bz))
        s = seed * 1000 + i
        out.append((float(t[i]), Workload("request %d" % i, p,
                                          [random_unit_vectors(s, p.shape)], seed=s)))
    return out
