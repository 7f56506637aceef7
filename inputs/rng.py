"""Counter-based random numbers for the synthetic initial states.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) is used as a counter-based generator: the n-th
output of the stream with seed `s` is mix(s + (n + 1) * 0x9E3779B97F4A7C15).
Every (sublattice, cell, draw) triple has its own counter, so a value never
depends on the order of generation or on the grid traversal.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, counter):
    """SplitMix64 output for `counter` (uint64 array) in the stream `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed, counter):
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _counters(n_cells, sub, draw, n_draws):
    cell = np.arange(n_cells, dtype=np.uint64)
    return (np.uint64(sub) * np.uint64(n_cells) + cell) * np.uint64(n_draws) + np.uint64(draw)


def random_unit_vectors(seed, shape, sub=0):
    """Uniformly distributed unit vectors, SoA float32 [3][nz][ny][nx].

    z = 2 u1 - 1 and phi = 2 pi u2, drawn in FP64 and rounded once to FP32.
    `shape` is (nx, ny, nz).
    """
    nx, ny, nz = shape
    n = nx * ny * nz
    u1 = uniform01(seed, _counters(n, sub, 0, 2))
    u2 = uniform01(seed, _counters(n, sub, 1, 2))
    z = 2.0 * u1 - 1.0
    phi = 2.0 * np.pi * u2
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    m = np.stack([s * np.cos(phi), s * np.sin(phi), z])
    return m.reshape(3, nz, ny, nx).astype(np.float32)


def noisy_axis_vectors(seed, shape, axis, max_angle_deg, sub=0):
    """Unit vectors tilted off `axis` by a polar angle uniform in
    [0, max_angle_deg] with a uniform azimuth; FP64 then rounded to FP32."""
    nx, ny, nz = shape
    n = nx * ny * nz
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    theta = np.deg2rad(max_angle_deg) * uniform01(seed, _counters(n, sub, 0, 2))
    phi = 2.0 * np.pi * uniform01(seed, _counters(n, sub, 1, 2))
    # orthonormal frame (e1, e2, a)
    helper = np.array([0.0, 0.0, 1.0]) if abs(a[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = np.cross(helper, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    st, ct = np.sin(theta), np.cos(theta)
    m = (ct[None, :] * a[:, None] + (st * np.cos(phi))[None, :] * e1[:, None]
         + (st * np.sin(phi))[None, :] * e2[:, None])
    return m.reshape(3, nz, ny, nx).astype(np.float32)
