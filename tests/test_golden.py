"""Pins against values the paper prints (tests/golden/)."""
import os

import numpy as np

from inputs import Problem, config_c3

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()[:2]
            vals[k] = float(v)
    return vals


def test_oracle_shear_wave_speed_matches_printed_pulse_speed():
    """The oracle's elastic force on a long transverse wave u_z = sin(k x),
    read at interior cells, gives omega^2 = f_z / (-rho u_z); omega / k with
    the printed NiO stiffness and density must be the printed pulse speed
    (about 4 km/s, so within 3 %)."""
    from oracle import elastic
    g = _load("nio_racetrack.txt")
    n, h = 256, 2e-9
    p = Problem((n, 1, 1), (h, h, h), 1, frozenset({"ELASTIC"}))
    p.glob.update(C11=g["C11"], C12=g["C12"], C44=g["C44"], RHO=g["RHO"], ETA=0.0)
    k = 2 * np.pi / (64 * h)
    x = (np.arange(n) + 0.5) * h
    u = np.zeros((3, 1, 1, n))
    u[2, 0, 0, :] = np.sin(k * x)
    f = elastic.elastic_force(u, np.zeros_like(u), p)
    mid = slice(8, n - 8)
    uz = u[2, 0, 0, mid]
    sel = np.abs(uz) > 0.5
    omega2 = -f[2, 0, 0, mid][sel] / (g["RHO"] * uz[sel])
    speed = np.sqrt(omega2) / k
    assert np.allclose(speed, speed.mean(), rtol=1e-9)          # one dispersion value in the bulk
    assert abs(speed.mean() / g["SHEAR_PULSE_SPEED"] - 1.0) < 0.03
    # and it is the continuum transverse speed sqrt(C44 / rho) up to the 4th-order stencil error
    assert abs(speed.mean() / np.sqrt(g["C44"] / g["RHO"]) - 1.0) < 1e-4


def test_antiferromagnet_workload_uses_the_printed_nio_constants():
    """The two-sublattice workload takes the lattice constant and the
    anisotropy magnitude from the printed NiO table."""
    g = _load("nio_racetrack.txt")
    p = config_c3().problem
    assert p.glob["LATTICE_A"] == g["LATTICE_A"]
    assert p.scal["KU1"][0, 0] == g["KU"] and p.scal["KU1"][1, 0] == g["KU"]
