"""Energy of every field term (mmp_energy) against the oracle's energies on
the same FP32 inputs: a two-region ferromagnet with demag, exchange,
uniaxial and cubic anisotropy, iDMI and Zeeman, and the two-sublattice
magnetoelastic problem with random displacement and velocity."""
import numpy as np
import pytest

from inputs import config_small
from gpu_util import make_magnet

pytestmark = pytest.mark.gpu


def _close(got, ref, name):
    assert abs(got - ref) <= 2e-5 * abs(ref) + 1e-30, (name, got, ref)


def test_ferromagnet_term_energies():
    from oracle import demag, fields
    w = config_small((20, 16, 3), (2e-9, 2.5e-9, 1e-9), 141,
                     terms=("DEMAG", "EXCH", "ANIS", "DMI", "ZEEMAN", "CUBIC"), n_regions=2)
    p = w.problem
    mag = make_magnet(p, w.m0)
    got = mag.energy()
    ref = fields.energies(p, [w.m0[0].astype(np.float64)], noct=demag.tensor_octant(p.shape, p.cell))
    for name, key in (("DEMAG", "demag"), ("EXCH", "exch"), ("ANIS", "anis"), ("DMI", "dmi"),
                      ("ZEEMAN", "zeeman"), ("CUBIC", "cubic")):
        _close(got[name], ref[key], name)
    assert got["AFM"] == 0.0 and got["MEL"] == 0.0 and got["ELASTIC"] == 0.0
    assert mag.time()["evals"] == 0          # the demag-only evaluation is not a solver evaluation
    mag.close()


def test_magnetoelastic_antiferromagnet_energies():
    from oracle import demag, elastic, fields
    w = config_small((18, 12, 1), (2e-9, 2e-9, 2e-9), 151,
                     terms=("DEMAG", "EXCH", "ANIS", "AFM", "MEL", "ELASTIC", "ZEEMAN"), n_sub=2)
    p = w.problem
    rng = np.random.default_rng(5)
    u = (1e-11 * rng.standard_normal((3,) + p.shape[::-1])).astype(np.float32)
    v = (10.0 * rng.standard_normal((3,) + p.shape[::-1])).astype(np.float32)
    mag = make_magnet(p, w.m0, u, v)
    got = mag.energy()
    ms = [m.astype(np.float64) for m in w.m0]
    ref = fields.energies(p, ms, u.astype(np.float64), noct=demag.tensor_octant(p.shape, p.cell))
    for name, key in (("DEMAG", "demag"), ("EXCH", "exch"), ("ANIS", "anis"), ("AFM", "afm"),
                      ("MEL", "mel"), ("ZEEMAN", "zeeman")):
        _close(got[name], ref[key], name)
    strain_e, kinetic_e = elastic.elastic_energy(p, u.astype(np.float64), v.astype(np.float64))
    _close(got["ELASTIC"], strain_e + kinetic_e, "ELASTIC")
    mag.close()


def test_magnetoelastic_term_needs_elastic_term():
    import paper_2411_18194_gb300 as pkg
    w = config_small((8, 8, 1), (2e-9, 2e-9, 2e-9), 161, terms=("EXCH", "MEL"), n_sub=1)
    mag = make_magnet(w.problem, w.m0)
    with pytest.raises(pkg.MmpError) as e:
        mag.energy()
    assert e.value.status == -1 and "elastic" in str(e.value)
    mag.close()
