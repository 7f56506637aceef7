"""Batched stepping of uneven independent instances (mmp_batch_*).

A member runs the arithmetic of its own context, so its trajectory must be
bitwise the same alone (mmp_step / mmp_run / mmp_relax on its context, with
the batch shape) and inside a batch of other instances; sampled members are
also checked against the FP64 oracle."""
import numpy as np
import pytest

from inputs import Problem, random_unit_vectors
from gpu_util import make_magnet

pytestmark = pytest.mark.gpu

# uneven sizes: powers of two and 3*2^k, nz in {1, 2, 4, 3}
SHAPES = [(32, 32, 1), (48, 32, 2), (32, 96, 4), (64, 48, 1), (24, 40, 3), (96, 64, 2)]


def _problem(i, shape, terms=("DEMAG", "EXCH")):
    p = Problem(shape, (2e-9, 2e-9, 2e-9), 1, frozenset(terms))
    p.set("MS", 5e5 + 1e5 * i).set("AEX", 8e-12 + 2e-12 * i).set("ALPHA", 0.05 + 0.07 * i)
    if "ZEEMAN" in terms:
        p.set("B_EXT", (0.01 * i, 0.0, 0.03))
    return p


def _magnet(i, shape, terms=("DEMAG", "EXCH")):
    p = _problem(i, shape, terms)
    m0 = random_unit_vectors(9000 + i, shape)
    mag = make_magnet(p, [m0])
    mag.set_shape(R=1, stage_kernel=0, engine=0)
    return p, m0, mag


def _m(mag):
    import torch
    nx, ny, nz = mag.shape
    out = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    mag.get_m(0, out)
    return out.cpu().numpy()


def _dt(p):
    from inputs import stable_dt
    return stable_dt(p)


def test_batch_fixed_steps_bitwise_equal_to_solo():
    import paper_2411_18194_gb300 as pkg
    mags, solo = [], []
    for i, sh in enumerate(SHAPES):
        p, m0, mag = _magnet(i, sh)
        mag.set_solver(adaptive=False, dt=_dt(p))
        mags.append(mag)
        _, _, s = _magnet(i, sh)
        s.set_solver(adaptive=False, dt=_dt(p))
        solo.append(s)
    with pkg.Batch() as b:
        for mag in mags:
            b.add(mag, "steps", 12)
        assert b.advance() == 0
        for mag in mags:
            assert b.status(mag) == (True, 0)
        assert b.launches() > 0
    for mag, s in zip(mags, solo):
        s.step(12)
        assert np.array_equal(_m(mag), _m(s)), mag.shape
        tb, ts = mag.time(), s.time()
        assert tb["steps"] == ts["steps"] == 12 and tb["t"] == ts["t"]
    for x in mags + solo:
        x.close()


def test_batch_members_match_oracle():
    import paper_2411_18194_gb300 as pkg
    from oracle.dp45 import Oracle, State
    picks = [0, 1, 4]
    mags, probs, m0s = [], [], []
    for i in picks:
        p, m0, mag = _magnet(i, SHAPES[i])
        mag.set_solver(adaptive=False, dt=_dt(p))
        mags.append(mag)
        probs.append(p)
        m0s.append(m0)
    with pkg.Batch() as b:
        for mag in mags:
            b.add(mag, "steps", 10)
        b.advance()
    for mag, p, m0 in zip(mags, probs, m0s):
        st = Oracle(p).run_fixed(State([m0]), _dt(p), 10)
        assert np.abs(_m(mag) - st.ms[0]).max() <= 1e-4, p.shape
        mag.close()


def test_batch_adaptive_and_relax_goals_bitwise_equal_to_solo():
    import paper_2411_18194_gb300 as pkg
    terms = ("DEMAG", "EXCH", "ZEEMAN")
    a = [_magnet(i, SHAPES[i], terms) for i in (0, 1, 3)]
    s = [_magnet(i, SHAPES[i], terms) for i in (0, 1, 3)]
    for (p, _, mag), (_, _, sol) in zip(a, s):
        for x in (mag, sol):
            x.set_solver(adaptive=True, dt=1e-15, tol=1e-5)
            x.set_param("ALPHA", 0.5)
    with pkg.Batch() as b:
        b.add(a[0][2], "run", 5e-12)
        b.add(a[1][2], "relax", 2e-3, 2e-10)
        b.add(a[2][2], "steps", 30)
        left = b.advance()
        assert left == 0
    s[0][2].run(5e-12)
    s[1][2].relax(torque_tol=2e-3, max_time=2e-10)
    s[2][2].step(30)
    for (_, _, mag), (_, _, sol) in zip(a, s):
        assert np.array_equal(_m(mag), _m(sol)), mag.shape
        tm, ts = mag.time(), sol.time()
        assert (tm["t"], tm["steps"], tm["rejected"]) == (ts["t"], ts["steps"], ts["rejected"])
    for x in a + s:
        x[2].close()


def test_members_join_between_advances():
    """A member added while others are mid-run starts from its own state and
    ends bitwise equal to its solo run (continuous batching)."""
    import paper_2411_18194_gb300 as pkg
    first = [_magnet(i, SHAPES[i]) for i in (0, 2)]
    late_p, _, late = _magnet(5, SHAPES[5])
    _, _, late_solo = _magnet(5, SHAPES[5])
    for p, _, mag in first:
        mag.set_solver(adaptive=False, dt=_dt(p))
    late.set_solver(adaptive=False, dt=_dt(late_p))
    late_solo.set_solver(adaptive=False, dt=_dt(late_p))
    with pkg.Batch() as b:
        for _, _, mag in first:
            b.add(mag, "steps", 20)
        assert b.advance(7) == 2
        b.add(late, "steps", 9)
        b.advance(5)
        b.remove(first[0][2])
        b.advance()
        assert b.status(late) == (True, 0)
    late_solo.step(9)
    assert np.array_equal(_m(late), _m(late_solo))
    assert first[0][2].time()["steps"] == 12 and first[1][2].time()["steps"] == 20
    for x in [f[2] for f in first] + [late, late_solo]:
        x.close()


def test_batch_rejects_ineligible_members():
    import paper_2411_18194_gb300 as pkg
    p = _problem(0, (16, 16, 1))
    mag = make_magnet(p, [random_unit_vectors(1, (16, 16, 1))])
    with pkg.Batch() as b:
        mag.set_shape(R=1, stage_kernel=1, engine=0)
        with pytest.raises(pkg.MmpError):
            b.add(mag, "steps", 1)
        mag.set_shape(R=1, stage_kernel=0, engine=0)
        b.add(mag, "steps", 1)
        with pytest.raises(pkg.MmpError):
            b.add(mag, "steps", 1)      # already a member
    mag.close()


def test_autotune_keeps_results_within_tolerance():
    """The tuned shape changes only the FP32 rounding order."""
    from gpu_util import field_tolerance, gpu_eval, oracle_eval
    p = _problem(2, (96, 64, 2))
    m0 = random_unit_vectors(77, p.shape)
    mag = make_magnet(p, [m0])
    shape, ms = mag.autotune(batch=True, force=True)
    assert shape["R"] == 1 and shape["stage_kernel"] == 0 and ms > 0
    Bg, _ = gpu_eval(mag, p)
    Bo, _ = oracle_eval(p, [m0.astype(np.float64)])
    assert np.all(np.abs(Bg[0] - Bo[0]) <= field_tolerance(p, Bo[0]))
    shape2, _ = mag.autotune()
    assert mag.get_shape() == shape2
    mag.close()


def test_open_boundary_member_bitwise_equal_to_solo():
    """A member with DMI and the open boundary carries its boundary into the
    batched kernels: bitwise equal to its solo run, and different from the
    same member with the Neumann boundary."""
    import paper_2411_18194_gb300 as pkg
    terms = ("DEMAG", "EXCH", "DMI", "ZEEMAN")
    runs = []
    for bc in ("open", "open", "neumann"):
        p, m0, mag = _magnet(2, (48, 32, 2), terms)
        mag.set_param("DIND", 2e-3)
        mag.set_boundary(bc)
        mag.set_solver(adaptive=False, dt=_dt(p))
        runs.append(mag)
    batched, solo, neumann = runs
    with pkg.Batch() as b:
        b.add(batched, "steps", 10)
        b.add(neumann, "steps", 10)
        assert b.advance() == 0
    solo.step(10)
    assert np.array_equal(_m(batched), _m(solo))
    assert not np.array_equal(_m(batched), _m(neumann))
    for x in runs:
        x.close()


def test_warp_engine_members_bitwise_equal_to_solo():
    """Members whose shape runs the warp passes A, B and C (Px = 2048, folded
    y length 1024: one with R = 1, one with a two-CTA cluster per plane)
    get their own launches beside the work lists of block-engine members;
    fixed steps and an adaptive relax are bitwise those of the same
    contexts alone."""
    import paper_2411_18194_gb300 as pkg
    shapes = [(1000, 500, 1), (1000, 900, 1), (64, 48, 2)]
    for goal in ("steps", "relax"):
        mags, solo = [], []
        for i, sh in enumerate(shapes):
            p = _problem(i, sh, ("DEMAG", "EXCH", "ZEEMAN"))
            m0 = random_unit_vectors(9100 + i, sh)
            pair = []
            for _ in range(2):
                mag = make_magnet(p, [m0])
                if sh[0] < 769:
                    mag.set_shape(R=1, stage_kernel=0, engine=0)
                else:
                    assert mag.get_shape()["engine"] == 3, mag.get_shape()
                if goal == "steps":
                    mag.set_solver(adaptive=False, dt=_dt(p))
                else:
                    mag.set_solver(adaptive=True, dt=1e-14)
                pair.append(mag)
            mags.append(pair[0])
            solo.append(pair[1])
        with pkg.Batch() as b:
            for mag in mags:
                if goal == "steps":
                    b.add(mag, "steps", 6)
                else:
                    b.add(mag, "relax", 1e-3, 2e-12)
            while b.advance(4):
                pass
            for mag in mags:
                assert b.status(mag)[1] == 0
        for mag, s in zip(mags, solo):
            if goal == "steps":
                s.step(6)
            else:
                s.relax(torque_tol=1e-3, max_time=2e-12)
            assert np.array_equal(_m(mag), _m(s)), (goal, mag.shape)
            assert mag.time()["t"] == s.time()["t"] and mag.time()["steps"] == s.time()["steps"]
        for x in mags + solo:
            x.close()
