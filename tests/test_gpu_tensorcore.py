"""Parity of the split-TF32 tensor-core DFT stage (the final length-32 DFT
of every y transform of pass B as a dense GEMM on tcgen05, engine bit
MMP_ENGINE_TC_Y) with the FP64 oracle, at the per-cell 1e-5 mu0 Ms bar.
Grids: cells of the large ferromagnet (128x128x8, its materials), the
largest batched instance (512x512x1, Ms 1.4e6), a plane split over a
two-CTA cluster (Py = 2048), the full 1024x1024x8 ferromagnet on sampled
cells against the direct sum; and agreement with the CUDA-core transform."""
import numpy as np
import pytest

from inputs import MU0, Problem, config_c2, config_small, random_unit_vectors
from gpu_util import field_tolerance, torque_tolerance, make_magnet, gpu_eval, oracle_eval

pytestmark = pytest.mark.gpu

WARP_B, WARP_X, TC_Y = 1, 2, 4


def _with_tc(mag):
    sh = mag.get_shape()
    mag.set_shape(engine=sh["engine"] | TC_Y)
    assert mag.get_shape()["engine"] & TC_Y
    return mag


def _c2_cells(shape):
    w = config_c2()
    p = w.problem
    p.shape = shape
    p.regions = np.zeros(shape[::-1], dtype=np.uint8)
    return p, [random_unit_vectors(w.seed, shape)]


def _largest_batched_instance():
    p = Problem((512, 512, 1), (2e-9, 2e-9, 2e-9), 1, frozenset({"DEMAG", "EXCH"}))
    p.set("MS", 1.4e6).set("AEX", 2e-11).set("ALPHA", 0.5)
    return p, [random_unit_vectors(777, p.shape)]


def _cluster_plane():
    w = config_small((3, 1000, 8), (2e-9, 2e-9, 1e-9), 71)
    return w.problem, w.m0


@pytest.mark.parametrize("make", [lambda: _c2_cells((128, 128, 8)), _largest_batched_instance, _cluster_plane],
                         ids=["c2-cells-128x128x8", "batched-512x512x1", "cluster-3x1000x8"])
def test_tensor_core_stage_parity(make):
    p, m0 = make()
    mag = _with_tc(make_magnet(p, m0))
    Bg, Tg = gpu_eval(mag, p)
    mag.close()
    Bo, To = oracle_eval(p, [m.astype(np.float64) for m in m0])
    tolB = field_tolerance(p, Bo[0])
    err = np.abs(Bg[0] - Bo[0])
    assert np.all(err <= tolB), (err.max(), (err / tolB).max())
    assert np.all(np.abs(Tg[0] - To[0]) <= torque_tolerance(p, Bo[0], tolB))


def test_tensor_core_stage_agrees_with_cuda_cores():
    """Same state, the two transforms of pass B: they differ only by FP32-level
    rounding (split TF32 keeps about 21 bits of each product)."""
    p, m0 = _c2_cells((64, 512, 8))
    mag = make_magnet(p, m0)
    B0, _ = gpu_eval(mag, p)
    _with_tc(mag)
    B1, _ = gpu_eval(mag, p)
    mag.close()
    scale = np.abs(B0[0]).max()
    assert np.abs(B1[0] - B0[0]).max() <= 1e-5 * scale


def test_tensor_core_stage_full_size_sampled():
    """The full 1024x1024x8 ferromagnet with every warp pass and the tensor-core
    stage: B_eff at sampled cells against the oracle's direct sum of the demag
    definition plus its local terms."""
    from oracle import demag, fields
    w = config_c2()
    p = w.problem
    nx, ny, nz = p.shape
    mag = _with_tc(make_magnet(p, w.m0))
    assert mag.get_shape()["engine"] == WARP_B | WARP_X | TC_Y
    Bg, _ = gpu_eval(mag, p)
    mag.close()
    m = w.m0[0].astype(np.float64)
    noct = demag.tensor_octant(p.shape, p.cell)
    P = fields.cell_params(p)
    local = sum(fields.effective_fields(
        p.__class__(p.shape, p.cell, 1, frozenset(p.terms - {"DEMAG"}), p.regions, p.scal, p.vec, p.glob),
        [m], P=P))
    rng = np.random.default_rng(11)
    picks = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (1023, 0, 3), (0, 1023, 5), (511, 512, 4)]
    picks += [tuple(int(v) for v in (rng.integers(nx), rng.integers(ny), rng.integers(nz))) for _ in range(11)]
    cells = [x + nx * (y + ny * z) for x, y, z in picks]
    Bd = demag.demag_direct(p.shape, p.cell, P["MS"][0] * m, noct=noct, cells=cells)
    bar = 1e-5 * MU0 * 1.1e6
    for (x, y, z), bd in zip(picks, Bd.T):
        ref = bd + local[:, z, y, x]
        assert np.abs(Bg[0][:, z, y, x] - ref).max() <= bar, ((x, y, z), Bg[0][:, z, y, x], ref)
