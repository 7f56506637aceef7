"""Precision study of tensor-core DFT stages for the demag convolution
(no GPU): is a split-BF16 or TF32 DFT-GEMM form of the FFT's small radix
stages accurate enough to replace the FP32 CUDA-core FFT?

The zero-padded demag convolution (Methods, Magnetostatic field) is run with
every axis transform as a four-step FFT whose radix-16 stages are dense DFT
matrices applied as GEMMs, with the operands rounded the way a tensor-core
MMA would take them:

* ``bf16x3``: split BF16, a = a_hi + a_lo, products a_hi b_hi + a_hi b_lo +
  a_lo b_hi (the lo*lo term dropped);
* ``tf32``: one TF32 product;
* ``tf32x3``: split TF32, three products as above;

and the twiddles between the stages and the kernel multiply in FP32.  The
products are summed in FP64 and rounded once per GEMM, which is at least as
accurate as an FP32 tensor-core accumulator, so an error found here is a
lower bound for the real kernel.  The FP32 reference point is the plain FP32
FFT.  The bar is the field tolerance 1e-5 mu0 Ms against the FP64 oracle.

Finding: split BF16 (the cheaper form) and single TF32 miss the bar on a
random state (split BF16 from 128^2 x 8 cells on, by a factor that grows with
the grid); only split TF32 (three TF32 products per product) keeps the field
well within it."""
import numpy as np
import pytest

from inputs import MU0, random_unit_vectors
from oracle import demag

RADIX = 16


def _round_mantissa(x, keep_bits):
    """Round float32 values to `keep_bits` explicit mantissa bits (nearest,
    ties to even): 7 for BF16, 10 for TF32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    drop = 23 - keep_bits
    half = (1 << (drop - 1)) - 1
    u = (u + half + ((u >> drop) & 1)) & ~np.uint64((1 << drop) - 1) & 0xFFFFFFFF
    return u.astype(np.uint32).view(np.float32)


def _split(a, mode):
    keep = 7 if mode.startswith("bf16") else 10
    hi = _round_mantissa(a, keep)
    lo = _round_mantissa(a.astype(np.float32) - hi, keep)
    return hi.astype(np.float64), lo.astype(np.float64)


def _real_gemm(A, B, mode):
    """A (n x n) @ B (n x m) as the tensor core would form it (see above)."""
    if mode == "tf32":
        keep = 10
        return _round_mantissa(A, keep).astype(np.float64) @ _round_mantissa(B, keep).astype(np.float64)
    ah, al = _split(A, mode)
    bh, bl = _split(B, mode)
    return ah @ bh + ah @ bl + al @ bh


def _dft_gemm(D, inverse, mode):
    """Dense DFT (radix-sized) of the columns of complex64 D [n][m]."""
    n = D.shape[0]
    k = np.arange(n)
    sign = 1.0 if inverse else -1.0
    F = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
    Fr, Fi = F.real.astype(np.float32), F.imag.astype(np.float32)
    Dr, Di = D.real.astype(np.float32), D.imag.astype(np.float32)
    re = _real_gemm(Fr, Dr, mode) - _real_gemm(Fi, Di, mode)
    im = _real_gemm(Fr, Di, mode) + _real_gemm(Fi, Dr, mode)
    return (re + 1j * im).astype(np.complex64)


def _fft_axis0(x, inverse, mode):
    """Unnormalised DFT along axis 0 of complex64 x [L][m] by the four-step
    split L = N1 N2 (N1 = RADIX): n = N2 n1 + n2, k = k1 + N1 k2."""
    L, m = x.shape
    if L <= RADIX:
        return _dft_gemm(x, inverse, mode)
    assert L % RADIX == 0
    N1, N2 = RADIX, L // RADIX
    # step 1: length-N1 DFTs over n1 for every n2 (one GEMM)
    Y = _dft_gemm(x.reshape(N1, N2 * m), inverse, mode).reshape(N1, N2, m)
    # step 2: twiddles w_L^(n2 k1) in FP32
    sign = 1.0 if inverse else -1.0
    tw = np.exp(sign * 2j * np.pi * np.outer(np.arange(N1), np.arange(N2)) / L).astype(np.complex64)
    Y = Y * tw[:, :, None]
    # step 3: length-N2 DFTs over n2 for every k1 (recursively)
    Z = _fft_axis0(np.moveaxis(Y, 1, 0).reshape(N2, N1 * m), inverse, mode).reshape(N2, N1, m)
    # output k = k1 + N1 k2: [k2][k1] is already in natural order
    return Z.reshape(L, m)


def _fftn(x, inverse, mode):
    """3-D transform of complex64 x [c][Pz][Py][Px] over the last three axes."""
    if mode == "fp32":
        f = np.fft.ifftn if inverse else np.fft.fftn
        y = f(x.astype(np.complex64), axes=(1, 2, 3))
        if inverse:
            y = y * np.float32(np.prod(x.shape[1:]))   # unnormalised, like the others
        return y.astype(np.complex64)
    y = x.astype(np.complex64)
    for ax in (3, 2, 1):
        moved = np.moveaxis(y, ax, 0)
        shp = moved.shape
        out = _fft_axis0(moved.reshape(shp[0], -1), inverse, mode)
        y = np.moveaxis(out.reshape(shp), 0, ax)
    return y


def _kernel_spectrum(shape, cell):
    """FP64 spectrum of the six padded kernel components, rounded to FP32."""
    nx, ny, nz = shape
    Px, Py, Pz = demag.padded_sizes(shape)
    noct = demag.tensor_octant(shape, cell)

    def fold(n, P):
        pos = np.arange(P)
        off = np.where(pos < n, pos, pos - P)
        valid = np.abs(off) < n
        return np.where(valid, np.abs(off), 0), np.sign(off), valid

    ix, sx, vx = fold(nx, Px)
    iy, sy, vy = fold(ny, Py)
    iz, sz, vz = fold(nz, Pz)
    mask = vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
    out = []
    for comp in range(6):
        K = noct[comp][np.ix_(iz, iy, ix)] * mask
        ox, oy, oz = demag.ODD[comp]
        if ox:
            K = K * sx[None, None, :]
        if oy:
            K = K * sy[None, :, None]
        if oz:
            K = K * sz[:, None, None]
        out.append(np.fft.fftn(K).astype(np.complex64))
    return out, noct


def demag_emulated(shape, cell, M, mode):
    """B_demag with the transforms in `mode` (fp32, bf16x3, tf32, tf32x3)."""
    nx, ny, nz = shape
    Px, Py, Pz = demag.padded_sizes(shape)
    Khat, _ = _kernel_spectrum(shape, cell)
    Mp = np.zeros((3, Pz, Py, Px), dtype=np.complex64)
    Mp[:, :nz, :ny, :nx] = M.astype(np.float32)
    Mh = _fftn(Mp, False, mode)
    xx, yy, zz, xy, xz, yz = Khat
    Hh = np.stack([xx * Mh[0] + xy * Mh[1] + xz * Mh[2],
                   xy * Mh[0] + yy * Mh[1] + yz * Mh[2],
                   xz * Mh[0] + yz * Mh[1] + zz * Mh[2]]).astype(np.complex64)
    H = _fftn(Hh, True, mode).real / np.float32(Px * Py * Pz)
    return -MU0 * H[:, :nz, :ny, :nx].astype(np.float64)


def test_round_mantissa_matches_the_formats():
    """BF16 / TF32 rounding: exact for representable values, relative error
    at most 2^-8 / 2^-11, ties to even."""
    rng = np.random.default_rng(1)
    x = rng.normal(size=4096).astype(np.float32)
    for keep in (7, 10):
        r = _round_mantissa(x, keep)
        assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -(keep + 1))
        assert np.array_equal(_round_mantissa(r, keep), r)
    assert _round_mantissa(np.float32(1.0 + 2.0 ** -8), 7) == np.float32(1.0)           # tie -> even
    assert _round_mantissa(np.float32(1.0 + 3 * 2.0 ** -8), 7) == np.float32(1.0 + 2.0 ** -6)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32", "tf32x3"])
def test_four_step_transform_is_the_dft(mode):
    """The emulated four-step transform is the DFT up to its operand rounding."""
    rng = np.random.default_rng(2)
    x = (rng.normal(size=(256, 3)) + 1j * rng.normal(size=(256, 3))).astype(np.complex64)
    ref = np.fft.fft(x.astype(np.complex128), axis=0)
    got = _fft_axis0(x, False, mode)
    rel = np.abs(got - ref).max() / np.abs(ref).max()
    bound = {"bf16x3": 2e-4, "tf32": 3e-3, "tf32x3": 2e-6}[mode]
    assert rel < bound, rel
    back = _fft_axis0(got, True, mode) / 256
    assert np.abs(back - x).max() < 10 * bound * np.abs(x).max()


@pytest.mark.parametrize("shape,cell,Ms", [
    ((128, 128, 8), (2e-9, 2e-9, 1e-9), 1.1e6),   # the large ferromagnet's cell and Ms
    ((512, 512, 1), (2e-9, 2e-9, 2e-9), 1.4e6),   # the largest batched instance, the top of its Ms range
], ids=["ferromagnet-128x128x8", "instance-512x512x1"])
def test_tensor_core_dft_stages_against_the_field_bar(shape, cell, Ms):
    """Random state (the hardest spectrum): the FP32 FFT and split TF32 stay
    far within 1e-5 mu0 Ms of the FP64 oracle (about 2 % and 3 % of it),
    split BF16 and single TF32 do not (split BF16 is at 0.91-0.93 of the bar
    on 64^2 x 8 and 256 x 128 x 4 cells and above it from 128^2 x 8 on,
    growing with the grid)."""
    m = random_unit_vectors(20241131, shape).astype(np.float64)
    M = Ms * m
    ref = demag.demag_fft(shape, cell, M)
    bar = 1e-5 * MU0 * Ms
    err = {mode: np.abs(demag_emulated(shape, cell, M, mode) - ref).max() / bar
           for mode in ("fp32", "bf16x3", "tf32", "tf32x3")}
    assert err["fp32"] < 0.1, err
    assert err["tf32x3"] < 0.1, err
    assert err["bf16x3"] > 1.0, err
    assert err["tf32"] > 10.0, err
