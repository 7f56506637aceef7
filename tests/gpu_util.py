"""Helpers shared by the GPU tests: run the CUDA path through the C-ABI
binding and the FP64 oracle on the same seeded FP32 inputs."""
import numpy as np

from inputs import GAMMA, MU0

F32_EPS = 2.0 ** -24   # half an FP32 ulp, relative


def cell_ms(problem, sub=0):
    """Ms of sublattice `sub` at every cell, [nz][ny][nx]; a cell with Ms = 0
    (empty) takes the largest Ms among its six neighbours (the scale of the
    fields around it), or the largest of the problem if they are empty too."""
    ms = problem.scal["MS"][sub][problem.regions].astype(np.float64)
    empty = ms == 0
    if not empty.any():
        return ms
    nb = np.zeros_like(ms)
    for ax in range(3):
        for d in (-1, 1):
            sh = np.roll(ms, d, axis=ax)
            idx = [slice(None)] * 3
            idx[ax] = 0 if d == 1 else -1     # the wrapped row is not a neighbour
            sh[tuple(idx)] = 0.0
            nb = np.maximum(nb, sh)
    nb = np.where(nb > 0, nb, problem.scal["MS"].max())
    return np.where(empty, nb, ms)


def field_tolerance(problem, B_ref, sub=0):
    """Per-evaluation field bar, per cell: 1e-5 mu0 Ms of the cell's own
    sublattice and region (the stated tolerance, read as an H error of
    1e-5 Ms), plus the unavoidable rounding of an FP32 output, half an ulp
    of |B| (only matters where |B| exceeds ~1e2 T, e.g. the homogeneous AFM
    exchange field of ~2e3 T)."""
    return 1e-5 * MU0 * cell_ms(problem, sub)[None] + F32_EPS * np.abs(B_ref)


def torque_tolerance(problem, B_ref, tol_B):
    """|d tau| <= gamma (1 + alpha) |d B| for unit m, plus FP32 rounding of
    the two cross products (a few ulp of gamma |B|)."""
    return GAMMA * (2.0 * tol_B + 8.0 * F32_EPS * np.abs(B_ref).max(axis=0, keepdims=True))


def make_magnet(problem, m0s, u=None, v=None):
    import torch
    import paper_2411_18194_gb300 as pkg
    mag = pkg.Magnet.from_problem(problem)
    for s, m in enumerate(m0s):
        mag.set_m(s, torch.from_numpy(np.ascontiguousarray(m, dtype=np.float32)).cuda())
    if u is not None:
        mag.set_elastic(torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda(),
                        torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda())
    return mag


def gpu_eval(mag, problem):
    """B and tau of every sublattice (numpy float64)."""
    import torch
    nx, ny, nz = problem.shape
    Bs, Ts = [], []
    for s in range(problem.n_sub):
        B = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
        T = torch.empty_like(B)
        mag.eval_field(s, B, T)
        Bs.append(B.cpu().numpy().astype(np.float64))
        Ts.append(T.cpu().numpy().astype(np.float64))
    return Bs, Ts


def oracle_eval(problem, m0s, u=None, noct=None):
    from oracle import fields
    ms = [np.asarray(m, dtype=np.float64) for m in m0s]
    uu = None if u is None else np.asarray(u, dtype=np.float64)
    P = fields.cell_params(problem)
    Bs = fields.effective_fields(problem, ms, uu, noct=noct, P=P)
    Ts = fields.torques(problem, ms, Bs, P)
    return Bs, Ts
