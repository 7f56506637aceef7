"""The allocation-free entry point, mmp_demag_noalloc, against the context
path.

It serves callers that cannot call cudaMalloc (device memory owned by a
host framework, loops that must not allocate once running): its working
memory is a static array inside the library.  It must give the same demag
field as mmp_eval_field of a context with only the demag term, on
consecutive calls (the second reuses the tables of the first) and in a
fresh process or after any other test.  This file is collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _context_demag(shape, cell, M):
    import torch
    import paper_2411_18194_gb300 as pkg
    from inputs import Problem
    p = Problem(shape, cell, 1, frozenset({"DEMAG"}))
    p.set("MS", 1.0)                      # B = demag field of 1 * m = M
    mag = pkg.Magnet.from_problem(p)
    mag.set_m(0, M)
    B = torch.empty_like(M)
    mag.eval_field(0, B, None)
    mag.close()
    return B.cpu().numpy()


def test_noalloc_matches_context_path_on_two_calls():
    import torch
    import paper_2411_18194_gb300 as pkg
    from inputs import MU0, random_unit_vectors
    shape, cell = (45, 37, 3), (2e-9, 2.5e-9, 1.5e-9)
    Ms = 8e5
    bar = 1e-5 * MU0 * Ms          # the per-evaluation field tolerance of the tests
    for seed in (11, 12):          # two calls in a row, different inputs
        M = torch.from_numpy(random_unit_vectors(seed, shape) * np.float32(Ms)).cuda()
        B = torch.full_like(M, float("nan"))
        pkg.demag_noalloc(shape, cell, M, B)
        torch.cuda.synchronize()
        ref = _context_demag(shape, cell, M)
        got = B.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= bar, np.abs(got - ref).max()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    import paper_2411_18194_gb300 as pkg
    shape = (1024, 1024, 1)
    M = torch.zeros((3, 1, 1024, 1024), dtype=torch.float32, device="cuda")
    B = torch.empty_like(M)
    with pytest.raises(pkg.MmpError) as e:
        pkg.demag_noalloc(shape, (1e-9, 1e-9, 1e-9), M, B)
    assert e.value.status == -1 and "scratch" in str(e.value)
