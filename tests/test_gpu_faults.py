"""Failure paths of the library driven from the host, with no fault on the
GPU: a device allocator that refuses allocations (MMP_E_OOM, the context
still usable once memory is there again) and a wall-clock deadline that
passes inside mmp_relax (MMP_E_TIMEOUT)."""
import time

import numpy as np
import pytest

from inputs import config_small

pytestmark = pytest.mark.gpu

FM = ("DEMAG", "EXCH", "ANIS", "DMI", "ZEEMAN")


class RefusingAllocator:
    """Device allocations through PyTorch's caching allocator; every request
    after the first `allow` is refused (returns NULL)."""

    def __init__(self, allow):
        import torch
        from paper_2411_18194_gb300.binding import ALLOC_FN, FREE_FN
        self.torch = torch
        self.allow = allow
        self.count = 0
        self.refused = 0
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        self.count += 1
        if self.count > self.allow:
            self.refused += 1
            return None
        t = self.torch
        return t.cuda.caching_allocator_alloc(int(nbytes), t.cuda.current_device(), t.cuda.current_stream())

    def _free(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)


def _setup_steps(w):
    """The calls of a context's life that may allocate, in order."""
    import torch
    from paper_2411_18194_gb300 import Magnet
    p = w.problem
    state = {}

    def create(alloc):
        state["mag"] = Magnet.from_problem(p, allocator=alloc)

    def set_m(alloc):
        state["mag"].set_m(0, torch.from_numpy(np.ascontiguousarray(w.m0[0], dtype=np.float32)).cuda())

    def field(alloc):
        nx, ny, nz = p.shape
        B = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
        T = torch.empty_like(B)
        state["mag"].eval_field(0, B, T)
        state["B"] = B.cpu().numpy()

    def steps(alloc):
        state["mag"].set_solver(adaptive=False, dt=1e-14)
        state["mag"].step(3)
    return state, [create, set_m, field, steps]


def test_refused_allocations_give_oom_and_leave_the_context_usable():
    """For every allocation the library makes while a context is created,
    filled, evaluated and stepped: refusing it makes that call fail with
    MMP_E_OOM; with memory available again the same call succeeds and the
    field is bitwise the one of a context that never saw a refusal."""
    from paper_2411_18194_gb300 import MmpError
    w = config_small((24, 20, 2), (2e-9, 2e-9, 1e-9), 81, terms=FM)
    ref_alloc = RefusingAllocator(allow=10 ** 9)
    ref, calls = _setup_steps(w)
    for c in calls:
        c(ref_alloc)
    total = ref_alloc.count
    assert total >= 5
    ref["mag"].close()
    for k in range(total):
        alloc = RefusingAllocator(allow=k)
        st, calls = _setup_steps(w)
        failed = None
        for i, c in enumerate(calls):
            try:
                c(alloc)
            except MmpError as e:
                assert e.status == -2, (k, i, e)      # MMP_E_OOM
                failed = i
                break
        assert failed is not None and alloc.refused == 1, k
        if failed == 0:
            continue                                   # creation failed: nothing to resume
        alloc.allow = 10 ** 9
        for c in calls[failed:]:
            c(alloc)
        assert np.array_equal(st["B"], ref["B"]), k
        st["mag"].close()


def test_relax_deadline_returns_timeout_and_keeps_the_state():
    """A relax whose wall-clock deadline passes returns MMP_E_TIMEOUT after
    the attempt in flight; the state is an accepted one (finite, unit
    length) and the context keeps stepping."""
    import torch
    from paper_2411_18194_gb300 import MmpError
    from gpu_util import make_magnet
    w = config_small((64, 64, 2), (2e-9, 2e-9, 1e-9), 82, terms=FM)
    p = w.problem
    mag = make_magnet(p, w.m0)
    mag.set_solver(adaptive=True, dt=1e-14, tol=1e-5)
    t0 = time.perf_counter()
    with pytest.raises(MmpError) as ei:
        mag.relax(torque_tol=1e-12, max_time=1e-6, timeout_s=0.2)
    took = time.perf_counter() - t0
    assert ei.value.status == -5 and 0.2 <= took < 5.0
    m = torch.empty((3,) + p.shape[::-1], dtype=torch.float32, device="cuda")
    mag.get_m(0, m)
    mm = m.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(mm)) and np.abs(np.sqrt((mm ** 2).sum(axis=0)) - 1).max() < 1e-5
    mag.set_solver(adaptive=False, dt=1e-14)
    mag.step(2)
    mag.close()
