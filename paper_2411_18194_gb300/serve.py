"""Continuous-batching server of relaxation solves on one GPU.

Requests (a magnet, its initial state and a relax goal) arrive over time.
The server admits them in arrival order while a device-memory budget
allows, adds each admitted context to one mmp_batch, and advances the batch
a few lock-step attempts at a time, so a request that arrives while others
are on the GPU joins at the next lock step and its work overlaps theirs.
Finished members leave the batch and free their memory.  All arithmetic
runs in libmmp (mmp_batch_advance); this module is host bookkeeping only.

A member computes exactly what the same context computes alone (same shape,
same FP32 stage coefficients, same FP64 step control), so a request's result
is bitwise the same in the mix and served by itself.

Memory accounting (bytes, FP32 state), what stays resident:
* per request, while it runs: the state, six stage vectors and the stage
  buffer (9 x 12 B per cell), the x-transformed spectrum (3 nz ny (Px/2 + 1)
  complex64) and the coefficient table;
* per (grid, cell size), while any request of it runs: the demag kernel
  spectrum, which the library shares between those contexts and frees with
  the last of them.
A request whose kernel spectrum is not resident also needs the FP64 build
buffers during its admission (the build synchronises and frees them before
the request joins), so they count against the budget at admission only.

A new geometry's context (and its kernel spectrum) is built on a worker
thread, on its own CUDA stream, while the batch keeps advancing the members
already admitted; the request joins at the first lock step after its build
has finished.  Requests of the same geometry wait for that build (arrival
order is kept).  A request may carry a wall-clock deadline (seconds after
its arrival): past it, the request leaves the queue or the batch with the
status MMP_E_TIMEOUT.
"""
import collections
import concurrent.futures
import time

import numpy as np

from .binding import Batch, Magnet


def _nice(n):
    """Padded FFT length of the library: the smallest even 2^a or 3 * 2^a
    at least 2n - 1 (1 when n = 1)."""
    if n == 1:
        return 1
    p2, p3 = 2, 6
    while p2 < 2 * n - 1:
        p2 *= 2
    while p3 < 2 * n - 1:
        p3 *= 2
    return min(p2, p3)


def _dims(shape):
    nx, ny, nz = shape
    Px, Py, Pz = _nice(nx), _nice(ny), _nice(nz)
    return nx * ny * nz, Px // 2 + 1, Py // 2 + 1, Pz // 2 + 1


def state_bytes(shape):
    """Resident bytes of one request while it runs (its own buffers)."""
    nx, ny, nz = shape
    n, kxn, _, _ = _dims(shape)
    return 9 * 12 * n + 3 * nz * ny * kxn * 8 + 2 * 256 * 160 + 64 * 1024


def spectrum_bytes(shape):
    """The demag kernel spectrum of a (grid, cell size), shared by its requests."""
    _, kxn, kyn, kzn = _dims(shape)
    krow = (6 * kzn + 3) // 4 * 4
    return kxn * kyn * krow * 4


def build_bytes(shape):
    """FP64 buffers of the kernel-spectrum build (freed when the build ends)."""
    nx, ny, nz = shape
    n, kxn, kyn, kzn = _dims(shape)
    ext = max(n, kxn * ny * nz, kxn * kyn * nz, kxn * kyn * kzn)
    return 2 * 6 * 8 * ext


def request_bytes(shape, spectrum_resident):
    """Peak bytes a request needs at admission: its state, plus the spectrum
    and its build buffers when the spectrum is not resident yet."""
    b = state_bytes(shape)
    if not spectrum_resident:
        b += spectrum_bytes(shape) + build_bytes(shape)
    return b


MMP_E_TIMEOUT = -5     # status of include/mmp.h: a host-side deadline passed
MMP_E_CUDA = -3


class Request:
    def __init__(self, rid, workload, arrival, torque_tol, max_time, deadline=None):
        self.id = rid
        self.workload = workload
        self.arrival = float(arrival)
        self.torque_tol = float(torque_tol)
        self.max_time = float(max_time)
        self.deadline = None if deadline is None else float(deadline)   # wall seconds after arrival
        self.accepted = None          # left the queue (its build started, or it joined)
        self.admitted = None
        self.done = None
        self.status = None
        self.mag = None
        self.bytes = 0
        self.result = None
        self.sim_time = None          # simulated time at the end of the solve (s)

    @property
    def time_capped(self):
        """The solve ended on its simulated-time limit, not on the torque tolerance."""
        return self.sim_time is not None and self.sim_time >= self.max_time * (1.0 - 1e-9)

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival

    def expired(self, now):
        return self.deadline is not None and now > self.arrival + self.deadline


def _make_magnet(w, dt0):
    import torch
    mag = Magnet.from_problem(w.problem)
    mag.set_m(0, torch.from_numpy(np.ascontiguousarray(w.m0[0])).cuda())
    mag.set_solver(adaptive=True, dt=dt0, tol=w.tol, dt_min=w.dt_min, dt_max=w.dt_max)
    sh = mag.get_shape()
    ny = w.problem.shape[1]
    if not (sh["engine"] == 3 and _nice(ny) // sh["R"] == 1024):
        mag.autotune(batch=True)      # cached per geometry: the batch shape (block engine)
    # else: the warp passes A, B and C (Px = 2048, folded y length 1024), which a
    # batch member runs with launches of its own
    return mag


def _build_async(w, dt0):
    """_make_magnet on the worker thread, on a CUDA stream of its own (the
    context keeps it), finished on the device before it returns."""
    import torch
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        mag = _make_magnet(w, dt0)
        side.synchronize()
    return mag


class RelaxServer:
    """Admission by memory budget + continuous batching of relax solves."""

    def __init__(self, budget_bytes=150e9, attempts_per_round=4, dt0=1e-14, keep_results=False,
                 build_async=True):
        self.budget = float(budget_bytes)
        self.attempts = int(attempts_per_round)
        self.dt0 = float(dt0)
        self.keep = keep_results
        self.batch = Batch()
        self.queue = collections.deque()
        self.active = []
        self.pending = []                         # (request, future): contexts being built
        self.building = {}                        # (shape, cell) -> future of its first context
        self.finished = []
        self.used = 0.0                           # resident bytes: states + resident spectra (+ builds)
        self.spectra = collections.Counter()      # (shape, cell) -> requests using its spectrum
        self.peak_members = 0
        self.builds_overlapped = 0                # lock steps run while a build was in flight
        self._pool = concurrent.futures.ThreadPoolExecutor(max_workers=1) if build_async else None

    def submit(self, req):
        self.queue.append(req)

    def _key(self, req):
        p = req.workload.problem
        return (tuple(p.shape), tuple(p.cell))

    def _finish(self, req, now, status):
        req.done = now
        req.status = status
        self.finished.append(req)

    def _join(self, req, now):
        key = self._key(req)
        self.spectra[key] += 1
        self.batch.add(req.mag, "relax", req.torque_tol, req.max_time)
        req.admitted = now
        self.active.append(req)

    def _admit(self, now):
        while self.queue and self.queue[0].arrival <= now:
            req = self.queue[0]
            if req.expired(now):                       # never admitted: deadline passed in the queue
                self.queue.popleft()
                self._finish(req, now, MMP_E_TIMEOUT)
                continue
            key, shape = self._key(req), req.workload.problem.shape
            if key in self.building:
                break                                  # its spectrum is being built (FIFO)
            new = self.spectra[key] == 0
            if (self.active or self.pending) and self.used + request_bytes(shape, not new) > self.budget:
                break                                  # wait for memory (FIFO)
            self.queue.popleft()
            req.accepted = now
            req.bytes = state_bytes(shape)
            if new and self._pool is not None:
                # build on the worker thread while the batch keeps stepping
                self.used += req.bytes + spectrum_bytes(shape) + build_bytes(shape)
                fut = self._pool.submit(_build_async, req.workload, self.dt0)
                self.building[key] = fut
                self.pending.append((req, fut))
                continue
            req.mag = _make_magnet(req.workload, self.dt0)   # builds the spectrum if new (and frees the buffers)
            self.used += req.bytes + (spectrum_bytes(shape) if new else 0)
            self._join(req, now)
        self.peak_members = max(self.peak_members, len(self.active))

    def _collect(self, now):
        """Requests whose context build has finished join the batch (in
        order); a failed build ends its request with the library's status."""
        while self.pending and self.pending[0][1].done():
            req, fut = self.pending.pop(0)
            key, shape = self._key(req), req.workload.problem.shape
            del self.building[key]
            self.used -= build_bytes(shape)
            try:
                req.mag = fut.result()
            except Exception as e:                     # noqa: BLE001 - reported as the request's status
                self.used -= req.bytes + spectrum_bytes(shape)
                self._finish(req, now, getattr(e, "status", MMP_E_CUDA))
                continue
            if req.expired(now):
                req.mag.close()
                req.mag = None
                self.used -= req.bytes + spectrum_bytes(shape)
                self._finish(req, now, MMP_E_TIMEOUT)
                continue
            self._join(req, now)
        self.peak_members = max(self.peak_members, len(self.active))

    def _release(self, req):
        req.mag.close()
        req.mag = None
        self.used -= req.bytes
        key = self._key(req)
        self.spectra[key] -= 1
        if self.spectra[key] == 0:                     # the library freed the shared spectrum
            self.used -= spectrum_bytes(req.workload.problem.shape)

    def _retire(self, now):
        keep = []
        for req in self.active:
            done, status = self.batch.status(req.mag)
            if not done and not req.expired(now):
                keep.append(req)
                continue
            self.batch.remove(req.mag)
            req.sim_time = _sim_time(req.mag)
            if not done:
                status = MMP_E_TIMEOUT
            elif self.keep:
                req.result = _read_m(req.mag)
            self._release(req)
            self._finish(req, now, status)
        self.active = keep

    def run(self, requests, clock=time.perf_counter):
        """Serve `requests` (arrival times relative to the start) in real
        time; returns them with admitted/done times filled in."""
        for r in sorted(requests, key=lambda r: r.arrival):
            self.submit(r)
        t0 = clock()
        while self.queue or self.active or self.pending:
            now = clock() - t0
            self._collect(now)
            self._admit(now)
            if not self.active:
                if self.pending:
                    concurrent.futures.wait([self.pending[0][1]], timeout=0.01)
                elif self.queue:
                    time.sleep(max(0.0, min(0.01, self.queue[0].arrival - now)))
                continue
            if self.pending:
                self.builds_overlapped += 1
            self.batch.advance(self.attempts)
            self._retire(clock() - t0)
        return self.finished

    def close(self):
        for req, fut in self.pending:
            try:
                fut.result().close()
            except Exception:                          # noqa: BLE001 - closing anyway
                pass
        self.pending = []
        if self._pool is not None:
            self._pool.shutdown(wait=True)
        for req in self.active:
            self.batch.remove(req.mag)
            req.mag.close()
        self.active = []
        self.batch.close()


def _sim_time(mag):
    try:
        return float(mag.time()["t"])
    except (AttributeError, KeyError, TypeError):
        return None


def _read_m(mag):
    import torch
    nx, ny, nz = mag.shape
    out = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    mag.get_m(0, out)
    return out.cpu().numpy()


def serve_one_at_a_time(requests, dt0=1e-14, keep_results=False, clock=time.perf_counter):
    """The plain path: each request relaxed alone (mmp_relax) in arrival
    order, the next one starting when the previous has finished."""
    t0 = clock()
    out = []
    for req in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if now < req.arrival:
            time.sleep(req.arrival - now)
        req.admitted = clock() - t0
        mag = _make_magnet(req.workload, dt0)
        mag.relax(torque_tol=req.torque_tol, max_time=req.max_time)
        req.sim_time = _sim_time(mag)
        if keep_results:
            req.result = _read_m(mag)
        mag.close()
        req.done = clock() - t0
        req.status = 0
        out.append(req)
    return out


def latency_stats(reqs):
    lat = np.array([r.latency for r in reqs], dtype=np.float64)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    capped = [getattr(r, "time_capped", False) for r in reqs]
    return {"solves": len(reqs), "solves_per_s": len(reqs) / span, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()), "span_s": span,
            "time_capped_fraction": float(np.mean(capped)) if capped else 0.0}
