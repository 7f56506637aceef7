"""ctypes binding of libmmp.so (include/mmp.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device memory comes from PyTorch's caching allocator (passed to
mmp_create as the context allocator) and work is enqueued on the current
PyTorch CUDA stream unless another stream is given.  If the library is
missing the import-time lookup fails loudly; there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MMP_CHECK_BOUNDS=1 loads the bounds-checked debug build (build.py
# build(checked=True)): every kernel index check armed, MMP_E_BOUNDS on a
# failed one.  It is a debugging aid, slower, never the default.
_CHECKED = os.environ.get("MMP_CHECK_BOUNDS", "") == "1"
_LIB_PATH = (os.path.join(_HERE, "_lib", "checked", "libmmp_checked.so") if _CHECKED
             else os.path.join(_HERE, "_lib", "libmmp.so"))

TERM_BITS = {"DEMAG": 1, "EXCH": 2, "ANIS": 4, "DMI": 8, "ZEEMAN": 16, "AFM": 32, "MEL": 64,
             "ELASTIC": 128, "CUBIC": 256}
PARAM_IDS = {"MS": 0, "AEX": 1, "ALPHA": 2, "KU1": 3, "KU2": 4, "KB1": 5, "DIND": 6, "B1": 7, "B2": 8,
             "KC1": 9}
PARAM3_IDS = {"ANIS_U": 0, "ANIS_UB": 1, "B_EXT": 2, "ANIS_C1": 3, "ANIS_C2": 4}
GLOBAL_IDS = {"A0": 0, "A12": 1, "LATTICE_A": 2, "C11": 3, "C12": 4, "C44": 5, "RHO": 6, "ETA": 7}
STATUS = {0: "MMP_OK", -1: "MMP_E_INVAL", -2: "MMP_E_OOM", -3: "MMP_E_CUDA", -4: "MMP_E_NONFINITE",
          -5: "MMP_E_TIMEOUT", -6: "MMP_E_STATE", -7: "MMP_E_BOUNDS"}

GOALS = {"steps": 0, "run": 1, "relax": 2}
METHODS = {"DP45": 0, "HEUN": 1, "BS23": 2, "CASHKARP": 3, "RKF45": 4}
TUNE_BATCH, TUNE_FORCE = 1, 2
BOUNDARIES = {"neumann": 0, "open": 1}


class Shape(ctypes.Structure):
    """mmp_shape: launch shape of the demag passes."""
    _fields_ = [("ty", ctypes.c_int), ("radix_x", ctypes.c_int), ("radix_y", ctypes.c_int),
                ("R", ctypes.c_int), ("stage_kernel", ctypes.c_int), ("tyc", ctypes.c_int),
                ("engine", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_c = ctypes
_SIGS = {
    "mmp_version": ([], _c.c_int),
    "mmp_last_error": ([], _c.c_char_p),
    "mmp_create": ([_c.POINTER(_c.c_void_p), _c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_double,
                    _c.c_double, _c.c_int, _c.c_void_p, ALLOC_FN, FREE_FN, _c.c_void_p], _c.c_int),
    "mmp_destroy": ([_c.c_void_p], _c.c_int),
    "mmp_set_region_map": ([_c.c_void_p, _c.c_void_p], _c.c_int),
    "mmp_set_param": ([_c.c_void_p, _c.c_int, _c.c_int, _c.c_int, _c.c_double], _c.c_int),
    "mmp_set_param3": ([_c.c_void_p, _c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_double,
                        _c.c_double], _c.c_int),
    "mmp_set_global": ([_c.c_void_p, _c.c_int, _c.c_double], _c.c_int),
    "mmp_enable_terms": ([_c.c_void_p, _c.c_uint], _c.c_int),
    "mmp_set_boundary": ([_c.c_void_p, _c.c_int], _c.c_int),
    "mmp_set_m": ([_c.c_void_p, _c.c_int, _c.c_void_p, _c.c_int], _c.c_int),
    "mmp_get_m": ([_c.c_void_p, _c.c_int, _c.c_void_p], _c.c_int),
    "mmp_set_elastic": ([_c.c_void_p, _c.c_void_p, _c.c_void_p], _c.c_int),
    "mmp_get_elastic": ([_c.c_void_p, _c.c_void_p, _c.c_void_p], _c.c_int),
    "mmp_set_solver": ([_c.c_void_p, _c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_double,
                        _c.c_double], _c.c_int),
    "mmp_eval_field": ([_c.c_void_p, _c.c_int, _c.c_void_p, _c.c_void_p], _c.c_int),
    "mmp_step": ([_c.c_void_p, _c.c_int], _c.c_int),
    "mmp_run": ([_c.c_void_p, _c.c_double], _c.c_int),
    "mmp_relax": ([_c.c_void_p, _c.c_double, _c.c_double, _c.c_double], _c.c_int),
    "mmp_get_time": ([_c.c_void_p, _c.POINTER(_c.c_double), _c.POINTER(_c.c_double),
                      _c.POINTER(_c.c_longlong), _c.POINTER(_c.c_longlong), _c.POINTER(_c.c_longlong)],
                     _c.c_int),
    "mmp_get_state": ([_c.c_void_p, _c.c_void_p, _c.POINTER(_c.c_size_t)], _c.c_int),
    "mmp_set_state": ([_c.c_void_p, _c.c_void_p, _c.c_size_t], _c.c_int),
    "mmp_sync": ([_c.c_void_p], _c.c_int),
    "mmp_profile": ([_c.c_void_p, _c.c_int], _c.c_int),
    "mmp_demag_noalloc": ([_c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_double, _c.c_void_p,
                           _c.c_void_p, _c.c_void_p], _c.c_int),
    "mmp_profile_read": ([_c.c_void_p, _c.c_int, _c.POINTER(_c.c_longlong), _c.POINTER(_c.c_double)],
                         _c.c_int),
    "mmp_get_shape": ([_c.c_void_p, _c.POINTER(Shape)], _c.c_int),
    "mmp_energy": ([_c.c_void_p, _c.POINTER(_c.c_double)], _c.c_int),
    "mmp_set_shape": ([_c.c_void_p, _c.POINTER(Shape)], _c.c_int),
    "mmp_autotune": ([_c.c_void_p, _c.c_int, _c.POINTER(Shape), _c.POINTER(_c.c_double)], _c.c_int),
    "mmp_batch_create": ([_c.POINTER(_c.c_void_p), _c.c_void_p], _c.c_int),
    "mmp_batch_destroy": ([_c.c_void_p], _c.c_int),
    "mmp_batch_add": ([_c.c_void_p, _c.c_void_p, _c.c_int, _c.c_double, _c.c_double], _c.c_int),
    "mmp_batch_remove": ([_c.c_void_p, _c.c_void_p], _c.c_int),
    "mmp_batch_size": ([_c.c_void_p, _c.POINTER(_c.c_int)], _c.c_int),
    "mmp_batch_advance": ([_c.c_void_p, _c.c_int, _c.POINTER(_c.c_int)], _c.c_int),
    "mmp_batch_status": ([_c.c_void_p, _c.c_void_p, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)], _c.c_int),
    "mmp_batch_launches": ([_c.c_void_p, _c.POINTER(_c.c_longlong)], _c.c_int),
    "mmp_batch_profile": ([_c.c_void_p, _c.c_int], _c.c_int),
    "mmp_batch_profile_read": ([_c.c_void_p, _c.c_int, _c.POINTER(_c.c_longlong), _c.POINTER(_c.c_double)],
                               _c.c_int),
    "mmp_fp32_peak": ([_c.c_void_p, _c.c_int, _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)], _c.c_int),
}
KERNEL_IDS = {"pass_a": 0, "pass_b": 1, "field": 2, "assemble": 3, "strain": 4, "elastic": 5}

_lib = None


def library_path():
    return _LIB_PATH


def library():
    """The loaded libmmp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("%s not found: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                               " (the bounds-checked one with `python -m paper_2411_18194_gb300.build "
                               "--checked`)" % _LIB_PATH)
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


class MmpError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, message))
        self.status = status


def _check(status):
    if status != 0:
        raise MmpError(status, library().mmp_last_error().decode(errors="replace"))
    return status


def _ptr(a):
    """Raw pointer of a torch tensor (device or host) or a numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr()


class _TorchAllocator:
    """Device allocations of the library served by PyTorch's caching allocator."""

    def __init__(self, device, stream):
        import torch
        self._torch = torch
        self._device = device
        self._stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self._device, self._stream)
        except Exception:
            return None

    def _free(self, ptr, user):
        self._torch.cuda.caching_allocator_delete(ptr)


def demag_noalloc(shape, cell, M, B, stream=None):
    """B = demag field of M (device float32 tensors [3][nz][ny][nx]) through
    mmp_demag_noalloc: no device allocation, static scratch inside the
    library (see include/mmp.h for its size limit and sharing rules)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    nx, ny, nz = (int(v) for v in shape)
    cx, cy, cz = (float(c) for c in cell)
    _check(library().mmp_demag_noalloc(nx, ny, nz, cx, cy, cz, _ptr(M), _ptr(B), ctypes.c_void_p(handle)))
    return B


def fp32_peak(reps=20, stream=None):
    """Measured FP32 FMA throughput of the current device: (GFLOP/s, ms per
    launch) of the best of `reps` launches (mmp_fp32_peak)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    g, ms = ctypes.c_double(), ctypes.c_double()
    _check(library().mmp_fp32_peak(ctypes.c_void_p(handle), int(reps), ctypes.byref(g), ctypes.byref(ms)))
    return g.value, ms.value


class Magnet:
    """One magnet on a regular grid (an mmp_ctx).

    Vector fields are float32 [3][nz][ny][nx]; methods accept torch tensors
    (device or host) or C-contiguous numpy arrays.
    """

    def __init__(self, shape, cell, n_sub=1, stream=None, torch_allocator=True, allocator=None):
        """`allocator`: an object with ctypes callbacks `alloc` (ALLOC_FN) and
        `free` (FREE_FN) serving the context's device allocations (e.g. one
        that refuses some, to exercise the MMP_E_OOM paths); default
        PyTorch's caching allocator (`torch_allocator`), else cudaMalloc."""
        lib = library()
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nx, ny, nz)
        self.cell = tuple(float(c) for c in cell)
        self.n_sub = int(n_sub)
        self._alloc = None
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        alloc_fn, free_fn = ALLOC_FN(), FREE_FN()
        if allocator is not None:
            self._alloc = allocator
            alloc_fn, free_fn = allocator.alloc, allocator.free
        elif torch_allocator:
            self._alloc = _TorchAllocator(torch.cuda.current_device(), stream)
            alloc_fn, free_fn = self._alloc.alloc, self._alloc.free
        ctx = ctypes.c_void_p()
        _check(lib.mmp_create(ctypes.byref(ctx), nx, ny, nz, *self.cell, self.n_sub,
                              ctypes.c_void_p(handle), alloc_fn, free_fn, None))
        self._ctx = ctx

    # ------------------------------------------------------------ lifetime --
    def close(self):
        if getattr(self, "_ctx", None):
            library().mmp_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------- parameters --
    def set_region_map(self, regions):
        regions = np.ascontiguousarray(regions, dtype=np.uint8) if isinstance(regions, np.ndarray) else regions
        _check(library().mmp_set_region_map(self._ctx, _ptr(regions)))

    def set_param(self, name, value, sub=-1, region=-1):
        _check(library().mmp_set_param(self._ctx, sub, PARAM_IDS[name], region, float(value)))

    def set_param3(self, name, vec, sub=-1, region=-1):
        x, y, z = (float(v) for v in vec)
        _check(library().mmp_set_param3(self._ctx, sub, PARAM3_IDS[name], region, x, y, z))

    def set_global(self, name, value):
        _check(library().mmp_set_global(self._ctx, GLOBAL_IDS[name], float(value)))

    def set_boundary(self, bc):
        """Boundary condition of the exchange and DMI stencils: "neumann" or "open"."""
        _check(library().mmp_set_boundary(self._ctx, BOUNDARIES[bc]))

    def enable_terms(self, terms):
        mask = terms if isinstance(terms, int) else sum(TERM_BITS[t] for t in terms)
        _check(library().mmp_enable_terms(self._ctx, mask))

    # --------------------------------------------------------------- state --
    def set_m(self, sub, m, normalize=False):
        _check(library().mmp_set_m(self._ctx, sub, _ptr(m), int(bool(normalize))))

    def get_m(self, sub, out):
        _check(library().mmp_get_m(self._ctx, sub, _ptr(out)))
        return out

    def set_elastic(self, u=None, v=None):
        _check(library().mmp_set_elastic(self._ctx, _ptr(u), _ptr(v)))

    def get_elastic(self, u=None, v=None):
        _check(library().mmp_get_elastic(self._ctx, _ptr(u), _ptr(v)))
        return u, v

    # -------------------------------------------------------------- solver --
    def set_solver(self, adaptive=False, dt=1e-13, tol=1e-5, dt_min=1e-18, dt_max=1e-11, method="DP45"):
        _check(library().mmp_set_solver(self._ctx, METHODS[method], int(bool(adaptive)), dt, tol, dt_min, dt_max))

    def eval_field(self, sub=0, B=None, tau=None):
        _check(library().mmp_eval_field(self._ctx, sub, _ptr(B), _ptr(tau)))
        return B, tau

    def step(self, nsteps=1):
        _check(library().mmp_step(self._ctx, int(nsteps)))

    def run(self, duration):
        _check(library().mmp_run(self._ctx, float(duration)))

    def relax(self, torque_tol=1e-4, max_time=10e-9, timeout_s=0.0):
        _check(library().mmp_relax(self._ctx, float(torque_tol), float(max_time), float(timeout_s)))

    def time(self):
        t, dt = ctypes.c_double(), ctypes.c_double()
        s, r, e = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(library().mmp_get_time(self._ctx, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(s),
                                      ctypes.byref(r), ctypes.byref(e)))
        return dict(t=t.value, dt=dt.value, steps=s.value, rejected=r.value, evals=e.value)

    def get_state(self):
        size = ctypes.c_size_t()
        _check(library().mmp_get_state(self._ctx, None, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        _check(library().mmp_get_state(self._ctx, buf, ctypes.byref(size)))
        return bytes(buf.raw[:size.value])

    def set_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(library().mmp_set_state(self._ctx, buf, len(blob)))

    def sync(self):
        _check(library().mmp_sync(self._ctx))

    def profile(self, enable=True):
        """Start (reset) or stop per-kernel CUDA-event timing."""
        _check(library().mmp_profile(self._ctx, int(bool(enable))))

    def profile_read(self):
        """{kernel: (launches, total device ms)} since the last reset."""
        out = {}
        for name, k in KERNEL_IDS.items():
            n, ms = ctypes.c_longlong(), ctypes.c_double()
            _check(library().mmp_profile_read(self._ctx, k, ctypes.byref(n), ctypes.byref(ms)))
            if n.value:
                out[name] = (n.value, ms.value)
        return out

    def energy(self):
        """{term name: energy (J)} of the enabled terms (mmp_energy)."""
        buf = (ctypes.c_double * 9)()
        _check(library().mmp_energy(self._ctx, buf))
        return {name: buf[bit.bit_length() - 1] for name, bit in TERM_BITS.items()}

    # -------------------------------------------------------------- shape --
    def get_shape(self):
        sh = Shape()
        _check(library().mmp_get_shape(self._ctx, ctypes.byref(sh)))
        return sh.as_dict()

    def set_shape(self, **kw):
        """Change fields of the launch shape (ty, radix_x, radix_y, R, stage_kernel, tyc)."""
        d = self.get_shape()
        d.update(kw)
        sh = Shape(**d)
        _check(library().mmp_set_shape(self._ctx, ctypes.byref(sh)))
        return d

    def autotune(self, batch=False, force=False):
        """Time the valid shapes, keep the fastest; returns (shape, ms per evaluation)."""
        sh, ms = Shape(), ctypes.c_double()
        flags = (TUNE_BATCH if batch else 0) | (TUNE_FORCE if force else 0)
        _check(library().mmp_autotune(self._ctx, flags, ctypes.byref(sh), ctypes.byref(ms)))
        return sh.as_dict(), ms.value

    # ------------------------------------------------------------ helpers --
    @classmethod
    def from_problem(cls, problem, **kw):
        """A context set up from an object with the attributes of
        inputs.Problem (shape, cell, n_sub, regions, scal, vec, glob, terms,
        open_bc)."""
        mag = cls(problem.shape, problem.cell, problem.n_sub, **kw)
        regions = np.ascontiguousarray(problem.regions, dtype=np.uint8)
        used = np.unique(regions)
        if used.size > 1 or used[0] != 0:
            mag.set_region_map(regions)
        for name in PARAM_IDS:
            table = problem.scal[name]
            for s in range(problem.n_sub):
                vals = table[s, used]
                if np.all(vals == vals[0]):
                    mag.set_param(name, vals[0], s, -1)
                else:
                    for r in used:
                        mag.set_param(name, table[s, r], s, int(r))
        for name in PARAM3_IDS:
            table = problem.vec[name]
            for s in range(problem.n_sub):
                vals = table[s, used]
                if np.all(vals == vals[0]):
                    mag.set_param3(name, vals[0], s, -1)
                else:
                    for r in used:
                        mag.set_param3(name, table[s, r], s, int(r))
        for name in GLOBAL_IDS:
            mag.set_global(name, problem.glob.get(name, 0.0))
        mag.enable_terms(sorted(problem.terms))
        if getattr(problem, "open_bc", False):
            mag.set_boundary("open")
        return mag


class Batch:
    """A set of Magnets advanced together (an mmp_batch).

    Members keep their own state; between advance() calls each Magnet can be
    read as usual.  Goals: ("steps", n), ("run", duration), ("relax",
    torque_tol, max_time)."""

    def __init__(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        b = ctypes.c_void_p()
        _check(library().mmp_batch_create(ctypes.byref(b), ctypes.c_void_p(handle)))
        self._b = b
        self._members = {}

    def close(self):
        if getattr(self, "_b", None):
            library().mmp_batch_destroy(self._b)
            self._b = None
            self._members = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, mag, goal="steps", a=0.0, c=0.0):
        _check(library().mmp_batch_add(self._b, mag._ctx, GOALS[goal], float(a), float(c)))
        self._members[id(mag)] = mag

    def remove(self, mag):
        _check(library().mmp_batch_remove(self._b, mag._ctx))
        self._members.pop(id(mag), None)

    def __len__(self):
        n = ctypes.c_int()
        _check(library().mmp_batch_size(self._b, ctypes.byref(n)))
        return n.value

    def advance(self, max_attempts=1 << 30):
        """Lock-step attempts until every member's goal is met (or max_attempts);
        returns the number of members not done."""
        n = ctypes.c_int()
        _check(library().mmp_batch_advance(self._b, int(max_attempts), ctypes.byref(n)))
        return n.value

    def status(self, mag):
        """(done, status) of a member."""
        d, st = ctypes.c_int(), ctypes.c_int()
        _check(library().mmp_batch_status(self._b, mag._ctx, ctypes.byref(d), ctypes.byref(st)))
        return bool(d.value), st.value

    def launches(self):
        n = ctypes.c_longlong()
        _check(library().mmp_batch_launches(self._b, ctypes.byref(n)))
        return n.value

    def profile(self, enable=True):
        """Start (reset) or stop per-pass CUDA-event timing."""
        _check(library().mmp_batch_profile(self._b, int(bool(enable))))

    def profile_read(self):
        """{pass: (launches, total device ms)} since the last reset."""
        out = {}
        for name, k in (("pass_a", 0), ("pass_b", 1), ("field", 2)):
            n, ms = ctypes.c_longlong(), ctypes.c_double()
            _check(library().mmp_batch_profile_read(self._b, k, ctypes.byref(n), ctypes.byref(ms)))
            if n.value:
                out[name] = (n.value, ms.value)
        return out
