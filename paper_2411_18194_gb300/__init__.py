"""GB300-native micromagnetic field/torque engine (arXiv 2411.18194 method).

The computation runs in libmmp.so (hand-written sm_103a CUDA kernels behind
the C-ABI of include/mmp.h); this package is a thin ctypes binding.
"""
from .binding import (Magnet, Batch, Shape, MmpError, TERM_BITS, PARAM_IDS, PARAM3_IDS, GLOBAL_IDS,
                      KERNEL_IDS, GOALS, METHODS, library, library_path, demag_noalloc, fp32_peak)

__all__ = ["Magnet", "Batch", "Shape", "MmpError", "TERM_BITS", "PARAM_IDS", "PARAM3_IDS", "GLOBAL_IDS",
           "KERNEL_IDS", "GOALS", "METHODS", "library", "library_path", "demag_noalloc", "fp32_peak"]
