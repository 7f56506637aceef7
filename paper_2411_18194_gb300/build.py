"""Build libmmp.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit is compiled in its own nvcc process (in
parallel), then linked into paper_2411_18194_gb300/_lib/libmmp.so with the
CUDA runtime linked statically.

ptxas reports every kernel's registers and spills; the build fails if a
kernel spills more than SPILL_LIMIT bytes.  (A loop around an inlined FFT
body once made the compiler cut a kernel to 32 registers and spill
kilobytes per thread, several times slower, with no other symptom.)
"""
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT, "libmmp.so")
CHECKED_LIB = os.path.join(OUT, "checked", "libmmp_checked.so")
SOURCES = ["mmp.cu", "pass_a.cu", "pass_b.cu", "field.cu", "elastic.cu", "tensor.cu", "noalloc.cu", "batch.cu", "batch_a.cu", "batch_b.cu", "batch_c.cu", "energy.cu", "passb_w8.cu", "passb_w16.cu", "passb_w32.cu", "passa_w.cu", "field_w.cu", "peak.cu", "batch_w.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SPILL_LIMIT = 1024   # bytes of spill stores per thread
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
         "-I" + SRC]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def check_spills(ptxas_out):
    """Kernels whose spill stores exceed SPILL_LIMIT in a ptxas -v log."""
    bad, name = [], None
    for line in ptxas_out.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and name and int(m.group(1)) > SPILL_LIMIT:
            bad.append("%s: %s bytes spill stores" % (name, m.group(1)))
    return bad


def compile_command(src, obj, checked=False, extra=()):
    """nvcc command of one translation unit (the bounds-checked build adds
    -DMMP_CHECK_BOUNDS)."""
    cmd = [nvcc(), "-c", os.path.join(SRC, src), "-o", obj] + ARCH + FLAGS + ["-Xptxas", "-v"] + list(extra)
    if checked:
        cmd.append("-DMMP_CHECK_BOUNDS")
    return cmd


def build(verbose=False, extra=(), checked=False):
    """Compile every translation unit and link the library: libmmp.so, or
    with `checked` the bounds-checked debug build _lib/checked/libmmp_checked.so
    (every kernel index check armed; its spills are not limited)."""
    out = os.path.join(OUT, "checked") if checked else OUT
    lib_path = CHECKED_LIB if checked else LIB
    os.makedirs(out, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(out, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = compile_command(src, obj, checked, extra)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed, spills = [], []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append(" ".join(cmd))
        if not checked:
            spills += check_spills(out)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    if spills:
        raise RuntimeError("kernels spill more than %d bytes:\n" % SPILL_LIMIT + "\n".join(spills))
    tmp = lib_path + ".tmp"
    link = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout)
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, checked="--checked" in sys.argv))
