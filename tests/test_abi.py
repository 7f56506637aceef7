"""The C-ABI library loads and exports every function include/*.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mmp_[a-z0-9_]+)\s*\(", text,
                            flags=re.M)
    return sorted(set(names))


def _lib():
    from paper_2411_18194_gb300 import binding
    if not os.path.exists(binding.library_path()):
        pytest.skip("libmmp.so not built (run __graft_entry__.build())")
    return binding.library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mmp_create", "mmp_destroy", "mmp_set_region_map", "mmp_set_param", "mmp_set_param3",
              "mmp_set_global", "mmp_enable_terms", "mmp_set_boundary", "mmp_set_m", "mmp_get_m", "mmp_set_solver",
              "mmp_eval_field", "mmp_step", "mmp_run", "mmp_relax", "mmp_get_time", "mmp_get_state",
              "mmp_set_state", "mmp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_matches_header():
    lib = _lib()
    text = open(os.path.join(ROOT, "include", "mmp.h")).read()
    ver = int(re.search(r"#define MMP_VERSION (\d+)", text).group(1))
    assert lib.mmp_version() == ver


def test_binding_ids_match_header_enums():
    from paper_2411_18194_gb300 import binding
    text = open(os.path.join(ROOT, "include", "mmp.h")).read()
    enums = dict((k, int(v)) for k, v in re.findall(r"(MMP_[A-Z0-9_]+)\s*=\s*(-?\d+)", text))
    for name, v in binding.PARAM_IDS.items():
        assert enums["MMP_" + name] == v
    for name, v in binding.PARAM3_IDS.items():
        assert enums["MMP_" + name] == v
    for name, v in binding.GLOBAL_IDS.items():
        assert enums["MMP_" + name] == v
    for name, v in binding.TERM_BITS.items():
        assert enums["MMP_T_" + name] == v
    for name, v in binding.METHODS.items():
        assert enums["MMP_" + name] == v
    for name, v in binding.GOALS.items():
        assert enums["MMP_GOAL_" + name.upper()] == v
    for name, v in binding.BOUNDARIES.items():
        assert enums["MMP_BC_" + name.upper()] == v
    for v, name in binding.STATUS.items():
        if v:
            assert enums[name] == v


def test_create_rejects_bad_arguments_before_touching_the_device():
    lib = _lib()
    from paper_2411_18194_gb300 import binding
    ctx = ctypes.c_void_p()
    rc = lib.mmp_create(ctypes.byref(ctx), 0, 4, 4, 1e-9, 1e-9, 1e-9, 1, None, binding.ALLOC_FN(),
                        binding.FREE_FN(), None)
    assert rc == -1 and b"extents" in lib.mmp_last_error()
    rc = lib.mmp_create(ctypes.byref(ctx), 4, 4, 4, 1e-9, 1e-9, 1e-9, 3, None, binding.ALLOC_FN(),
                        binding.FREE_FN(), None)
    assert rc == -1 and b"sublattices" in lib.mmp_last_error()


def test_host_tableaux_equal_the_oracle_fractions():
    """The library's FP64 tableaux (csrc/dp45.h, compiled here with g++) equal
    the oracle's exact fractions to double rounding, for every method."""
    import shutil
    import subprocess
    import tempfile
    from oracle.dp45 import METHODS
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    src = r'''
#include <cstdio>
#include "dp45.h"
int main() {
  for (int m = 0; m < 5; ++m) {
    const mmp::Tableau& T = mmp::tableau(m);
    std::printf("%d %d %.17g\n", m, T.S, T.exponent);
    for (int i = 1; i <= T.S; ++i)
      for (int j = 0; j < i; ++j) std::printf("a %d %d %d %.17g\n", m, i, j, T.a[i][j]);
    for (int j = 0; j <= T.S; ++j) std::printf("e %d %d %.17g\n", m, j, T.e[j]);
  }
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call([gxx, "-std=c++17", "-I", os.path.join(ROOT, "paper_2411_18194_gb300", "csrc"),
                               c, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    ids = {0: "DP45", 1: "HEUN", 2: "BS23", 3: "CASHKARP", 4: "RKF45"}
    seen = 0
    for line in out:
        f = line.split()
        if not f:
            continue
        if f[0] == "a":
            m, i, j, v = ids[int(f[1])], int(f[2]), int(f[3]), float(f[4])
            row = METHODS[m]["A"][i]
            ref = float(row[j]) if j < len(row) else 0.0
            assert abs(v - ref) <= 4e-16 * max(1.0, abs(ref)), (m, i, j, v, ref)
            seen += 1
        elif f[0] == "e":
            m, j, v = ids[int(f[1])], int(f[2]), float(f[3])
            ref = float(METHODS[m]["E"][j])
            assert abs(v - ref) <= 4e-16 * max(1.0, abs(ref)) + 1e-17, (m, j, v, ref)
            seen += 1
        else:
            m = ids[int(f[0])]
            assert int(f[1]) == METHODS[m]["S"] and float(f[2]) == METHODS[m]["exponent"]
    assert seen > 50


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built library every entry point raises."""
    from paper_2411_18194_gb300 import binding
    monkeypatch.setattr(binding, "_LIB_PATH", str(tmp_path / "libmmp.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="libmmp.so not found"):
        binding.library()
    with pytest.raises(RuntimeError, match="libmmp.so not found"):
        binding.Magnet((4, 4, 1), (1e-9, 1e-9, 1e-9), 1)
