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
              "mmp_set_global", "mmp_enable_terms", "mmp_set_m", "mmp_get_m", "mmp_set_solver",
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
