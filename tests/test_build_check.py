"""The build's register-spill guard (paper_2411_18194_gb300/build.py)."""
import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _build_module():
    path = os.path.join(HERE, "..", "paper_2411_18194_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("mmp_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_spill_guard_flags_only_large_spills():
    b = _build_module()
    log = "\n".join([
        "ptxas info    : Compiling entry function '_Z4bigv' for 'sm_103a'",
        "ptxas info    : Function properties for _Z4bigv",
        "    4368 bytes stack frame, 20016 bytes spill stores, 17988 bytes spill loads",
        "ptxas info    : Used 32 registers, used 1 barriers",
        "ptxas info    : Compiling entry function '_Z5smallv' for 'sm_103a'",
        "    8 bytes stack frame, 20 bytes spill stores, 20 bytes spill loads",
    ])
    bad = b.check_spills(log)
    assert len(bad) == 1 and "_Z4bigv" in bad[0]
    assert b.check_spills("") == []
