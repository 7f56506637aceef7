"""The bounds-checked debug build (MMP_CHECK_BOUNDS) on CPU: its compile
command, the library the binding loads for it, and that the checked
sources compile for sm_103a (nvcc cross-compiles without a GPU)."""
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_defines_the_macro_and_has_its_own_library():
    from paper_2411_18194_gb300 import build
    plain = build.compile_command("field_w.cu", "x.o")
    checked = build.compile_command("field_w.cu", "x.o", checked=True)
    assert "-DMMP_CHECK_BOUNDS" in checked and "-DMMP_CHECK_BOUNDS" not in plain
    assert build.CHECKED_LIB != build.LIB and build.CHECKED_LIB.endswith("libmmp_checked.so")


def test_binding_loads_the_checked_library_when_asked():
    code = "import paper_2411_18194_gb300.binding as b; print(b.library_path())"
    env = dict(os.environ, MMP_CHECK_BOUNDS="1")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip().endswith(os.path.join("checked", "libmmp_checked.so"))
    env.pop("MMP_CHECK_BOUNDS")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.stdout.strip().endswith(os.path.join("_lib", "libmmp.so"))


def test_checked_pass_c_compiles(tmp_path):
    """The warp pass C with its index checks armed (the largest set: T
    gathers, stencil rows, neighbour planes, stores) compiles for sm_103a."""
    from paper_2411_18194_gb300 import build
    cmd = build.compile_command("field_w.cu", str(tmp_path / "field_w.o"), checked=True)
    t0 = time.time()
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert os.path.getsize(tmp_path / "field_w.o") > 0 and time.time() - t0 < 600
