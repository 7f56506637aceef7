"""The bounds-checked debug build (-DMMP_CHECK_BOUNDS, loaded with
MMP_CHECK_BOUNDS=1) on the GPU: every kernel index check armed, the odd
shapes, the warp engines and a multi-region grid with empty cells run one
field evaluation (checked against the oracle) and three adaptive steps
without any check failing (a failed one makes the call return
MMP_E_BOUNDS, which raises in the child process)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, "tests")
import numpy as np
from inputs import config_small
from gpu_util import field_tolerance, torque_tolerance, make_magnet, gpu_eval, oracle_eval
import paper_2411_18194_gb300 as pkg
assert pkg.library_path().endswith("libmmp_checked.so"), pkg.library_path()
FM = ("DEMAG", "EXCH", "ANIS", "DMI", "ZEEMAN")
CASES = [((3, 5, 1), 1, 0.0), ((6, 3, 2), 1, 0.0), ((1, 7, 1), 1, 0.0), ((24, 20, 2), 3, 0.1),
         ((1000, 6, 2), 1, 0.0), ((3, 1000, 8), 1, 0.0)]
out = []
for i, (shape, nreg, empty) in enumerate(CASES):
    w = config_small(shape, (2e-9, 2e-9, 1e-9), 90 + i, terms=FM, n_regions=nreg, empty_fraction=empty)
    p = w.problem
    mag = make_magnet(p, w.m0)
    Bg, Tg = gpu_eval(mag, p)
    Bo, To = oracle_eval(p, w.m0)
    tolB = field_tolerance(p, Bo[0])
    ok = bool(np.all(np.abs(Bg[0] - Bo[0]) <= tolB))
    ok = ok and bool(np.all(np.abs(Tg[0] - To[0]) <= torque_tolerance(p, Bo[0], tolB)))
    mag.set_solver(adaptive=True, dt=1e-14)
    mag.step(3)
    mag.close()
    out.append([list(shape), ok])
print(json.dumps(out))
'''


def test_checked_build_runs_without_a_bounds_error():
    from paper_2411_18194_gb300 import build
    if not os.path.exists(build.CHECKED_LIB):
        build.build(checked=True)
    env = dict(os.environ, MMP_CHECK_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(res) == 6 and all(ok for _, ok in res), res
