"""The bounds-checked build (-DGP_CHECK) on odd and ragged grids.

In libgp_sscn_check.so every global access of the sweep kernels is guarded: an index
outside its buffer records a status bit and the access is skipped (nothing traps), and
the next synchronising call returns GP_ERR_BOUNDS.  This test runs steps, observables
and densities on grids that exercise ragged tiles, chunks and segments (FP64 and FP32,
imaginary and real time, every kernel family) through the checked library in a child
process, requires that no check fired, and that the results are bit for bit those of
the normal library (the checks add branches, not arithmetic).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [((3, 3, 3), "f64"), ((5, 7, 9), "f64"), ((17, 33, 19), "f64"), ((70, 9, 37), "f64"),
         ((33, 65, 5), "f64"), ((40, 36, 1), "f64"), ((37, 29, 23), "f32"), ((240, 40, 32), "f32"),
         ((64, 48, 32), "f32"), ((300, 40, 30), "f32"), ((3, 70, 41), "f32"), ((48, 40, 1), "f32")]

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_1605_03958_gb300 as P
cases = json.loads(sys.argv[2])
out = {}
for k, (shape, prec) in enumerate(cases):
    nx, ny, nz = shape
    s = P.Solver(nx, ny, nz, 0.3, 0.25, 0.4, 0.01, 1.1, 1.7, 0.6, g=12.0, prec=prec)
    s.init_gaussian()
    s.step_imag(7)
    a = s.get_psi()
    o = s.observables()
    d = [s.density1d(ax) for ax in range(3 if nz > 1 else 2)]
    s.step_real(5)
    b = s.get_psi(as_complex=True)
    s.sync()
    out[str(k)] = {"imag": a.tolist(), "real_re": b.real.tolist(), "real_im": b.imag.tolist(),
                   "obs": o, "dens": [x.tolist() for x in d]}
    s.close()
json.dump(out, open(sys.argv[3], "w"))
"""


@pytest.fixture(scope="module")
def libs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1605_03958_gb300 import build
    return build.LIB, build.build(check=True)


def run(lib, path):
    env = dict(os.environ, GP_SSCN_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(CASES), path],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    with open(path) as f:
        return json.load(f)


def test_checked_build_fires_nothing_and_matches(libs, tmp_path):
    normal, checked = libs
    a = run(checked, str(tmp_path / "checked.json"))   # a GP_ERR_BOUNDS would fail the child
    b = run(normal, str(tmp_path / "normal.json"))
    for k in a:
        for key in ("imag", "real_re", "real_im"):
            assert np.array_equal(np.array(a[k][key]), np.array(b[k][key])), (CASES[int(k)], key)
        assert a[k]["obs"] == b[k]["obs"], CASES[int(k)]
        for x, y in zip(a[k]["dens"], b[k]["dens"]):
            assert np.array_equal(np.array(x), np.array(y)), CASES[int(k)]
