"""The GPU parity suites again, on the bounds-checked build of the library.

With -DLBM_BOUNDS_CHECK every population address and auxiliary-field index a
kernel computes is checked against its buffer; one outside it is redirected to
the buffer's first element and reported as LBM_ERR_BOUNDS, which the binding
raises.  Running the oracle-parity suites (every lattice, precision and wall
layout, the batch kernel, graph replay, the allocation-free step, evolved states) on that build
in a child process shows that no step of theirs computes an index outside its
buffer; the suites' own oracle checks hold there too (the checks change no
arithmetic).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_fp16dev.py", "tests/test_gpu_batch.py",
          "tests/test_gpu_evolved.py", "tests/test_gpu_graphs.py", "tests/test_zz_no_alloc.py"]


def test_parity_suites_stay_in_bounds_on_the_checked_build():
    from paper_2201_12404_gb300 import build
    lib = build.build_bounds_checked()
    env = dict(os.environ, LBM_LIBRARY=lib)
    probe = subprocess.run([sys.executable, "-c", "from paper_2201_12404_gb300 import lbm; print(lbm.lbm_version())"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0 and "bounds-checked" in probe.stdout, probe.stdout + probe.stderr
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider", *SUITES],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((res.stdout + res.stderr).splitlines()[-25:])
    assert res.returncode == 0, tail
    assert "LBM_ERR_BOUNDS" not in res.stdout, tail
