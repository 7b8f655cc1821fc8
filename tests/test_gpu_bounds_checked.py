"""The bounds-checking build (libzoomy_debug.so, build(debug=True)): every gather index of the stage,
lifting and VAM kernels -- structured rows and columns, the second-order stencil of radius 2,
triangle neighbours, ensemble member offsets, the closure's predictions, the VAM cells and the
block rows of its cyclic reduction -- is checked before its access; an index outside its buffer
would redirect the access to element 0 and make the call return ZOOMY_EBOUNDS.  This test runs the
GPU parity cases of those paths (the small ones; the full-size and long-run cases are left out)
against that library in a separate process.  It skips unless the library was built."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEBUG_LIB = os.path.join(ROOT, "paper_2601_04826_gb300", "libzoomy_debug.so")
FILES = ["tests/test_gpu_struct.py", "tests/test_gpu_tri.py", "tests/test_gpu_order2.py", "tests/test_gpu_ensemble.py",
         "tests/test_gpu_vam.py", "tests/test_gpu_lift.py", "tests/test_gpu_closure.py", "tests/test_gpu_source.py"]


def test_parity_cases_under_bounds_checks():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(DEBUG_LIB):
        pytest.skip("libzoomy_debug.so not built (paper_2601_04826_gb300.build.build(debug=True))")
    env = dict(os.environ, ZOOMY_LIBRARY=DEBUG_LIB)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        "-k", "not full_size and not long_line", *FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    tail = r.stdout[-3000:]
    print(tail)
    assert r.returncode == 0, tail
    assert " passed" in tail and "EBOUNDS" not in r.stdout
