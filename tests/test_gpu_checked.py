"""The GPU parity suite once more on the bounds-checked build (libsdg_checked.so, compiled with -DSDG_CHECKED):
every block index, trilinear-corner voxel address, dense-grid cell and ray row the render, traversal and query
kernels derive is checked before use, the first one out of range recorded in a device status word (no trap, the
access skipped).  The suite runs in a child process with SDG_LIBRARY pointing at that build; conftest asserts
after every GPU test that the status word is still 0, so the parity assertions and the bounds checks pass
together."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.path.join(ROOT, "paper_2305_13220_b300", "libsdg_checked.so")


def test_parity_suite_under_bounds_checks():
    assert os.path.exists(CHECKED), "libsdg_checked.so is not built (python paper_2305_13220_b300/build.py --checked)"
    env = dict(os.environ, SDG_LIBRARY="libsdg_checked.so", SDG_EXPECT_CHECKED="1")
    files = ["tests/test_gpu_render.py", "tests/test_gpu_fullsize.py", "tests/test_gpu_serve.py",
             "tests/test_gpu_normal.py", "tests/test_gpu_beta_ssi.py", "tests/test_gpu_query.py",
             "tests/test_gpu_ray_order.py", "tests/test_gpu_adam.py", "tests/test_gpu_activation.py",
             "tests/test_gpu_overflow.py", "tests/test_gpu_prepare.py", "tests/test_gpu_sem_table.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", *files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((r.stdout + r.stderr).strip().splitlines()[-15:])
    assert r.returncode == 0, tail
    print(tail.splitlines()[-1])
