"""The bounds-checking build (libdg_gb300_debug.so, DG_DEBUG_BOUNDS) runs the
ordinary parity suites without a false flag.

In that build every index a kernel gathers through the mesh tables is
checked against its range; an out-of-range index sets a device flag, which
dg_check_status reports as DG_ERR_DEVICE_BOUNDS, and is replaced by 0.  The
suites below (structured, curved, rotated-element, partitioned, boundary,
wall-modelled and adjoint cases) call dg_check_status after their
evaluations, so a flag raised by a valid mesh fails them.  They run in a
child process with DG_LIBRARY_VARIANT=debug, which makes the binding load the
checking build.  No invalid index is fed to the GPU."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_orientation.py", "tests/test_gpu_partition.py",
          "tests/test_gpu_boundaries.py", "tests/test_gpu_mixed.py", "tests/test_gpu_errors.py"]


def test_parity_suites_under_the_bounds_checking_build():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, DG_LIBRARY_VARIANT="debug")
    probe = ("from paper_2606_18927_gb300 import dg; print(dg.lib()._name)")
    r = subprocess.run([sys.executable, "-c", probe], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    assert "libdg_gb300_debug.so" in r.stdout
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + SUITES + \
          ["tests/test_gpu_adjoint.py", "-k", "not full_transpose_at_n7"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    print(r.stdout[-3000:])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
