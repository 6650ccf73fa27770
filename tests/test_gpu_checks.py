"""The bounds-checked build (compiled with ST_CHECKS; loaded when ST_CHECKS=1): indices read from device
data are checked before they index an array and a failed check makes the call return ST_ERR_CUDA.  The
parity tests of the flat and two-level traversal, the diffraction sampling, the gathers and the batched
form run on it in a child process and must pass unchanged (no check fires on valid inputs)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_passes_parity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    from paper_2602_19652_gb300 import build
    build.build(checks=True)
    env = dict(os.environ, ST_CHECKS="1")
    probe = subprocess.run([sys.executable, "-c", "import paper_2602_19652_gb300 as st; print(st.load().st_checked_build())"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0 and probe.stdout.strip() == "1", probe.stderr
    tests = ["tests/test_gpu_parity.py::test_clutter_small_full_parity",
             "tests/test_gpu_parity.py::test_vegetation_directivity_parity",
             "tests/test_gpu_instances.py::test_two_level_equals_flat",
             "tests/test_gpu_batch.py::test_batch_equals_single_pose_and_oracle",
             "tests/test_gpu_parity.py::test_stack_restarts_keep_results_exact"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", *tests], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
