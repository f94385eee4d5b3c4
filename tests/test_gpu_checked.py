"""The checked build (-DEMRI_FD_CHECKS=1, build.build(checked=True)).  Its hot kernels
test the run, mode, segment and bin indices they derive from the device-built run
lists, and a failed test latches EMRI_FD_ERR_INTERNAL instead of an out-of-bounds
access.  A child process that loads the checked library (EMRI_FD_LIBRARY) makes a set
of representative calls: none reports a failed check (every call returns
EMRI_FD_OK), and every result equals the normal build's bitwise (the checks change no
arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_12585_gb300 import build
    build.build()


def test_checked_build_reports_no_failed_check_and_equals_the_normal_build(tmp_path):
    from paper_2307_12585_gb300 import build
    from tests import checked_cases
    lib = build.build(checked=True)
    out = tmp_path / "checked.npz"
    env = dict(os.environ, EMRI_FD_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases", str(out)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    chk = np.load(out)
    assert str(chk["library"]).endswith("libemri_fd_checked.so")
    ref = checked_cases.run_cases()
    for k, v in ref.items():
        assert np.array_equal(chk[k], v), k
