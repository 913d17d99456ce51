"""The bounds-checked build (libspcn_checked.so, -DSPCN_CHECKED) over the odd
shapes of the parity tests.

In that build every buffer index and extent the kernels derive (chunk loads
and stores against each image's extent, re-read pixels of queued chunks,
window and histogram bins, density stores, sample and patch positions, float
batch indices) is checked on the device; a failure records
SPCN_ERR_INVALID_ARG in the context's error word, which the next
synchronising call returns, and the access is skipped (no trap).  The cases
run in a child process that loads the checked library and must finish
without any recorded failure, and their outputs must equal, bit for bit,
those of the normal library."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
from paper_1901_03088_b300 import spcn
assert spcn.LIB_PATH.endswith("libspcn_checked.so"), spcn.LIB_PATH
import checked_cases
np.savez(sys.argv[2], **checked_cases.run_cases(spcn, torch))
print("checked cases ok")
"""


def test_checked_build_runs_clean_and_matches(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_03088_b300 import build
    build.build()
    build.build(checked=True)
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, SPCN_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, path], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    from paper_1901_03088_b300 import spcn
    assert spcn.LIB_PATH.endswith("libspcn.so")
    import checked_cases
    want = checked_cases.run_cases(spcn, torch)
    got = np.load(path)
    assert sorted(got.files) == sorted(want)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
