"""CPU checks that the C ABI rejects invalid requests before any device work.

Every case below must be refused by the host-side argument checks, so the
entry points are called with a dummy context handle that is never used.  They
run in a child process: if a check were missing, the library would use the
dummy handle and the child would die, which the test reports as a failure
instead of taking the test run down with it."""
import json
import os
import subprocess
import sys

import pytest

from paper_1901_03088_b300 import build as spcn_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
from paper_1901_03088_b300 import spcn
lib = spcn._lib
CTX = ctypes.c_void_p(0x1000)      # never dereferenced by a rejected call
DATA = ctypes.c_void_p(0x2000)     # likewise
out = {}

def image(w, h, pitch=None):
    return spcn.Image(DATA, w, h, 3 * w if pitch is None else pitch)

def stats(W=((0.65, 0.07), (0.70, 0.99), (0.29, 0.11)), i0=(255.0, 255.0, 255.0)):
    return spcn.Stats.from_values(W, i0)

def pct(key, img, st=None, p=None):
    p99 = (ctypes.c_double * 2)()
    st = st or stats()
    p = p or spcn.params()
    out[key] = lib.spcn_stain_percentile(CTX, ctypes.byref(img), ctypes.byref(st),
                                         ctypes.byref(p), p99, None)
    print(key, out[key], file=sys.stderr, flush=True)

pct("negative_basis_entry", image(64, 64), stats(W=((0.65, 0.07), (-0.01, 0.99), (0.29, 0.11))))
pct("i0_zero", image(64, 64), stats(i0=(0.0, 255.0, 255.0)))
pct("i0_above_255", image(64, 64), stats(i0=(255.0, 256.0, 255.0)))
pct("parallel_columns", image(64, 64), stats(W=((0.6, 0.6), (0.7, 0.7), (0.3, 0.3))))
pct("too_many_pixels", image(1 << 20, 1 << 16))
pct("chunk_index_overflow", image(33, 1431655766))
pct("pitch_below_row", image(64, 64, pitch=3 * 64 - 1))
pct("white_thresh_256", image(64, 64), p=spcn.params(white_thresh=256))
pct("unknown_flag", image(64, 64), p=spcn.params(flags=0x100))
pct("patch_median_without_patches", image(64, 64),
    p=spcn.params(sample_mode="all", flags=spcn.FLAG_P99_PATCH_MEDIAN))
pct("patch_median_too_many_patches", image(64, 64),
    p=spcn.params(sample_mode="patches", n_patches=4097, patch_size=8,
                  flags=spcn.FLAG_P99_PATCH_MEDIAN))

st = stats()
out["normalize_out_pitch"] = lib.spcn_normalize(
    CTX, ctypes.byref(image(64, 64)), ctypes.byref(st), ctypes.byref(st),
    ctypes.byref(spcn.params()), DATA, 3 * 64 - 1, None, None)

st_out = spcn.Stats()
out["noalloc_sample_beyond_scratch"] = lib.spcn_estimate_basis_noalloc(
    ctypes.byref(image(1024, 1024)), ctypes.byref(spcn.params(sample_mode="all")),
    ctypes.byref(st_out), None)
# the rate is validated before the sample size is derived from it
for key, rate in (("noalloc_nan_rate", float("nan")), ("noalloc_negative_rate", -0.5)):
    p = spcn.params(sample_mode="hash")
    p.sample_rate = rate
    out[key] = lib.spcn_estimate_basis_noalloc(ctypes.byref(image(1024, 1024)), ctypes.byref(p),
                                               ctypes.byref(st_out), None)
out["noalloc_null_image"] = lib.spcn_estimate_basis_noalloc(
    None, ctypes.byref(spcn.params()), ctypes.byref(st_out), None)
print(json.dumps(out))
"""

INVALID, DEGENERATE, SCRATCH = -1, -5, -7
EXPECTED = {
    "negative_basis_entry": INVALID,
    "i0_zero": INVALID,
    "i0_above_255": INVALID,
    "parallel_columns": DEGENERATE,
    "too_many_pixels": INVALID,          # 2^36 pixels
    "chunk_index_overflow": INVALID,     # 3 * 1431655766 >= 2^32 chunks, below 2^36 pixels
    "pitch_below_row": INVALID,
    "white_thresh_256": INVALID,
    "unknown_flag": INVALID,
    "patch_median_without_patches": INVALID,
    "patch_median_too_many_patches": INVALID,
    "normalize_out_pitch": INVALID,
    "noalloc_sample_beyond_scratch": SCRATCH,   # 1 Mpx sample, above 524,288
    "noalloc_nan_rate": INVALID,
    "noalloc_negative_rate": INVALID,
    "noalloc_null_image": INVALID,
}


@pytest.fixture(scope="module")
def results():
    spcn_build.build()
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       timeout=300)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert r.returncode == 0 and lines, (
        f"the child died (rc {r.returncode}); last calls:\n{r.stderr[-2000:]}")
    return json.loads(lines[-1])


@pytest.mark.parametrize("case", sorted(EXPECTED))
def test_rejected_before_device_work(results, case):
    assert results[case] == EXPECTED[case], (case, results[case])
