"""CPU checks of the C ABI: the library builds, loads, exports every entry
point the header declares, and the ctypes records match the C layouts."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1901_03088_b300 import build as spcn_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spcn.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(spcn_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    spcn_build.build()
    from paper_1901_03088_b300 import spcn
    return spcn


def test_header_declares_the_paper_entry_points():
    d = _declared()
    for name in ("spcn_estimate_basis", "spcn_stain_densities", "spcn_normalize",
                 "spcn_stain_percentile", "spcn_context_create", "spcn_strerror"):
        assert name in d


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", spcn_build.LIB],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (spcn_[a-z0-9_]+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    for s in _declared():
        assert hasattr(lib.lib, s)
    assert set(lib.EXPORTED) >= set(_declared())


def test_record_layouts_match_c(lib, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "spcn.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(spcn_image), sizeof(spcn_params), sizeof(spcn_stats));
  printf("%zu %zu %zu %zu\n", offsetof(spcn_stats, p99), offsetof(spcn_stats, iters),
         offsetof(spcn_stats, n_sample), offsetof(spcn_stats, objective));
  printf("%zu %zu\n", offsetof(spcn_params, seed), offsetof(spcn_params, flags));
  printf("%zu %zu %zu\n", sizeof(spcn_batch_config), offsetof(spcn_batch_config, group_px),
         offsetof(spcn_batch_config, ms));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    S, P, I, B = lib.Stats, lib.Params, lib.Image, lib.BatchConfig
    want = [ctypes.sizeof(I), ctypes.sizeof(P), ctypes.sizeof(S),
            S.p99.offset, S.iters.offset, S.n_sample.offset, S.objective.offset,
            P.seed.offset, P.flags.offset,
            ctypes.sizeof(B), B.group_px.offset, B.ms.offset]
    assert [int(x) for x in got] == want


def test_defaults_are_the_paper_constants(lib):
    p = lib.params()
    assert abs(p.lambda_ - 0.1) < 1e-7 and p.white_thresh == 220
    assert p.i0_pct == 80.0 and p.stain_pct == 99.0 and p.i0_max_samples == 100000


def test_strerror_and_no_device_behaviour(lib):
    assert lib.lib.spcn_strerror(-4) == b"no non-white (tissue) pixel"
    assert lib.lib.spcn_strerror(0) == b"ok"
    # invalid arguments are rejected before any device work
    assert lib.lib.spcn_context_create(None, 0) == -1
    assert lib.lib.spcn_estimate_basis(None, None, None, None, None) == -1
    assert lib.lib.spcn_synchronize(None, None) == -1
    assert lib.lib.spcn_batch_create(None, 0, None, None, None, None, None, None, None) == -1
    assert lib.lib.spcn_batch_run(None, None) == -1
    assert lib.lib.spcn_batch_destroy(None) == 0
