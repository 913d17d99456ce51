"""The no-allocation basis estimation, checked against the context-based one.

spcn_estimate_basis_noalloc is for callers that cannot allocate device memory
(hosts that own the GPU through their own pool, plugin hosts that forbid the
CUDA allocator, pipelines that must not stall on it).  It takes its scratch
from a fixed array inside the library, so it must give the same statistics as
spcn_estimate_basis, call after call, while the array keeps the previous
call's contents.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1901_03088_b300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def spcn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_03088_b300 import build
    build.build()
    from paper_1901_03088_b300 import spcn as s
    return s


def _noalloc_abi(spcn, img, p):
    """Direct C-ABI call of spcn_estimate_basis_noalloc."""
    st = spcn.Stats()
    im = spcn.image_of(img)
    rc = spcn.lib.spcn_estimate_basis_noalloc(ctypes.byref(im), ctypes.byref(p), ctypes.byref(st),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, st


def _same(a, b):
    # the same kernels at the same launch configuration on the same image: the
    # whole statistics record (basis, i0, percentiles, counts, iterations,
    # objective) must be bitwise equal
    assert a.status == 0 and b.status == 0
    assert bytes(a) == bytes(b), (list(a.W), list(b.W), list(a.p99), list(b.p99))


def _cases(spcn):
    return [
        (synth.make_image(512, 512, 1000), spcn.params(sample_mode="all")),
        (synth.make_image(700, 600, 1005, blobs=True),
         spcn.params(sample_mode="hash", sample_rate=0.2, seed=3)),
        (synth.make_image(700, 600, 1005, blobs=True),
         spcn.params(sample_mode="hash", sample_rate=0.2, seed=3, flags=spcn.FLAG_ORDER_BLUE)),
        # patch sampling near the 4096-patch limit with small patches (the
        # candidate buffer and the per-patch percentile storage)
        (synth.make_image(1500, 1400, 1007, blobs=True),
         spcn.params(sample_mode="patches", n_patches=4000, patch_size=8, seed=5)),
        (synth.make_image(1500, 1400, 1007, blobs=True),
         spcn.params(sample_mode="patches", n_patches=4000, patch_size=8, seed=5,
                     flags=spcn.FLAG_P99_PATCH_MEDIAN)),
    ]


def test_noalloc_matches_context_path_on_two_calls_in_a_row(spcn):
    ctx = spcn.Context(0)
    for img_np, p in _cases(spcn):
        img = torch.from_numpy(img_np).cuda()
        want = ctx.estimate_basis(img, p)
        for _ in range(2):   # the array keeps the previous call's contents
            rc, got = _noalloc_abi(spcn, img, p)
            assert rc == 0, spcn.lib.spcn_strerror(rc)
            _same(got, want)
    ctx.close()


def test_noalloc_rejects_a_sample_beyond_its_scratch(spcn):
    img = torch.from_numpy(synth.make_image(1024, 1024, 1)).cuda()
    rc, _ = _noalloc_abi(spcn, img, spcn.params(sample_mode="all"))     # 1 Mpx > 524288
    assert rc == -7
    assert b"fixed scratch" in spcn.lib.spcn_strerror(rc)
    rc, _ = _noalloc_abi(spcn, img, spcn.params(sample_mode="patches", n_patches=5000,
                                                 patch_size=4))
    assert rc == -7
