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
    # the tolerances of the parity tests: W within 1e-5, i0 exact in FP32,
    # sampled percentile within 1e-4 relative, counts exact
    assert a.status == 0 and b.status == 0
    assert np.max(np.abs(np.array(a.W[:]) - np.array(b.W[:]))) <= 1e-5
    assert list(a.i0) == list(b.i0)
    for j in range(2):
        assert abs(a.p99[j] - b.p99[j]) <= 1e-4 * abs(b.p99[j])
    assert (a.n_sample, a.n_nonwhite, a.n_bright) == (b.n_sample, b.n_nonwhite, b.n_bright)


def test_noalloc_matches_context_path_on_two_calls_in_a_row(spcn):
    cases = [
        (synth.make_image(512, 512, 1000), spcn.params(sample_mode="all")),
        (synth.make_image(700, 600, 1005, blobs=True),
         spcn.params(sample_mode="hash", sample_rate=0.2, seed=3)),
    ]
    ctx = spcn.Context(0)
    for img_np, p in cases:
        img = torch.from_numpy(img_np).cuda()
        want = ctx.estimate_basis(img, p)
        rc, got = _noalloc_abi(spcn, img, p)
        assert rc == 0, spcn.lib.spcn_strerror(rc)
        _same(got, want)
    # the second case again right after: the array still holds its contents
    rc, again = _noalloc_abi(spcn, img, p)
    assert rc == 0
    _same(again, want)
    ctx.close()


def test_noalloc_rejects_a_sample_beyond_its_scratch(spcn):
    img = torch.from_numpy(synth.make_image(1024, 1024, 1)).cuda()
    rc, _ = _noalloc_abi(spcn, img, spcn.params(sample_mode="all"))     # 1 Mpx > 524288
    assert rc == -7
    assert b"fixed scratch" in spcn.lib.spcn_strerror(rc)
    rc, _ = _noalloc_abi(spcn, img, spcn.params(sample_mode="patches", n_patches=5000,
                                                 patch_size=4))
    assert rc == -7
