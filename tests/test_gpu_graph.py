"""The one-call path (spcn_normalize_estimated) captured into a CUDA graph.

Without a host statistics record the call puts only kernels and memsets into
the stream, every argument by value, so a graph captured once replays the
whole path: basis estimation (every sampling mode), window, pass 1, recovery
and pass 2.  A replay must give the bytes of a direct call, and after new
pixels are copied into the same source buffer, the bytes of a direct call on
the new pixels (nothing is left from the capture but pointers and
parameters)."""
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


@pytest.mark.parametrize("mode,kw", [("all", {}), ("hash", dict(sample_rate=0.05, seed=3)),
                                     ("patches", dict(n_patches=30, patch_size=64, seed=5))])
def test_captured_one_call_path_replays_like_direct_calls(spcn, mode, kw):
    ctx = spcn.Context(0)
    p = spcn.params(sample_mode=mode, **kw)
    a = synth.make_image(480, 640, 1201, blobs=True)
    b = synth.make_image(480, 640, 1202, blobs=True, W=synth.stain_basis(1300))
    tgt = torch.from_numpy(synth.make_image(256, 256, 1, blobs=True)).cuda()
    t_st = ctx.estimate_basis(tgt, spcn.params(sample_mode="all"))
    t_st.p99[0], t_st.p99[1] = ctx.stain_percentile(tgt, t_st)
    src = torch.from_numpy(a).cuda()
    out = torch.empty_like(src)
    want_a = ctx.normalize_estimated(src, t_st, p).clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.normalize_estimated(src, t_st, p, out=out)   # warm on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.normalize_estimated(src, t_st, p, out=out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    ctx.synchronize()
    assert torch.equal(out, want_a)
    src.copy_(torch.from_numpy(b))
    want_b = ctx.normalize_estimated(src, t_st, p).clone()
    assert not torch.equal(want_a, want_b)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    ctx.synchronize()
    assert torch.equal(out, want_b)
    ctx.close()
