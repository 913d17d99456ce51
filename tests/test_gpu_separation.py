"""Stain separation as a module of its own (§4.3): basis estimation and the
densities of every pixel in one stream-ordered call
(spcn_stain_densities_estimated), bit-identical to spcn_estimate_basis
followed by spcn_stain_densities (whose densities the parity tests check
against the oracle), for every sampling mode and the pseudo-inverse variant;
and its error reporting."""
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


@pytest.fixture(scope="module")
def ctx(spcn):
    c = spcn.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kw", [dict(sample_mode="all"),
                                dict(sample_mode="hash", sample_rate=0.05, seed=3),
                                dict(sample_mode="patches", n_patches=9, patch_size=64, seed=1),
                                dict(sample_mode="all", flags=0x10)])
def test_densities_estimated_matches_two_calls(spcn, ctx, kw):
    img = synth.make_image_torch(600, 733, 1401, device="cuda", blobs=True)
    p = spcn.params(**kw)
    st = ctx.estimate_basis(img, p)
    ref = ctx.stain_densities(img, st, p)
    out, st2 = ctx.stain_densities_estimated(img, p, return_stats=True)
    assert torch.equal(out, ref)
    assert list(st2.W) == list(st.W) and list(st2.i0) == list(st.i0)
    assert st2.p99[0] == st.p99[0] and st2.p99[1] == st.p99[1] and st2.iters == st.iters
    # asynchronous form, pitched output
    buf = torch.full((2, 600 * 733 + 5), -7.0, device="cuda")
    ctx.stain_densities_estimated(img, p, out=buf)
    ctx.synchronize()
    assert torch.equal(buf[:, :600 * 733], ref)
    assert torch.all(buf[:, 600 * 733:] == -7.0)


def test_densities_estimated_reports_no_tissue(spcn, ctx):
    white = torch.full((64, 80, 3), 250, dtype=torch.uint8, device="cuda")
    with pytest.raises(spcn.SpcnError):
        ctx.stain_densities_estimated(white, spcn.params(sample_mode="all"), return_stats=True)
    ctx.stain_densities_estimated(white, spcn.params(sample_mode="all"))
    with pytest.raises(spcn.SpcnError):
        ctx.synchronize()
    # the context stays usable
    img = synth.make_image_torch(64, 80, 1402, device="cuda", blobs=False)
    ctx.stain_densities_estimated(img, spcn.params(sample_mode="all"), return_stats=True)
