"""The window-miss recovery of the exact whole-image percentile (Eq. 3's P99
over the non-white pixels, §3.1 item 2), through the C ABI.

Pass 1 counts the pixels below a window of keys around a hint and histograms
the keys inside it.  When a rank falls outside, counting passes over ladders
of key ranges locate it and an exact histogram of a narrow span selects it;
ranks that stay far apart are left to the radix select.  Whatever the route,
the percentile must equal, bit for bit, the type-7 percentile of the library's
own FP32 densities over the non-white pixels, and each launch that had a rank
to find is counted once."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import spcn_oracle as O  # noqa: E402
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


def type7_of_f32(values, p):
    a = np.sort(values.astype(np.float32)).astype(np.float64)
    pos = (a.size - 1) * (p / 100.0)
    k = int(math.floor(pos))
    if k + 1 >= a.size:
        return float(a[-1])
    return float(a[k]) + (pos - k) * (float(a[k + 1]) - float(a[k]))


def check(spcn, ctx, img, st, p=None, pct=99.0):
    dev = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    before = ctx.exact_fallbacks
    got = ctx.stain_percentile(dev, st, p) if p is not None else ctx.stain_percentile(dev, st)
    misses = ctx.exact_fallbacks - before
    H = ctx.stain_densities(dev, st).cpu().numpy()
    thr = p.white_thresh if p is not None else 220
    nw = O.nonwhite_mask(img.reshape(-1, 3), thr)
    level = float(np.float32(pct))   # spcn_params.stain_pct is an FP32 level
    for j in range(2):
        assert got[j] == type7_of_f32(H[j][nw], level), (j, got[j])
    return misses


def stats_with_hint(spcn, img, factor):
    o = O.full_stats(img)
    st = spcn.Stats.from_values(np.float32(o.W), np.float32(o.i0), o.p99)
    st.p99[0], st.p99[1] = o.p99[0] * factor, o.p99[1] * factor
    return st


@pytest.mark.parametrize("factor", [1.0, 0.97, 1.03, 0.8, 1.25, 0.5, 2.0, 0.1, 10.0, 1e-3, 300.0])
def test_percentile_after_a_miss_on_either_side(spcn, ctx, factor):
    img = synth.make_image(700, 901, 1101, blobs=True)
    misses = check(spcn, ctx, img, stats_with_hint(spcn, img, factor))
    if factor == 1.0:
        assert misses == 0
    if factor in (0.5, 2.0, 0.1, 10.0, 1e-3, 300.0):
        assert misses == 1


def test_percentile_with_no_hint(spcn, ctx):
    img = synth.make_image(513, 1029, 1102, blobs=True)
    assert check(spcn, ctx, img, stats_with_hint(spcn, img, 0.0)) == 1


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (37, 1), (3, 17)])
def test_tiny_images(spcn, ctx, shape):
    img = synth.make_image(*shape, 1103 + shape[1])
    img[0, 0] = (90, 60, 120)   # at least one non-white pixel
    W = synth.stain_basis(5)
    st = spcn.Stats.from_values(np.float32(W), [250.0, 250.0, 250.0], [7.0, 7.0])
    check(spcn, ctx, img, st)


def test_ranks_on_either_side_of_a_gap(spcn, ctx):
    # two tissue colours: exactly k+1 light pixels, then dark ones, so ranks k
    # and k+1 of each stain sit far apart with no pixel in between
    n = 10000
    k = int(math.floor(0.99 * (n - 1)))
    light, dark = (200, 170, 210), (60, 20, 90)
    px = np.array([light] * (k + 1) + [dark] * (n - k - 1) + [(255, 255, 255)] * 2400,
                  dtype=np.uint8)
    px = px[np.random.default_rng(1).permutation(px.shape[0])]
    img = px.reshape(100, 124, 3)
    W = synth.stain_basis(6)
    st = spcn.Stats.from_values(np.float32(W), [250.0, 250.0, 250.0], [0.0, 0.0])
    assert check(spcn, ctx, img, st) == 1


def test_other_levels_and_thresholds(spcn, ctx):
    img = synth.make_image(400, 600, 1104, blobs=True)
    for pct, thr in ((50.0, 220), (1.0, 220), (99.9, 128), (99.0, 255)):
        p = spcn.params(stain_pct=pct, white_thresh=thr)
        o = O.full_stats(img, O.Params(stain_pct=pct, white_thresh=thr))
        st = spcn.Stats.from_values(np.float32(o.W), np.float32(o.i0), (o.p99[0] * 3, o.p99[1] * 3))
        check(spcn, ctx, img, st, p, pct)
