"""Pass 1 (the windowed P99 count) on images with large white regions.

Pass 1 drops full chunks whose every byte passes a conservative all-white
test and hands the remaining chunks to full warps through a per-warp stack;
a row's last, partial chunk is counted pixel by pixel.  These tests run it on
a 3000 x 4099 image (several loop iterations per warp, a 3-pixel chunk at the
end of every row) with white rectangles of uneven widths painted over it, at
several white thresholds including 255 (no pixel is white), and require the
percentile to equal, bit for bit, the type-7 percentile (§3.2 item 4) of the
GPU's own FP32 densities over the non-white pixels of that threshold
(§3.1 item 2: a pixel is white when every channel is above the threshold).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1901_03088_b300 import synth  # noqa: E402

H, W_PX = 3000, 4099


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


@pytest.fixture(scope="module")
def image():
    dev = torch.device("cuda", 0)
    img = synth.make_image_torch(H, W_PX, 4242, device=dev, blobs=True)
    g = torch.Generator(device="cpu")
    g.manual_seed(7)
    # white rectangles (bytes 236..255) of widths from 5 to 900 pixels
    for _ in range(60):
        h = int(torch.randint(20, 600, (1,), generator=g))
        w = int(torch.randint(5, 900, (1,), generator=g))
        y = int(torch.randint(0, H - h, (1,), generator=g))
        x = int(torch.randint(0, W_PX - w, (1,), generator=g))
        val = torch.randint(236, 256, (h, w, 3), generator=g, dtype=torch.int32)
        img[y:y + h, x:x + w] = val.to(torch.uint8).to(dev)
    return img


def type7(values, p):
    a = torch.sort(values.float())[0].double()
    n = a.numel()
    pos = (n - 1) * (p / 100.0)
    k = int(math.floor(pos))
    t = pos - k
    if k + 1 >= n:
        return float(a[n - 1])
    lo, hi = float(a[k]), float(a[k + 1])
    return lo + t * (hi - lo)


@pytest.mark.parametrize("thresh", [220, 128, 100, 254, 255])
@pytest.mark.parametrize("hint", ["exact", "none"])
def test_percentile_with_white_regions(spcn, ctx, image, thresh, hint):
    st = spcn.Stats.from_values(synth.stain_basis(4242), [255.0, 255.0, 255.0])
    Hd = ctx.stain_densities(image, st)                         # (2, H*W) FP32
    nw = (image.reshape(-1, 3).amin(dim=1) <= thresh)
    assert 0.05 < nw.float().mean().item() <= 1.0
    ref = [type7(Hd[j][nw], 99.0) for j in range(2)]
    if hint == "exact":
        st.p99[0], st.p99[1] = ref
    p = spcn.params(white_thresh=thresh)
    got = ctx.stain_percentile(image, st, p)
    assert got[0] == ref[0] and got[1] == ref[1]


def test_white_chunks_are_a_real_share(image):
    """The image exercises the skip: many full chunks are entirely white."""
    full = (W_PX // 16) * 16
    px = image[:, :full].reshape(H, -1, 16, 3)
    white_chunk = (px.amin(dim=(2, 3)) > 220)
    frac = white_chunk.float().mean().item()
    assert 0.2 < frac < 0.8


def faint_colour_image(h, w, seed, dev):
    """Half light-gray pixels (channels 140-255), half faintly red ones
    (R 100-128, G and B 200-255), drawn independently per pixel."""
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    gray = torch.randint(140, 256, (h, w, 3), generator=g)
    red = torch.stack([torch.randint(100, 129, (h, w), generator=g),
                       torch.randint(200, 256, (h, w), generator=g),
                       torch.randint(200, 256, (h, w), generator=g)], dim=-1)
    pick = torch.rand((h, w), generator=g) < 0.5
    return torch.where(pick.unsqueeze(-1), gray, red).to(torch.uint8).to(dev)


def test_percentile_when_white_pixels_reach_the_window(spcn, ctx):
    """Pass 1 may count a tissue chunk without testing each pixel for white
    only when every white pixel provably lies below both window starts.  Here
    the first stain points along the gray direction, so at threshold 128 the
    light-gray (white) pixels get larger densities than the 99th percentile of
    the faintly coloured non-white ones: the per-pixel masks are needed, and
    the window (an exact hint) holds the ranks.  The image is 1037 wide, so
    every row ends with a partial chunk."""
    dev = torch.device("cuda", 0)
    img = faint_colour_image(1024, 1037, 11, dev)
    W = np.array([[1.0, 0.1], [1.0, 0.7], [1.0, 0.7]])
    W = W / np.linalg.norm(W, axis=0)
    st = spcn.Stats.from_values(W, [255.0, 255.0, 255.0])
    thresh = 128
    Hd = ctx.stain_densities(img, st)
    nw = (img.reshape(-1, 3).amin(dim=1) <= thresh)
    assert 0.3 < nw.float().mean().item() < 0.7
    ref = [type7(Hd[j][nw], 99.0) for j in range(2)]
    # the premise: white pixels reach above the first stain's percentile
    assert Hd[0][~nw].max().item() > ref[0]
    st.p99[0], st.p99[1] = ref
    got = ctx.stain_percentile(img, st, spcn.params(white_thresh=thresh))
    assert got[0] == ref[0] and got[1] == ref[1]
