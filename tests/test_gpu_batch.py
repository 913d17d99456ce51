"""Batched normalisation (one persistent launch over many uneven tiles with
per-slide statistics) against the single-image path.

The batch computes, per tile, exactly what spcn_normalize computes for that
tile alone (same tables, densities, keys and reconstruction), so the bar is
bit-identical output bytes and percentiles, under every schedule, with good,
missing and misleading window hints, for contiguous and pitched tiles, and in
CUDA-graph replays.  Two tiles are also checked against the FP64 oracle at
the single-image tolerances (uint8 within 1 on >= 99.99% of pixels).
"""
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


@pytest.fixture(scope="module")
def setup(spcn, ctx):
    """4 slides x 6 tiles, sides log-uniform in [40, 600] (plus ragged widths),
    per-slide statistics estimated on a 384^2 sample of each slide."""
    layout = synth.batch_layout(4, 6, 40, 600, seed=7)
    layout[0] = (0, 1, 37)          # one-row tile, width not a multiple of 16
    layout[1] = (0, 33, 1)          # one-column tile
    tiles, slide_stats = [], []
    p = spcn.params(sample_mode="all")
    for s in range(4):
        W = synth.stain_basis(2000 + s)
        sample = synth.make_image_torch(384, 384, 2100 + s, W=W, device="cuda")
        slide_stats.append(ctx.estimate_basis(sample, p))
    for k, (s, h, w) in enumerate(layout):
        tiles.append(synth.make_image_torch(h, w, 3000 + k, W=synth.stain_basis(2000 + s),
                                            device="cuda", blobs=False))
    stats = [slide_stats[s] for (s, _, _) in layout]
    tgt = ctx.estimate_basis(synth.make_image_torch(256, 256, 1, device="cuda"), p)
    return tiles, stats, tgt, spcn.params()


def sequential(ctx, tiles, stats, tgt, p):
    outs, p99 = [], []
    for t, st in zip(tiles, stats):
        o, q = ctx.normalize(t, st, tgt, p, return_p99=True)
        outs.append(o)
        p99.append(q)
    return outs, p99


# the fused persistent launch, the staged launches and the staged steps as
# phases of one persistent launch, at the default item size
SCHEDS = ["phased", "staged", "persistent"]


def run_batch(spcn, ctx, tiles, stats, tgt, outs, p, sched):
    """Create a batch under schedule `sched`, run it once; (p99, status, fallback)."""
    b = spcn.Batch(ctx, tiles, stats, tgt, outs, p)
    b.set_config(16 * 1024, sched)
    b.run()
    res = b.results(fallback=True)
    b.close()
    return res


def assert_same(outs, ref_outs, p99, ref_p99):
    for i, (a, b) in enumerate(zip(outs, ref_outs)):
        assert torch.equal(a, b), f"tile {i}: {(a != b).sum().item()} bytes differ"
    for i, (a, b) in enumerate(zip(p99, ref_p99)):
        assert a[0] == b[0] and a[1] == b[1], (i, a, b)


def test_batch_equals_sequential_calls(spcn, ctx, setup):
    tiles, stats, tgt, p = setup
    ref_outs, ref_p99 = sequential(ctx, tiles, stats, tgt, p)
    outs = [torch.empty_like(t) for t in tiles]
    p99, status = spcn.normalize_batched(ctx, tiles, stats, tgt, outs, p)
    assert status == [0] * len(tiles)
    assert_same(outs, ref_outs, p99, ref_p99)
    for sched in SCHEDS:
        outs = [torch.empty_like(t) for t in tiles]
        p99, status, _ = run_batch(spcn, ctx, tiles, stats, tgt, outs, p, sched)
        assert status == [0] * len(tiles)
        assert_same(outs, ref_outs, p99, ref_p99)


@pytest.mark.parametrize("sched", SCHEDS)
def test_batch_pitched_tiles(spcn, ctx, setup, sched):
    # tiles as views into wider buffers at odd byte offsets (generic traversal)
    tiles, stats, tgt, p = setup
    views, outs = [], []
    for t in tiles:
        h, w, _ = t.shape
        buf = torch.zeros((h, 3 * w + 29), dtype=torch.uint8, device="cuda")
        v = torch.as_strided(buf, (h, w, 3), (buf.shape[1], 3, 1), storage_offset=7)
        v.copy_(t)
        views.append(v)
        ob = torch.zeros((h, 3 * w + 19), dtype=torch.uint8, device="cuda")
        outs.append(torch.as_strided(ob, (h, w, 3), (ob.shape[1], 3, 1), storage_offset=3))
    ref_outs, ref_p99 = sequential(ctx, tiles, stats, tgt, p)
    p99, status, _ = run_batch(spcn, ctx, views, stats, tgt, outs, p, sched)
    assert_same(outs, ref_outs, p99, ref_p99)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("hint", ["none", "far_low", "far_high", "exact"])
def test_batch_window_hints(spcn, ctx, setup, hint, sched):
    # no hint or a misleading one sends tiles to the exact fallback; results stay identical
    tiles, stats, tgt, p = setup
    ref_outs, ref_p99 = sequential(ctx, tiles, stats, tgt, p)
    hs = []
    for st, q in zip(stats, ref_p99):
        s = st.copy()
        f = {"none": 0.0, "far_low": 0.2, "far_high": 5.0, "exact": 1.0}[hint]
        base = q if hint == "exact" else (s.p99[0], s.p99[1])
        s.p99[0], s.p99[1] = base[0] * f, base[1] * f
        hs.append(s)
    outs = [torch.empty_like(t) for t in tiles]
    p99, _, fallback = run_batch(spcn, ctx, tiles, hs, tgt, outs, p, sched)
    assert_same(outs, ref_outs, p99, ref_p99)
    # no hint: no window, every tile takes the exact fallback.  With a hint,
    # a tile whose pilot sample holds enough tissue chunks starts its window
    # at the pilot's low quantile whatever the hint, so tiles of 4096 pixels
    # or more never fall back; smaller tiles start at 0.75 x hint, and fall
    # back when that lies above their percentile (far_high)
    big = [f for f, t in zip(fallback, tiles) if t.shape[0] * t.shape[1] >= 4096]
    if hint == "none":
        assert all(fallback), fallback
    else:
        assert not any(big), fallback


@pytest.mark.parametrize("item_chunks,schedule,group_px", [
    (1024, "phased", 0), (8192, "phased", 0), (1024, "interleaved", 200_000),
    (2048, "interleaved", 1), (1024, "staged", 0), (8192, "staged", 0),
    (1024, "persistent", 0)])
def test_batch_schedules_and_graph_replay(spcn, ctx, setup, item_chunks, schedule, group_px):
    tiles, stats, tgt, p = setup
    ref_outs, ref_p99 = sequential(ctx, tiles, stats, tgt, p)
    outs = [torch.zeros_like(t) for t in tiles]
    b = spcn.Batch(ctx, tiles, stats, tgt, outs, p)
    b.set_config(item_chunks, schedule, group_px)
    assert b.config["item_chunks"] == item_chunks and b.config["schedule"] == schedule
    b.run()
    p99, status = b.results()
    assert_same(outs, ref_outs, p99, ref_p99)
    # capture one run into a CUDA graph and replay it on fresh outputs
    for o in outs:
        o.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    p99, status = b.results()
    assert_same(outs, ref_outs, p99, ref_p99)
    b.close()


def test_batch_tuner(spcn, ctx, setup):
    tiles, stats, tgt, p = setup
    ref_outs, ref_p99 = sequential(ctx, tiles, stats, tgt, p)
    outs = [torch.zeros_like(t) for t in tiles]
    b = spcn.Batch(ctx, tiles, stats, tgt, outs, p)
    trials = b.tune(reps=1)
    assert len(trials) >= 4 and all(t["ms"] > 0 for t in trials)
    best = min(trials, key=lambda t: t["ms"])
    cfg = b.config
    assert (cfg["item_chunks"], cfg["schedule"]) == (best["item_chunks"], best["schedule"])
    b.run()
    p99, _ = b.results()
    assert_same(outs, ref_outs, p99, ref_p99)
    b.close()


@pytest.mark.parametrize("sched", SCHEDS)
def test_batch_no_tissue_and_list_overflow(spcn, ctx, setup, sched):
    tiles, stats, tgt, p = setup
    white = torch.full((50, 70, 3), 255, dtype=torch.uint8, device="cuda")
    flat = torch.empty((90, 130, 3), dtype=torch.uint8, device="cuda")
    flat[...] = torch.tensor([120, 80, 160], dtype=torch.uint8)
    # hint = the flat tile's own percentile: every pixel lands in the window,
    # more keys than the list holds, so the tile takes the exact fallback
    q = ctx.stain_percentile(flat, stats[0], p)
    st_flat = stats[0].copy()
    st_flat.p99[0], st_flat.p99[1] = q
    btiles = [tiles[5], white, flat, tiles[9]]
    bstats = [stats[5], stats[0], st_flat, stats[9]]
    outs = [torch.empty_like(t) for t in btiles]
    p99, status, _ = run_batch(spcn, ctx, btiles, bstats, tgt, outs, p, sched)
    assert status == [0, -4, 0, 0]
    ref_w = ctx.normalize(white, stats[0], tgt, p)
    with pytest.raises(spcn.SpcnError) as e:
        ctx.synchronize()
    assert e.value.kind == "NO_TISSUE"
    assert torch.equal(outs[1], ref_w) and p99[1] == (0.0, 0.0)
    for i in (0, 2, 3):
        ref, rq = ctx.normalize(btiles[i], bstats[i], tgt, p, return_p99=True)
        assert torch.equal(outs[i], ref) and tuple(p99[i]) == tuple(rq)


def test_batch_against_oracle(spcn, ctx, setup):
    tiles, stats, tgt, p = setup
    idx = [2, 13]
    outs = [torch.empty_like(tiles[i]) for i in idx]
    p99, _ = spcn.normalize_batched(ctx, [tiles[i] for i in idx], [stats[i] for i in idx], tgt,
                                    outs, p)
    Wt = np.asarray(np.array(tgt.basis, np.float32), np.float64)
    i0t = np.asarray(np.array(tgt.i0[:], np.float32), np.float64)
    for k, i in enumerate(idx):
        img = tiles[i].cpu().numpy()
        W = np.asarray(np.array(stats[i].basis, np.float32), np.float64)
        i0 = np.asarray(np.array(stats[i].i0[:], np.float32), np.float64)
        p_src = O.stain_percentile(img, W, i0)
        ref = O.to_uint8(O.normalize_float(img, W, i0, p_src, Wt, i0t, np.array(tgt.p99[:])))
        diff = np.abs(outs[k].cpu().numpy().astype(int) - ref.astype(int))
        assert np.mean(np.any(diff > 1, axis=-1)) <= 1e-4, diff.max()
        for j in range(2):
            assert abs(p99[k][j] - p_src[j]) <= 1e-5 * max(p_src[j], 1e-30)


def test_batch_many_tiles(spcn, ctx, setup):
    """More tiles than the grid-wide select (1024) and pass 2's preloaded
    tile table (2048) take: the staged schedule's percentiles then come from
    one block per tile and pass 2 reads each item's tile state.  Small tiles
    of every shape; bit-identical to sequential calls."""
    _, slide_stats, tgt, p = setup
    g = torch.Generator(device="cpu")
    g.manual_seed(5)
    tiles, stats = [], []
    for k in range(2100):
        h = int(torch.randint(8, 48, (1,), generator=g))
        w = int(torch.randint(8, 48, (1,), generator=g))
        tiles.append(synth.make_image_torch(h, w, 9000 + k, W=synth.stain_basis(2000 + k % 4),
                                            device="cuda", blobs=False))
        stats.append(slide_stats[k % 4])
    ref_outs, ref_p99 = sequential(ctx, tiles, stats, tgt, p)
    outs = [torch.empty_like(t) for t in tiles]
    p99, status, _ = run_batch(spcn, ctx, tiles, stats, tgt, outs, p, "staged")
    assert status == [0] * len(tiles)
    assert_same(outs, ref_outs, p99, ref_p99)
    # the persistent schedule needs the grid-wide select (at most 1024 tiles)
    b = spcn.Batch(ctx, tiles, stats, tgt, outs, p)
    with pytest.raises(spcn.SpcnError) as e:
        b.set_config(16 * 1024, "persistent")
    assert e.value.kind == "INVALID_ARG"
    b.close()


def test_batch_rejects_overlapping_output(spcn, ctx, setup):
    tiles, stats, tgt, p = setup
    with pytest.raises(spcn.SpcnError) as e:
        spcn.normalize_batched(ctx, [tiles[3]], [stats[3]], tgt, [tiles[3]], p)
    assert e.value.kind == "INVALID_ARG"


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("thresh", [220, 255])
def test_batch_white_regions(spcn, ctx, setup, thresh, sched):
    """Tiles with large white regions (blob background plus painted white
    rectangles) and ragged widths: pass 1 drops all-white chunks and counts
    row-end partial chunks pixel by pixel; at threshold 255 no pixel is white
    and the padding of partial chunks must not be counted.  Bit-identical to
    the single-image path."""
    _, slide_stats, tgt, _ = setup
    sizes = [(700, 999), (333, 1201), (1024, 1024), (45, 2000), (1500, 17), (600, 641)]
    g = torch.Generator(device="cpu")
    g.manual_seed(11)
    tiles = []
    for k, (h, w) in enumerate(sizes):
        t = synth.make_image_torch(h, w, 5000 + k, W=synth.stain_basis(2000 + k % 4),
                                   device="cuda", blobs=min(h, w) >= 256)
        for _ in range(6):
            rh = int(torch.randint(1, h, (1,), generator=g))
            rw = int(torch.randint(1, w, (1,), generator=g))
            y = int(torch.randint(0, h - rh + 1, (1,), generator=g))
            x = int(torch.randint(0, w - rw + 1, (1,), generator=g))
            t[y:y + rh, x:x + rw] = torch.randint(236, 256, (rh, rw, 3), generator=g,
                                                  dtype=torch.int32).to(torch.uint8).cuda()
        tiles.append(t)
    stats = [slide_stats[k % 4] for k in range(len(tiles))]
    p = spcn.params(white_thresh=thresh)
    ref_outs, ref_p99 = sequential(ctx, tiles, stats, tgt, p)
    outs = [torch.empty_like(t) for t in tiles]
    p99, status, _ = run_batch(spcn, ctx, tiles, stats, tgt, outs, p, sched)
    assert status == [0] * len(tiles)
    assert_same(outs, ref_outs, p99, ref_p99)


def test_batch_at_benchmark_tile_sizes_against_oracle(spcn, ctx):
    """The three largest tiles of the benchmark's 256-tile layout (about
    3700 x 3600 px each, blob images of 13.4, 11.6 and 10.7 Mpx) and five of
    its small ones, with per-slide statistics from a 1% hash sample of a
    2048^2 slide sample, under the default (staged) schedule: every tile's
    percentile within 1e-5 of the oracle's exact FP64 P99 over all of its
    non-white pixels, and 20000 seeded pixels per tile within 1 of the
    oracle's normalisation on >= 99.99% of them."""
    layout = synth.batch_layout(32, 8, 256, 4096, seed=3)
    by_size = sorted(range(len(layout)), key=lambda k: layout[k][1] * layout[k][2])
    pick = by_size[-3:] + by_size[:5]
    p = spcn.params(sample_mode="hash", sample_rate=0.01, seed=0)
    slide_st = {}
    for k in pick:
        s = layout[k][0]
        if s not in slide_st:
            smp = synth.make_image_torch(2048, 2048, 2100 + s, W=synth.stain_basis(2000 + s),
                                         device="cuda", blobs=True)
            slide_st[s] = ctx.estimate_basis(smp, p)
    tiles = [synth.make_image_torch(layout[k][1], layout[k][2], 3000 + k,
                                    W=synth.stain_basis(2000 + layout[k][0]), device="cuda",
                                    blobs=True) for k in pick]
    stats = [slide_st[layout[k][0]] for k in pick]
    tgt_img = synth.make_image_torch(2048, 2048, 1, device="cuda", blobs=True)
    tgt = ctx.estimate_basis(tgt_img, p)
    tgt.p99[0], tgt.p99[1] = ctx.stain_percentile(tgt_img, tgt, p)
    outs = [torch.empty_like(t) for t in tiles]
    b = spcn.Batch(ctx, tiles, stats, tgt, outs, p)
    assert b.config["schedule"] == "staged"
    b.run()
    p99, status, fallback = b.results(fallback=True)
    b.close()
    assert status == [0] * len(tiles)
    Wt = np.asarray(np.array(tgt.basis, np.float32), np.float64)
    i0t = np.asarray(np.array(tgt.i0[:], np.float32), np.float64)
    rng = np.random.default_rng(17)
    for k, (t, st) in enumerate(zip(tiles, stats)):
        img = t.cpu().numpy()
        W = np.asarray(np.array(st.basis, np.float32), np.float64)
        i0 = np.asarray(np.array(st.i0[:], np.float32), np.float64)
        p_src = O.stain_percentile(img, W, i0)
        for j in range(2):
            assert abs(p99[k][j] - p_src[j]) <= 1e-5 * max(p_src[j], 1e-30), (k, j, p99[k], p_src)
        n = min(20000, img.shape[0] * img.shape[1])
        flat = rng.choice(img.shape[0] * img.shape[1], size=n, replace=False)
        px = img.reshape(-1, 3)[flat][None]
        ref = O.to_uint8(O.normalize_float(px, W, i0, p_src, Wt, i0t, np.array(tgt.p99[:])))[0]
        got = outs[k].cpu().numpy().reshape(-1, 3)[flat]
        diff = np.abs(got.astype(int) - ref.astype(int))
        assert np.mean(np.any(diff > 1, axis=-1)) <= 1e-4, (k, diff.max())
