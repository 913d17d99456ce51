"""The paper's earlier choices as flags (spcn_params.flags), each against the
FP64 oracle's matching option, through the C ABI.

* SPCN_FLAG_I0_255           -- §2.1 Eq. 1, i0 fixed at 255;
* SPCN_FLAG_ORDER_BLUE       -- §3.1 item 3's original heuristic (reading R14);
* SPCN_FLAG_P99_SAMPLED      -- §3.1 item 2's sub-sampled percentile used for
                                Eq. 3 (no pass 1);
* SPCN_FLAG_P99_PATCH_MEDIAN -- §3.2 item 4, median of per-patch percentiles.

Tolerances are those of the default path: basis 1e-5, uint8 within 1 on
>= 99.99% of pixels; the patch median is also checked bit for bit against the
type-7 statistics of the library's own FP32 densities of each patch.
"""
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


def to_dev(img):
    return torch.from_numpy(np.ascontiguousarray(img)).cuda()


def type7(a, p):
    a = np.sort(np.asarray(a, dtype=np.float32)).astype(np.float64)
    n = a.size
    pos = (n - 1) * (p / 100.0)
    k = int(math.floor(pos))
    t = pos - k
    if k + 1 >= n:
        return float(a[n - 1])
    return float(a[k]) + t * (float(a[k + 1]) - float(a[k]))


def close_uint8(a, b):
    d = np.abs(a.astype(int) - b.astype(int))
    assert (d > 1).mean() <= 1e-4, d.max()


def test_i0_255(spcn, ctx):
    img = synth.make_image(512, 512, 1301, white=(240.0, 232.0, 247.0))
    o = O.estimate_basis(img, O.Params(sample_mode="all", i0_fixed_255=True))
    g = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="all", flags=spcn.FLAG_I0_255))
    assert list(g.i0) == [255.0, 255.0, 255.0]
    assert np.max(np.abs(np.array(g.basis) - o.W)) <= 1e-5
    for j in range(2):
        assert abs(g.p99[j] - o.p99[j]) <= 1e-4 * o.p99[j]
    d = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="all"))
    assert max(d.i0) < 250.0


def test_order_blue_swaps_blue_tinged_eosin(spcn, ctx):
    hema = np.array([0.75, 0.45, 0.49]); hema /= np.linalg.norm(hema)
    eosin = np.array([0.10, 0.80, 0.59]); eosin /= np.linalg.norm(eosin)
    W = np.column_stack([hema, eosin])
    img = synth.make_image(384, 384, 1302, W=W, pure=True)
    o_rb = O.estimate_basis(img, O.Params(sample_mode="all"))
    o_b = O.estimate_basis(img, O.Params(sample_mode="all", order="blue"))
    assert np.allclose(o_b.W, o_rb.W[:, ::-1])
    g_rb = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="all"))
    g_b = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="all", flags=spcn.FLAG_ORDER_BLUE))
    assert np.max(np.abs(np.array(g_rb.basis) - o_rb.W)) <= 1e-5
    assert np.max(np.abs(np.array(g_b.basis) - o_b.W)) <= 1e-5
    for j in range(2):
        assert abs(g_b.p99[j] - o_b.p99[j]) <= 1e-4 * o_b.p99[j]


@pytest.mark.parametrize("shape", [(512, 512), (77, 123)])
def test_p99_sampled_normalize(spcn, ctx, shape):
    h, w = shape
    img = synth.make_image(h, w, 1303 + h)
    tgt_img = synth.make_image(256, 256, 1)
    p = spcn.params(sample_mode="all")
    src = ctx.estimate_basis(to_dev(img), p)          # p99 over the sampled non-white pixels
    tgt = ctx.estimate_basis(to_dev(tgt_img), p)
    pf = spcn.params(sample_mode="all", flags=spcn.FLAG_P99_SAMPLED)
    ctx.kernel_timing(True)
    out, used = ctx.normalize(to_dev(img), src, tgt, pf, return_p99=True)
    assert ctx.kernel_times("pass1")[1] == 0
    ctx.kernel_timing(False)
    assert used[0] == src.p99[0] and used[1] == src.p99[1]
    so = O.Stats(W=np.array(src.basis, dtype=np.float32).astype(np.float64),
                 i0=np.float32(src.i0).astype(np.float64), p99=np.array(src.p99[:]))
    to = O.Stats(W=np.array(tgt.basis, dtype=np.float32).astype(np.float64),
                 i0=np.float32(tgt.i0).astype(np.float64), p99=np.array(tgt.p99[:]))
    close_uint8(out.cpu().numpy(), O.normalize(img, so, to))
    # the one-call path with the flag gives the same bytes and reports the sampled percentile
    out2, st2 = ctx.normalize_estimated(to_dev(img), tgt, pf, return_stats=True)
    assert torch.equal(out, out2)
    assert st2.p99[0] == src.p99[0] and st2.p99[1] == src.p99[1]


def test_p99_sampled_rejects_negative_percentile(spcn, ctx):
    img = to_dev(synth.make_image(64, 64, 1304))
    st = ctx.estimate_basis(img, spcn.params(sample_mode="all"))
    st.p99[0] = -1.0
    with pytest.raises(spcn.SpcnError):
        ctx.normalize(img, st, st, spcn.params(flags=spcn.FLAG_P99_SAMPLED))


def test_patch_median_against_oracle_and_own_densities(spcn, ctx):
    img = synth.make_image(600, 700, 1305, blobs=True)
    kw = dict(sample_mode="patches", n_patches=7, patch_size=64, seed=9)
    o = O.estimate_basis(img, O.Params(p99_patch_median=True, **kw))
    g = ctx.estimate_basis(to_dev(img), spcn.params(flags=spcn.FLAG_P99_PATCH_MEDIAN, **kw))
    assert np.max(np.abs(np.array(g.basis) - o.W)) <= 1e-5
    for j in range(2):
        assert abs(g.p99[j] - o.p99[j]) <= 1e-4 * o.p99[j]
    # bit for bit: per kept patch the type-7 P99 of the library's own FP32
    # densities over its non-white pixels, then the type-7 median
    pp = O.Params(**kw)
    per = []
    for patch in O.select_patches(img, pp):
        P = 64
        pim = patch.reshape(P, P, 3)
        Hd = ctx.stain_densities(to_dev(pim), g).cpu().numpy()
        nw = O.nonwhite_mask(patch)
        per.append([type7(Hd[j][nw], 99.0) for j in range(2)])
    per = np.array(per)
    for j in range(2):
        v = np.sort(per[:, j])
        n = v.size
        pos = (n - 1) * 0.5
        k = int(math.floor(pos))
        t = pos - k
        med = v[k] if k + 1 >= n else v[k] + t * (v[k + 1] - v[k])
        assert g.p99[j] == med, (j, g.p99[j], med)


def test_patch_median_with_even_count_and_one_patch(spcn, ctx):
    img = synth.make_image(600, 700, 1306, blobs=True)
    for n in (1, 6):
        kw = dict(sample_mode="patches", n_patches=n, patch_size=48, seed=4)
        o = O.estimate_basis(img, O.Params(p99_patch_median=True, **kw))
        g = ctx.estimate_basis(to_dev(img), spcn.params(flags=spcn.FLAG_P99_PATCH_MEDIAN, **kw))
        for j in range(2):
            assert abs(g.p99[j] - o.p99[j]) <= 1e-4 * o.p99[j]
    one = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="patches", n_patches=1,
                                                      patch_size=48, seed=4))
    med = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="patches", n_patches=1,
                                                      patch_size=48, seed=4,
                                                      flags=spcn.FLAG_P99_PATCH_MEDIAN))
    assert one.p99[0] == med.p99[0] and one.p99[1] == med.p99[1]


def test_flag_validation(spcn, ctx):
    img = to_dev(synth.make_image(64, 64, 1307))
    with pytest.raises(spcn.SpcnError):
        ctx.estimate_basis(img, spcn.params(sample_mode="all", flags=spcn.FLAG_P99_PATCH_MEDIAN))
    with pytest.raises(spcn.SpcnError):
        ctx.estimate_basis(img, spcn.params(sample_mode="all", flags=0x100))
    st = ctx.estimate_basis(img, spcn.params(sample_mode="all"))
    out = torch.empty_like(img)
    with pytest.raises(spcn.SpcnError):
        spcn.normalize_batched(ctx, [img], [st], st, [out], spcn.params(flags=spcn.FLAG_P99_SAMPLED))


# ---------------------------------------------------------------- SPCN_FLAG_H_PINV (§2.1)
def pinv_stats(spcn, img_seed=1310):
    W = synth.stain_basis(img_seed)
    i0 = np.array([250.0, 247.0, 253.0])
    return W, i0, spcn.Stats.from_values(W, i0)


def test_pinv_densities_match_oracle(spcn, ctx):
    img = synth.make_image(130, 257, 1310)
    W, i0, st = pinv_stats(spcn)
    p = spcn.params(flags=spcn.FLAG_H_PINV)
    Hg = ctx.stain_densities(to_dev(img), st, p).cpu().numpy()
    Ho = O.stain_densities(img, np.float32(W).astype(np.float64), np.float32(i0).astype(np.float64),
                           h_solve="pinv")
    assert (Ho < 0).mean() > 0.05                      # signed densities really occur
    assert np.all(np.abs(Hg - Ho) <= 1e-5 * np.maximum(np.abs(Ho), 1.0)), np.max(np.abs(Hg - Ho))


@pytest.mark.parametrize("pct,hint", [(99.0, "exact"), (99.0, "none"), (1.0, "none"), (1.0, "exact"),
                                      (50.0, "exact")])
def test_pinv_percentile_bit_exact(spcn, ctx, pct, hint):
    img = synth.make_image(300, 411, 1311)
    W, i0, st = pinv_stats(spcn)
    p = spcn.params(flags=spcn.FLAG_H_PINV, stain_pct=pct)
    dev = to_dev(img)
    Hg = ctx.stain_densities(dev, st, p).cpu().numpy()
    nw = O.nonwhite_mask(img.reshape(-1, 3))
    ref = [type7(Hg[j][nw], pct) for j in range(2)]
    if pct == 1.0:
        assert ref[0] < 0 or ref[1] < 0                # the signed keys are exercised
    if hint == "exact":
        st.p99[0], st.p99[1] = ref
    got = ctx.stain_percentile(dev, st, p)
    assert got[0] == ref[0] and got[1] == ref[1], (got, ref)
    o = O.stain_percentile(img, np.float32(W).astype(np.float64), np.float32(i0).astype(np.float64),
                           O.Params(h_solve="pinv", stain_pct=pct))
    for j in range(2):
        assert abs(got[j] - o[j]) <= 1e-5 * max(abs(o[j]), 1.0)


def test_pinv_normalize_matches_oracle(spcn, ctx):
    img = synth.make_image(256, 320, 1312)
    tgt_img = synth.make_image(128, 128, 1)
    pe = spcn.params(sample_mode="all")
    src = ctx.estimate_basis(to_dev(img), pe)
    tgt = ctx.estimate_basis(to_dev(tgt_img), pe)
    p = spcn.params(flags=spcn.FLAG_H_PINV)
    tgt.p99[0], tgt.p99[1] = ctx.stain_percentile(to_dev(tgt_img), tgt, p)
    out, p99 = ctx.normalize(to_dev(img), src, tgt, p, return_p99=True)
    so = O.Stats(W=np.array(src.basis, dtype=np.float32).astype(np.float64),
                 i0=np.float32(src.i0).astype(np.float64), p99=np.array(p99))
    to = O.Stats(W=np.array(tgt.basis, dtype=np.float32).astype(np.float64),
                 i0=np.float32(tgt.i0).astype(np.float64), p99=np.array(tgt.p99[:]))
    ref = O.normalize(img, so, to, h_solve="pinv")
    op = O.stain_percentile(img, so.W, so.i0, O.Params(h_solve="pinv"))
    for j in range(2):
        assert abs(p99[j] - op[j]) <= 1e-5 * max(abs(op[j]), 1.0)
    close_uint8(out.cpu().numpy(), ref)
    # pixels the pseudo-inverse makes brighter than the target white are clamped
    raw = O.normalize_float(img, so.W, so.i0, so.p99, to.W, to.i0, to.p99, h_solve="pinv")
    assert np.any(raw > 255.0)


def test_pinv_estimate_and_one_call_path(spcn, ctx):
    img = synth.make_image(600, 700, 1313, blobs=True)
    tgt = ctx.estimate_basis(to_dev(synth.make_image(128, 128, 1)), spcn.params(sample_mode="all"))
    for kw in (dict(sample_mode="all"), dict(sample_mode="patches", n_patches=9, patch_size=64,
                                             seed=2)):
        o = O.estimate_basis(img, O.Params(h_solve="pinv", **{k: v for k, v in kw.items()}))
        p = spcn.params(flags=spcn.FLAG_H_PINV, **kw)
        g = ctx.estimate_basis(to_dev(img), p)
        assert np.max(np.abs(np.array(g.basis) - o.W)) <= 1e-5
        for j in range(2):
            assert abs(g.p99[j] - o.p99[j]) <= 1e-4 * max(abs(o.p99[j]), 1.0)
        out1, p99 = ctx.normalize(to_dev(img), g, tgt, p, return_p99=True)
        out2, st2 = ctx.normalize_estimated(to_dev(img), tgt, p, return_stats=True)
        assert torch.equal(out1, out2) and st2.p99[0] == p99[0] and st2.p99[1] == p99[1]
    # with the patch median
    kw = dict(sample_mode="patches", n_patches=9, patch_size=64, seed=2)
    o = O.estimate_basis(img, O.Params(h_solve="pinv", p99_patch_median=True, **kw))
    g = ctx.estimate_basis(to_dev(img), spcn.params(
        flags=spcn.FLAG_H_PINV | spcn.FLAG_P99_PATCH_MEDIAN, **kw))
    for j in range(2):
        assert abs(g.p99[j] - o.p99[j]) <= 1e-4 * max(abs(o.p99[j]), 1.0)


def test_pinv_rejected_where_not_available(spcn, ctx):
    img = to_dev(synth.make_image(64, 64, 1314))
    st = ctx.estimate_basis(img, spcn.params(sample_mode="all"))
    out = torch.empty_like(img)
    with pytest.raises(spcn.SpcnError):
        spcn.normalize_batched(ctx, [img], [st], st, [out], spcn.params(flags=spcn.FLAG_H_PINV))
    x = torch.rand((1, 3, 8, 8), device="cuda") * 255
    wt = torch.tensor(np.array(st.basis, dtype=np.float32), device="cuda")
    with pytest.raises(spcn.SpcnError):
        spcn.normalize_f32(ctx, x, wt, [st], st, p=spcn.params(flags=spcn.FLAG_H_PINV))


# ---------------------------------------------------------------- SPCN_FLAG_I0_OUT_255 (Eq. 4)
def test_i0_out_255_all_entry_points(spcn, ctx):
    img = synth.make_image(300, 411, 1320)
    tgt_img = synth.make_image(128, 128, 1, white=(232.0, 240.0, 246.0))
    pe = spcn.params(sample_mode="all")
    src = ctx.estimate_basis(to_dev(img), pe)
    tgt = ctx.estimate_basis(to_dev(tgt_img), pe)
    tgt.p99[0], tgt.p99[1] = ctx.stain_percentile(to_dev(tgt_img), tgt, pe)
    assert max(tgt.i0) < 250
    pf = spcn.params(sample_mode="all", flags=spcn.FLAG_I0_OUT_255)
    out, p99 = ctx.normalize(to_dev(img), src, tgt, pf, return_p99=True)
    so = O.Stats(W=np.array(src.basis, dtype=np.float32).astype(np.float64),
                 i0=np.float32(src.i0).astype(np.float64), p99=np.array(p99))
    to = O.Stats(W=np.array(tgt.basis, dtype=np.float32).astype(np.float64),
                 i0=np.float32(tgt.i0).astype(np.float64), p99=np.array(tgt.p99[:]))
    close_uint8(out.cpu().numpy(), O.normalize(img, so, to, i0_out_255=True))
    bg = ~O.nonwhite_mask(img.reshape(-1, 3))
    assert np.mean(out.cpu().numpy().reshape(-1, 3)[bg] >= 250) > 0.9   # white maps to white
    out2 = ctx.normalize_estimated(to_dev(img), tgt, pf)
    out3 = ctx.normalize(to_dev(img), src, tgt, pf)
    assert torch.equal(out2, out3)
    # batch: bit-identical to the single-image path with the flag
    tiles = [to_dev(img), to_dev(synth.make_image(97, 130, 1321))]
    stats = [src, ctx.estimate_basis(tiles[1], pe)]
    outs = [torch.empty_like(t) for t in tiles]
    spcn.normalize_batched(ctx, tiles, stats, tgt, outs, pf)
    for t, s_, o in zip(tiles, stats, outs):
        assert torch.equal(o, ctx.normalize(t, s_, tgt, pf))
    # float path: i0_t replaced by 255 scales every output channel by 255 / i0_t
    x = torch.from_numpy(np.ascontiguousarray(img[:64, :64].transpose(2, 0, 1)[None]).astype(np.float32)).cuda()
    wt = torch.tensor(np.array(tgt.basis, dtype=np.float32), device="cuda")
    src.p99[0], src.p99[1] = p99
    y0 = spcn.normalize_f32(ctx, x, wt, [src], tgt, p=pe)
    y1 = spcn.normalize_f32(ctx, x, wt, [src], tgt, p=pf)
    ratio = torch.tensor([255.0 / v for v in tgt.i0], device="cuda").view(1, 3, 1, 1)
    assert torch.allclose(y1, y0 * ratio, rtol=1e-5, atol=1e-3)
