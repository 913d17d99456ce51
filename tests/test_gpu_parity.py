"""GPU parity of the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (written here, derived from the arithmetic):
  * densities H: |dh| <= 1e-5 max(|h|, 1) (FP32 vs FP64); a pixel may differ
    more only where the oracle's solution sits within 1e-5 of an active-set
    change (KKT margin), and such pixels are at most 1e-4 of the image;
  * percentile: bit-exact against the type-7 percentile of the GPU's own FP32
    densities over the same non-white mask;
  * uint8 output: within 1 on >= 99.99% of pixels;
  * basis: max |dW| <= 1e-5; i0 equal to the oracle's value rounded to FP32.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import spcn_oracle as O  # noqa: E402
from paper_1901_03088_b300 import synth  # noqa: E402

H_TOL = 1e-5
KINK = 1e-5


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


def f32_stats(spcn, st):
    """Oracle statistics rounded to the FP32 record the library takes."""
    return spcn.Stats.from_values(np.float32(st.W), np.float32(st.i0), st.p99)


def as64(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def oracle_kkt_margin(img, W, i0, lam=0.1):
    V = O.optical_density(img.reshape(-1, 3), i0).T
    H = O.lasso2(V, W, lam)
    g = (W.T @ W) @ H - W.T @ V + lam
    m = np.where(H > 0, H, g)           # active: distance to leaving; inactive: gradient
    return H, np.min(np.abs(m), axis=0)


def check_h(H_gpu, H_ref, margin):
    bad = np.abs(H_gpu - H_ref) > H_TOL * np.maximum(np.abs(H_ref), 1.0)
    badpx = np.any(bad, axis=0)
    assert np.all(margin[badpx] < KINK), np.max(np.abs(H_gpu - H_ref))
    assert badpx.mean() <= 1e-4


def gpu_type7(values, p):
    a = np.sort(values.astype(np.float32)).astype(np.float64)
    n = a.size
    pos = (n - 1) * (p / 100.0)
    k = int(math.floor(pos))
    t = pos - k
    if k + 1 >= n:
        return float(a[n - 1])
    lo, hi = float(a[k]), float(a[k + 1])
    return lo + t * (hi - lo)


# ------------------------------------------------------------------ densities
@pytest.mark.parametrize("shape", [(512, 512), (1, 1), (1, 37), (37, 1), (45, 83), (130, 257)])
def test_densities_match_oracle(spcn, ctx, shape):
    h, w = shape
    img = synth.make_image(h, w, 1000 + h + w)
    W = synth.stain_basis(7)
    i0 = np.array([250.0, 247.0, 253.0])
    st = spcn.Stats.from_values(W, i0)
    H_gpu = ctx.stain_densities(to_dev(img), st).cpu().numpy()
    H_ref, margin = oracle_kkt_margin(img, as64(W), as64(i0))
    check_h(H_gpu, H_ref, margin)
    assert not np.any(np.signbit(H_gpu))          # zeros are +0, keys stay ordered


def test_densities_pitched_and_unaligned(spcn, ctx):
    img = synth.make_image(67, 91, 5)
    big = np.zeros((67, 91 * 3 + 29), np.uint8)          # pitch 302 bytes, not 16-aligned
    big[:, 1:1 + 91 * 3] = img.reshape(67, -1)              # start at byte 1
    dev = to_dev(big)
    view = torch.as_strided(dev, (67, 91, 3), (big.shape[1], 3, 1), storage_offset=1)
    W = synth.stain_basis(8)
    st = spcn.Stats.from_values(W, [255, 255, 255])
    H_gpu = ctx.stain_densities(view, st).cpu().numpy()
    H_ref, margin = oracle_kkt_margin(img, as64(W), as64([255, 255, 255]))
    check_h(H_gpu, H_ref, margin)


# ------------------------------------------------------------------ percentile
@pytest.mark.parametrize("hint", ["oracle", "none", "far_low", "far_high"])
def test_percentile_bit_exact_on_gpu_densities(spcn, ctx, hint):
    img = synth.make_image(300, 411, 1001)
    o = O.full_stats(img)
    st = f32_stats(spcn, o)
    if hint == "none":
        st.p99[0] = st.p99[1] = 0.0
    elif hint == "far_low":
        st.p99[0], st.p99[1] = o.p99[0] * 0.5, o.p99[1] * 0.5
    elif hint == "far_high":
        st.p99[0], st.p99[1] = o.p99[0] * 3.0, o.p99[1] * 3.0
    dev = to_dev(img)
    p_gpu = ctx.stain_percentile(dev, st)
    H_gpu = ctx.stain_densities(dev, st).cpu().numpy()
    nw = O.nonwhite_mask(img.reshape(-1, 3))
    for j in range(2):
        assert p_gpu[j] == gpu_type7(H_gpu[j][nw], 99.0)
        assert abs(p_gpu[j] - o.p99[j]) <= 1e-5 * o.p99[j]


def test_percentile_other_levels(spcn, ctx):
    img = synth.make_image(200, 200, 1002)
    o = O.full_stats(img)
    st = f32_stats(spcn, o)
    dev = to_dev(img)
    H_gpu = ctx.stain_densities(dev, st).cpu().numpy()
    nw = O.nonwhite_mask(img.reshape(-1, 3))
    for pct in (0.0, 50.0, 100.0, 97.5):
        p = spcn.params(stain_pct=pct)
        got = ctx.stain_percentile(dev, st, p)
        for j in range(2):
            assert got[j] == gpu_type7(H_gpu[j][nw], pct)


# ------------------------------------------------------------------ normalize
@pytest.mark.parametrize("shape", [(512, 512), (77, 123), (1, 1)])
def test_normalize_matches_oracle(spcn, ctx, shape):
    h, w = shape
    src = synth.make_image(h, w, 1000)
    if h * w == 1:
        src[...] = (120, 80, 150)
    tgt = synth.make_image(256, 256, 1)
    so = O.full_stats(synth.make_image(256, 256, 1000)) if h * w == 1 else O.full_stats(src)
    to = O.full_stats(tgt)
    s_st, t_st = f32_stats(spcn, so), f32_stats(spcn, to)
    Ws, i0s, Wt, i0t = as64(so.W), as64(so.i0), as64(to.W), as64(to.i0)
    p_src = O.stain_percentile(src, Ws, i0s)
    p_tgt = np.array(t_st.p99[:])
    ref = O.to_uint8(O.normalize_float(src, Ws, i0s, p_src, Wt, i0t, p_tgt))
    out, p_gpu = ctx.normalize(to_dev(src), s_st, t_st, return_p99=True)
    out = out.cpu().numpy()
    diff = np.abs(out.astype(int) - ref.astype(int))
    assert np.mean(np.any(diff > 1, axis=-1)) <= 1e-4, diff.max()
    for j in range(2):
        assert abs(p_gpu[j] - p_src[j]) <= 1e-5 * max(p_src[j], 1e-30)


def test_normalize_pitched_output(spcn, ctx):
    src = synth.make_image(64, 100, 1003)
    o = O.full_stats(src)
    st = f32_stats(spcn, o)
    dev = to_dev(src)
    flat = ctx.normalize(dev, st, st).cpu().numpy()
    buf = torch.zeros((64, 100 * 3 + 13), dtype=torch.uint8, device="cuda")
    view = torch.as_strided(buf, (64, 100, 3), (buf.shape[1], 3, 1), storage_offset=5)
    ctx.normalize(dev, st, st, out=view)
    assert np.array_equal(view.cpu().numpy(), flat)
    assert np.all(buf.cpu().numpy()[:, :5] == 0)


def test_identity_normalisation_is_near_identity(spcn, ctx):
    # same statistics on both sides: Eq. 3's scale is 1 and Eq. 4 inverts Eq. 1
    # except where the lasso shrinks densities, so compare with the oracle
    src = synth.make_image(128, 128, 1004)
    o = O.full_stats(src)
    st = f32_stats(spcn, o)
    out = ctx.normalize(to_dev(src), st, st).cpu().numpy()
    W, i0 = as64(o.W), as64(o.i0)
    p = O.stain_percentile(src, W, i0)
    ref = O.to_uint8(O.normalize_float(src, W, i0, p, W, i0, p))
    assert np.abs(out.astype(int) - ref.astype(int)).max() <= 1


# ------------------------------------------------------------------ basis estimation
def test_estimate_basis_all_pixels(spcn, ctx):
    img = synth.make_image(512, 512, 1000)
    p = O.Params(sample_mode="all")
    o = O.estimate_basis(img, p)
    g = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="all"))
    assert g.n_sample == o.n_sample and g.n_nonwhite == o.n_nonwhite and g.n_bright == o.n_bright
    assert np.array_equal(np.array(g.i0[:], np.float32), np.float32(o.i0))
    Wg = np.array(g.basis)
    assert np.max(np.abs(Wg - o.W)) <= 1e-5, (Wg, o.W)
    for j in range(2):
        assert abs(g.p99[j] - o.p99[j]) <= 1e-4 * o.p99[j]


def test_estimate_basis_hash_sample(spcn, ctx):
    img = synth.make_image(1024, 768, 1005, blobs=True)
    p = O.Params(sample_mode="hash", sample_rate=0.05, seed=77)
    o = O.estimate_basis(img, p)
    g = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="hash", sample_rate=0.05, seed=77))
    assert g.n_sample == o.n_sample and g.n_nonwhite == o.n_nonwhite and g.n_bright == o.n_bright
    assert np.array_equal(np.array(g.i0[:], np.float32), np.float32(o.i0))
    assert np.max(np.abs(np.array(g.basis) - o.W)) <= 1e-5


def test_estimate_basis_patches(spcn, ctx):
    img = synth.make_image(600, 700, 1006, blobs=True)
    p = O.Params(sample_mode="patches", n_patches=12, patch_size=64, seed=5)
    o = O.estimate_basis(img, p)
    g = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="patches", n_patches=12,
                                                    patch_size=64, seed=5))
    assert g.n_sample == o.n_sample and g.n_nonwhite == o.n_nonwhite
    assert np.array_equal(np.array(g.i0[:], np.float32), np.float32(o.i0))
    assert np.max(np.abs(np.array(g.basis) - o.W)) <= 1e-5


@pytest.mark.parametrize("patch_size", [1, 2, 3, 37, 50])
def test_estimate_basis_patches_odd_sizes_and_sample_order(spcn, ctx, patch_size):
    """Patch sampling at sizes whose last group of four rows is partial or that
    are too small for the per-patch split (1, 2: the general compaction).
    i0 from every k-th bright pixel (a small cap, over a tinted background
    whose bright pixels differ) depends on the order of the bright list,
    which must be the sample order: patches in acceptance order, each in
    raster order."""
    img = synth.make_image(300, 260, 1011, blobs=True, white=(232.0, 240.0, 247.0))
    kw = dict(sample_mode="patches", n_patches=30, patch_size=patch_size, seed=8,
              i0_max_samples=40)
    o = O.estimate_basis(img, O.Params(**kw))
    g = ctx.estimate_basis(to_dev(img), spcn.params(**kw))
    assert g.n_sample == o.n_sample and g.n_nonwhite == o.n_nonwhite and g.n_bright == o.n_bright
    assert np.array_equal(np.array(g.i0[:], np.float32), np.float32(o.i0))
    assert np.max(np.abs(np.array(g.basis) - o.W)) <= 1e-5


def test_estimate_basis_i0_cap_and_tinted_background(spcn, ctx):
    img = synth.make_image(700, 700, 1007, white=(224.0, 236.0, 250.0))
    p = O.Params(sample_mode="all", i0_max_samples=5000)
    o = O.estimate_basis(img, p)
    g = ctx.estimate_basis(to_dev(img), spcn.params(sample_mode="all", i0_max_samples=5000))
    assert np.array_equal(np.array(g.i0[:], np.float32), np.float32(o.i0))
    assert np.max(np.abs(np.array(g.basis) - o.W)) <= 1e-5


# ------------------------------------------------------------------ properties
def test_deterministic_runs(spcn, ctx):
    img = to_dev(synth.make_image(640, 480, 1008, blobs=True))
    tgt = to_dev(synth.make_image(256, 256, 1))
    p = spcn.params(sample_mode="hash", sample_rate=0.2)
    a1 = ctx.estimate_basis(img, p)
    a2 = ctx.estimate_basis(img, p)
    assert bytes(a1) == bytes(a2)
    t = ctx.estimate_basis(tgt, p)
    t.p99[0], t.p99[1] = ctx.stain_percentile(tgt, t)
    o1, q1 = ctx.normalize(img, a1, t, return_p99=True)
    o2, q2 = ctx.normalize(img, a1, t, return_p99=True)
    assert torch.equal(o1, o2) and q1 == q2


def test_errors_are_reported(spcn, ctx):
    white = torch.full((64, 64, 3), 250, dtype=torch.uint8, device="cuda")
    with pytest.raises(spcn.SpcnError) as e:
        ctx.estimate_basis(white, spcn.params(sample_mode="all"))
    assert e.value.kind == "NO_TISSUE"
    for size in (16, 2):   # per-patch split and general compaction: no patch kept
        with pytest.raises(spcn.SpcnError) as e:
            ctx.estimate_basis(white, spcn.params(sample_mode="patches", n_patches=5,
                                                  patch_size=size, seed=1))
        assert e.value.kind == "NO_TISSUE"
    st = spcn.Stats.from_values(synth.stain_basis(1), [255, 255, 255], [1.0, 1.0])
    with pytest.raises(spcn.SpcnError) as e:
        ctx.normalize(white, st, st, return_p99=True)
    assert e.value.kind == "NO_TISSUE"
    bad = spcn.Stats.from_values([[0.6, 0.6], [0.7, 0.7], [0.3, 0.3]], [255, 255, 255])
    img = to_dev(synth.make_image(32, 32, 3))
    with pytest.raises(spcn.SpcnError) as e:
        ctx.stain_densities(img, bad)
    assert e.value.kind == "DEGENERATE_BASIS"
    neg = spcn.Stats.from_values([[-0.1, 0.6], [0.7, 0.7], [0.3, 0.3]], [255, 255, 255])
    with pytest.raises(spcn.SpcnError) as e:
        ctx.stain_densities(img, neg)
    assert e.value.kind == "INVALID_ARG"
    hi = spcn.Stats.from_values(synth.stain_basis(1), [256, 255, 255])
    with pytest.raises(spcn.SpcnError) as e:
        ctx.stain_densities(img, hi)
    assert e.value.kind == "INVALID_ARG"
    # the context stays usable
    ctx.synchronize()
    ctx.stain_densities(img, st)
    ctx.synchronize()


def test_grid_wait_gives_up_without_fault(spcn, ctx):
    assert ctx.debug_barrier_timeout(0, 1_000_000_000) == 0
    assert ctx.debug_barrier_timeout(1, 20_000_000) == -6      # TIMEOUT
    assert ctx.debug_barrier_timeout(0, 1_000_000_000) == 0
    img = to_dev(synth.make_image(64, 64, 9))
    st = spcn.Stats.from_values(synth.stain_basis(9), [255, 255, 255])
    ctx.stain_densities(img, st)
    ctx.synchronize()


# ------------------------------------------------------------------ estimate + normalise, one call
@pytest.mark.parametrize("mode", ["all", "hash", "patches"])
def test_normalize_estimated_matches_two_calls(spcn, ctx, mode):
    # the device-resident hand-off gives the bytes and statistics of
    # spcn_estimate_basis followed by spcn_normalize
    src = to_dev(synth.make_image(300, 420, 1007, blobs=True))
    tgt = to_dev(synth.make_image(256, 256, 1))
    p = spcn.params(sample_mode=mode, sample_rate=0.2, n_patches=12, patch_size=48, seed=3)
    t_st = ctx.estimate_basis(tgt, spcn.params(sample_mode="all"))
    t_st.p99[0], t_st.p99[1] = ctx.stain_percentile(tgt, t_st)
    s_st = ctx.estimate_basis(src, p)
    ref, ref_p99 = ctx.normalize(src, s_st, t_st, p, return_p99=True)
    out, st = ctx.normalize_estimated(src, t_st, p, return_stats=True)
    assert torch.equal(out, ref)
    assert list(st.W) == list(s_st.W) and list(st.i0) == list(s_st.i0)
    assert (st.p99[0], st.p99[1]) == ref_p99
    assert st.iters == s_st.iters and st.n_nonwhite == s_st.n_nonwhite
    # asynchronous form
    out2 = ctx.normalize_estimated(src, t_st, p)
    ctx.synchronize()
    assert torch.equal(out2, ref)


def test_normalize_estimated_reports_no_tissue(spcn, ctx):
    white = torch.full((64, 80, 3), 250, dtype=torch.uint8, device="cuda")
    tgt = to_dev(synth.make_image(128, 128, 1))
    t_st = ctx.estimate_basis(tgt, spcn.params(sample_mode="all"))
    with pytest.raises(spcn.SpcnError) as e:
        ctx.normalize_estimated(white, t_st, spcn.params(sample_mode="all"), return_stats=True)
    assert e.value.kind == "NO_TISSUE"
    ctx.normalize_estimated(white, t_st, spcn.params(sample_mode="all"))
    with pytest.raises(spcn.SpcnError):
        ctx.synchronize()
    # the context stays usable
    out = ctx.normalize_estimated(tgt, t_st, spcn.params(sample_mode="all"))
    ctx.synchronize()
    assert out.shape == tgt.shape
