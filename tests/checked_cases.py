"""Odd-shape cases run through the C ABI by tests/test_gpu_checked.py, once on
the bounds-checked library (in a child process, SPCN_LIBRARY=checked) and
once on the normal one.  Every call that synchronises returns the first error
any kernel recorded, so a failed device check in the checked build raises.
Returns a dict of numpy arrays (the outputs to compare bit for bit)."""
import numpy as np

from paper_1901_03088_b300 import synth


def _pitched(torch, img, extra, offset):
    """A device copy of img whose rows are `extra` bytes longer than the
    pixels and whose first byte sits `offset` bytes into the buffer."""
    h, w, _ = img.shape
    big = np.zeros((h, 3 * w + extra), np.uint8)
    big[:, offset:offset + 3 * w] = img.reshape(h, -1)
    dev = torch.from_numpy(big).cuda()
    return torch.as_strided(dev, (h, w, 3), (big.shape[1], 3, 1), storage_offset=offset), dev


def run_cases(spcn, torch):
    out = {}
    ctx = spcn.Context(0)
    W = synth.stain_basis(7)
    st = spcn.Stats.from_values(np.float32(W), [250.0, 247.0, 253.0], [2.3, 1.9])
    tgt = spcn.Stats.from_values(np.float32(synth.stain_basis(1)), [255.0, 254.0, 252.0],
                                 [2.4, 2.1])
    # densities and percentiles: odd shapes, row-end partial chunks
    for h, w in ((1, 1), (1, 37), (37, 1), (45, 83), (130, 257)):
        img = torch.from_numpy(synth.make_image(h, w, 1000 + h + w)).cuda()
        out[f"H_{h}x{w}"] = ctx.stain_densities(img, st).cpu().numpy()
        out[f"p99_{h}x{w}"] = np.array(ctx.stain_percentile(img, st))
    # pitched, unaligned source and output
    view, keep = _pitched(torch, synth.make_image(67, 91, 5), 29, 1)
    out["H_pitched"] = ctx.stain_densities(view, st).cpu().numpy()
    dst_view, dst_keep = _pitched(torch, np.zeros((67, 91, 3), np.uint8), 13, 3)
    ctx.normalize(view, st, tgt, out=dst_view)
    out["norm_pitched"] = dst_view.cpu().numpy()
    # the exact percentile after window misses (recovery and radix select)
    img = torch.from_numpy(synth.make_image(300, 411, 1001, blobs=True)).cuda()
    base = ctx.stain_percentile(img, st)
    for f in (0.0, 0.5, 2.0, 1.0):
        s2 = st.copy()
        s2.p99[0], s2.p99[1] = base[0] * f, base[1] * f
        out[f"p99_hint_{f}"] = np.array(ctx.stain_percentile(img, s2))
    # basis estimation and the one-call path, every sampling mode
    img = torch.from_numpy(synth.make_image(700, 600, 1005, blobs=True)).cuda()
    for mode, kw in (("all", {}), ("hash", dict(sample_rate=0.05, seed=3)),
                     ("patches", dict(n_patches=40, patch_size=32, seed=5))):
        p = spcn.params(sample_mode=mode, **kw)
        b = ctx.estimate_basis(img, p)
        out[f"basis_{mode}"] = np.frombuffer(bytes(b), np.uint8).copy()
        o, s_st = ctx.normalize_estimated(img, tgt, p, return_stats=True)
        out[f"est_{mode}"] = o.cpu().numpy()
    # a small batch of odd tiles, one of them pitched
    tiles = [torch.from_numpy(synth.make_image(h, w, 1100 + h)).cuda()
             for h, w in ((33, 47), (256, 129), (1, 500))]
    pv, pkeep = _pitched(torch, synth.make_image(40, 61, 77), 7, 5)
    tiles.append(pv)
    outs = [torch.zeros(t.shape, dtype=torch.uint8, device="cuda") for t in tiles]
    spcn.normalize_batched(ctx, tiles, [st] * len(tiles), tgt, outs)
    for i, o in enumerate(outs):
        out[f"batch_{i}"] = o.cpu().numpy()
    # the float form, forward and backward
    x = np.stack([synth.make_image(40, 48, 600 + b, as_float=True).transpose(2, 0, 1)
                  for b in range(3)]).astype(np.float32)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda().requires_grad_(True)
    Wd = torch.tensor(np.array(tgt.basis, np.float32), device="cuda", requires_grad=True)
    y = spcn.normalize_f32(ctx, xd, Wd, [st] * 3, tgt)
    gy = torch.from_numpy(np.random.default_rng(3).normal(size=x.shape).astype(np.float32)).cuda()
    (y * gy).sum().backward()
    out["f32_y"] = y.detach().cpu().numpy()
    out["f32_gx"] = xd.grad.cpu().numpy()
    out["f32_gw"] = Wd.grad.cpu().numpy()
    ctx.synchronize()
    ctx.close()
    return out
