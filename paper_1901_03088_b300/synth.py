"""Seeded synthetic H&E-like images: the inputs of the tests and the benchmark.

The paper's images (TCGA slides, §4.1) are not available, so every input is
generated from a stated staining model; nothing here is part of the method.
The model is Beer-Lambert absorption by two stains:

* stain basis W (3 x 2): the Ruifrok-Johnston hematoxylin and eosin OD vectors
  with N(0, 0.05) added to each entry, clipped at 0.01, columns renormalised;
* 30% background pixels (no stain); in tissue one stain dominates (chosen with
  probability 1/2): h_dom ~ Gamma(2, scale 0.4), h_other ~ Gamma(0.5, scale 0.1);
* pixel = clip(round(white * exp(-W h) + N(0, 2)), 0, 255) per channel;
* large images add smooth blobs: a Gaussian-filtered noise field (sigma = 64
  px, built at 1/16 resolution and bilinearly upsampled); background is where
  the field is below its 30% quantile and the field multiplies h by
  (0.5 + field).

``make_image`` (numpy, CPU) serves small cases and the oracle's own tests;
``make_image_torch`` builds large images band by band with torch on any device
(the 8-gigapixel slide is generated directly in device memory).  The two use
different random streams; each is deterministic for its seed.
"""
from __future__ import annotations

import math

import numpy as np

RUIFROK_HE = np.array([[0.650, 0.072],
                       [0.704, 0.990],
                       [0.286, 0.105]], dtype=np.float64)

BLOB_SIGMA = 64.0
BLOB_DOWN = 16
BACKGROUND_FRACTION = 0.3


def stain_basis(seed: int, jitter: float = 0.05) -> np.ndarray:
    """Seeded 3x2 column-normalised stain basis near H&E hues."""
    rng = np.random.default_rng(seed)
    W = RUIFROK_HE + rng.normal(0.0, jitter, size=(3, 2))
    W = np.maximum(W, 0.01)
    return W / np.linalg.norm(W, axis=0, keepdims=True)


def _densities_np(rng, n, background, pure=False):
    bg = rng.random(n) < background
    dom = rng.random(n) < 0.5
    h_dom = rng.gamma(2.0, 0.4, size=n)
    h_oth = np.zeros(n) if pure else rng.gamma(0.5, 0.1, size=n)
    H = np.empty((2, n))
    H[0] = np.where(dom, h_dom, h_oth)
    H[1] = np.where(dom, h_oth, h_dom)
    H[:, bg] = 0.0
    return H


def _blob_field_np(rng, height, width):
    from scipy.ndimage import gaussian_filter
    hl = height // BLOB_DOWN + 2
    wl = width // BLOB_DOWN + 2
    f = gaussian_filter(rng.normal(size=(hl, wl)), BLOB_SIGMA / BLOB_DOWN, mode="wrap")
    f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
    gy = np.arange(height) / BLOB_DOWN
    gx = np.arange(width) / BLOB_DOWN
    y0 = np.floor(gy).astype(int)
    x0 = np.floor(gx).astype(int)
    ty = (gy - y0)[:, None]
    tx = (gx - x0)[None, :]
    f00 = f[y0][:, x0]
    f01 = f[y0][:, x0 + 1]
    f10 = f[y0 + 1][:, x0]
    f11 = f[y0 + 1][:, x0 + 1]
    up = (f00 * (1 - tx) + f01 * tx) * (1 - ty) + (f10 * (1 - tx) + f11 * tx) * ty
    return up, float(np.quantile(f, BACKGROUND_FRACTION))


def make_image(height: int, width: int, seed: int, W=None, blobs: bool = False,
               background: float = BACKGROUND_FRACTION, white=(255.0, 255.0, 255.0),
               noise: float = 2.0, pure: bool = False, as_float: bool = False):
    """Seeded H x W x 3 synthetic image (uint8 unless ``as_float``)."""
    rng = np.random.default_rng(seed)
    W = stain_basis(seed) if W is None else np.asarray(W, dtype=np.float64)
    n = height * width
    if blobs:
        field, q = _blob_field_np(rng, height, width)
        H = _densities_np(rng, n, 0.0, pure)
        H = H * (0.5 + field.reshape(1, -1))
        H[:, (field < q).reshape(-1)] = 0.0
    else:
        H = _densities_np(rng, n, background, pure)
    I = np.asarray(white, dtype=np.float64)[:, None] * np.exp(-(W @ H))
    if noise > 0:
        I = I + rng.normal(0.0, noise, size=I.shape)
    I = np.ascontiguousarray(I.T.reshape(height, width, 3))
    if as_float:
        return np.clip(I, 0.0, 255.0)
    return np.ascontiguousarray(np.clip(np.rint(I), 0, 255).astype(np.uint8))


# ---------------------------------------------------------------------------
# Band-wise generator in torch (any device) for images too large for numpy.
# ---------------------------------------------------------------------------
def _gauss_kernel_1d(torch, sigma, device):
    r = int(math.ceil(3 * sigma))
    x = torch.arange(-r, r + 1, dtype=torch.float32, device=device)
    k = torch.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum(), r


def _blob_field_torch(torch, gen, height, width, device):
    import torch.nn.functional as F
    hl = height // BLOB_DOWN + 2
    wl = width // BLOB_DOWN + 2
    f = torch.randn((1, 1, hl, wl), generator=gen, device=device)
    k, r = _gauss_kernel_1d(torch, BLOB_SIGMA / BLOB_DOWN, device)
    f = F.pad(f, (r, r, 0, 0), mode="circular")
    f = F.conv2d(f, k.view(1, 1, 1, -1))
    f = F.pad(f, (0, 0, r, r), mode="circular")
    f = F.conv2d(f, k.view(1, 1, -1, 1))[0, 0]
    f = (f - f.min()) / torch.clamp(f.max() - f.min(), min=1e-12)
    flat = f.flatten()
    if flat.numel() > 16_000_000:  # quantile on a strided subset (exact enough)
        flat = flat[:: flat.numel() // 16_000_000 + 1]
    q = torch.quantile(flat.float(), BACKGROUND_FRACTION).item()
    return f, q


def make_image_torch(height: int, width: int, seed: int, W=None, device="cpu",
                     blobs: bool = True, out=None, band_rows: int = 1024,
                     white=(255.0, 255.0, 255.0), noise: float = 2.0,
                     background: float = BACKGROUND_FRACTION):
    """Seeded H x W x 3 uint8 torch image built band by band on ``device``.

    ``out`` may be a preallocated (H, W, 3) uint8 tensor (or a view with a row
    pitch) to fill in place."""
    import torch
    W = stain_basis(seed) if W is None else np.asarray(W, dtype=np.float64)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    if out is None:
        out = torch.empty((height, width, 3), dtype=torch.uint8, device=device)
    Wt = torch.tensor(W, dtype=torch.float32, device=device)
    wt = torch.tensor(white, dtype=torch.float32, device=device).view(1, 1, 3)
    if blobs:
        field, q = _blob_field_torch(torch, gen, height, width, device)
        gx = torch.arange(width, device=device, dtype=torch.float32) / BLOB_DOWN
        x0 = torch.floor(gx).long()
        tx = (gx - x0.float()).view(1, -1)
    for r0 in range(0, height, band_rows):
        r1 = min(height, r0 + band_rows)
        nb = r1 - r0
        u1 = torch.rand((nb, width), generator=gen, device=device).clamp_(min=1e-12)
        u2 = torch.rand((nb, width), generator=gen, device=device).clamp_(min=1e-12)
        h_dom = -0.4 * (torch.log(u1) + torch.log(u2))            # Gamma(2, 0.4)
        z = torch.randn((nb, width), generator=gen, device=device)
        h_oth = 0.1 * 0.5 * z * z                                   # Gamma(0.5, 0.1)
        dom = torch.rand((nb, width), generator=gen, device=device) < 0.5
        h1 = torch.where(dom, h_dom, h_oth)
        h2 = torch.where(dom, h_oth, h_dom)
        del u1, u2, h_dom, z, h_oth, dom
        if blobs:
            gy = torch.arange(r0, r1, device=device, dtype=torch.float32) / BLOB_DOWN
            y0 = torch.floor(gy).long()
            ty = (gy - y0.float()).view(-1, 1)
            rows = field[y0] * (1 - ty) + field[y0 + 1] * ty       # nb x wl
            fb = rows[:, x0] * (1 - tx) + rows[:, x0 + 1] * tx      # nb x width
            del rows
            bg = fb < q
            scale = 0.5 + fb
            h1 = torch.where(bg, 0.0, h1 * scale)
            h2 = torch.where(bg, 0.0, h2 * scale)
            del fb, bg, scale
        else:
            bg = torch.rand((nb, width), generator=gen, device=device) < background
            h1 = torch.where(bg, 0.0, h1)
            h2 = torch.where(bg, 0.0, h2)
            del bg
        od = h1.unsqueeze(-1) * Wt[:, 0] + h2.unsqueeze(-1) * Wt[:, 1]   # nb x width x 3
        del h1, h2
        I = wt * torch.exp(-od)
        del od
        if noise > 0:
            I += noise * torch.randn(I.shape, generator=gen, device=device)
        out[r0:r1].copy_(torch.clamp(torch.round(I), 0, 255).to(torch.uint8))
        del I
    return out


def batch_layout(n_slides: int, per_slide: int, side_lo: int, side_hi: int, seed: int):
    """Tile sizes of a batch of uneven tiles: for each of ``n_slides`` slides,
    ``per_slide`` tiles whose width and height are drawn independently,
    log-uniformly in [side_lo, side_hi].  Returns (slide, height, width)
    triples, slide-major; slide s uses the basis ``stain_basis(2000 + s)``
    and tile k the image seed ``3000 + k``."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(side_lo), math.log(side_hi)
    out = []
    for s in range(n_slides):
        for _ in range(per_slide):
            h, w = (int(round(math.exp(rng.uniform(lo, hi)))) for _ in range(2))
            out.append((s, min(max(h, side_lo), side_hi), min(max(w, side_lo), side_hi)))
    return out
