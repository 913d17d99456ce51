"""FP64 CPU oracle for the improved structure-preserving colour normalisation
(SPCN) of Ramakrishnan, Anand & Sethi, "Fast GPU-Enabled Color Normalization
for Digital Pathology" (arXiv 1901.03088).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain definition that the
CUDA library is checked against.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does, and
it shares no code, table or constant generator with the CUDA sources.

Every step follows the paper's order and notation, in float64, with numpy as
the only arithmetic library (``np.sort`` for order statistics, elementwise
ufuncs for the per-pixel maps).  Nothing is blocked, fused or reordered.

Steps and the passages they follow:

* ``select_sample``     -- §3.1 item 2 and §3.2 item 2 (random non-white pixels
                           and non-background patches for the basis).
* ``estimate_i0``       -- §3.1 item 1 (<= 100,000 pixels brighter than 220,
                           80th percentile per channel).
* ``optical_density``   -- §2.1 Eq. 1 with the channel-wise i0 of §3.1 item 1.
* ``lasso2``            -- §2.1 Eq. 2, H-step for a fixed basis (non-negative
                           two-atom lasso, exact by active-set enumeration).
* ``snmf``              -- §2.1 Eq. 2, alternating minimisation over H and W.
* ``order_stains``      -- §3.1 item 3 (red-minus-blue ordering).
* ``percentile``        -- §2.1 Eq. 3's P99 and §3.1 item 1's P80.
* ``stain_percentile``  -- §3.1 item 2 (P99 over non-white pixels only).
* ``normalize``         -- §2.1 Eq. 3 and Eq. 4.
* ``normalize_grad``    -- derivative of Eq. 1-4 with respect to the input
                           intensities and the target basis (the percentile
                           scale, source basis and both i0 held fixed).

Readings where the paper is silent (each also listed in the design notes):

R1  "intensity above 220" means all three channels above 220 (bright);
    "non-white" is its complement (some channel <= 220).
R2  Percentiles are Hyndman-Fan type 7 ("linear").
R3  Eq. 2's squared Frobenius term carries a factor 1/2 (lambda = 0.1 refers
    to the 1/2-scaled problem).
R4  OD clamps the intensity at 1 (log(i0/0) is undefined); negative OD is kept.
R5  SNMF starts from the column-normalised Ruifrok-Johnston H&E vectors, runs a
    batch alternating minimisation (exact H-step, one exact block-coordinate
    pass over the two columns of W) and stops when max|dW| < tol or after
    max_iter iterations.
R6  Hematoxylin (column 0) is the column with the larger OD(red) - OD(blue).
R7  Eq. 3's P99 is exact over all non-white pixels of the image; if the
    source P99 of a stain is 0 its scale is 1.
R8  Eq. 4 uses the target's i0 (the background maps to the target's white).
R9  The i0 sample keeps every ceil(n/100000)-th bright sample pixel in
    sample order; with no bright pixel i0 = 255.
R10 Output rounding is round-half-even, clamped to [0, 255].
R11 Random choices use SplitMix64 outputs (Steele, Lea & Flood 2014) mapped
    to [0, n) by the multiply-high range reduction (Lemire 2019).

Variants of the paper's own earlier choices, each off by default (Params):

i0_fixed_255      §2.1 Eq. 1: i0 = 255 for every channel (the original method)
                  instead of §3.1 item 1's estimate.
order="blue"      §3.1 item 3's original heuristic, read as: hematoxylin is the
                  column with the larger blue optical density (R14).
p99_patch_median  §3.2 item 4: the reported P99 is, per stain, the median over
                  the kept patches of each patch's non-white P99 (patches
                  sampling only).
i0_out_255        Eq. 4 reconstructs with the neutral white 255 instead of the
                  target's i0 (the alternative to reading R8).
h_solve="pinv"    §2.1: H = pinv(W) v (unconstrained, may be negative) for the
                  densities that are scaled and reconstructed; the basis itself
                  is still learnt with Eq. 2.
Normalising with the P99 that ``estimate_basis`` reports (§3.1 item 2's
sub-sampled percentile) instead of the exact one is ``normalize`` called with
those statistics.

Parity pins (tests/test_oracle.py): OD(i0) = 0 and hand-computed OD values;
KKT conditions of every lasso solution; hand-solved lasso cases;
brute-force enumeration of the active sets and a grid search on tiny inputs;
soft-threshold closed form for orthogonal W; lambda = 0 against scipy's NNLS;
identity reconstruction; planted-basis recovery and permutation invariance;
objective monotonicity; percentile against ``np.percentile``; published
SplitMix64 output vectors and exact multiply-high against Python integers;
round-half-even of exact .5 values in ``to_uint8``; the analytic gradient
against central differences; each variant option (i0 = 255, blue-only
ordering, patch median, pseudo-inverse, i0_out_255) against its special
case; the swap and tinted-background regressions of §4.1.  End-to-end
quality on real stained slides is not pinned: the paper prints no worked
example and its images are not available.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Constants fixed by the paper
# --------------------------------------------------------------------------
LAMBDA = 0.1            # §2.1, sparsity weight of Eq. 2
WHITE_THRESH = 220      # §3.1 items 1-2
I0_PERCENTILE = 80.0    # §3.1 item 1
I0_MAX_SAMPLES = 100000  # §3.1 item 1
STAIN_PERCENTILE = 99.0  # §2.1 Eq. 3, §3.1 item 2

# Ruifrok & Johnston (2001) H&E optical-density vectors (R, G, B); only the
# starting point of the dictionary learning (reading R5).
RUIFROK_H = (0.650, 0.704, 0.286)
RUIFROK_E = (0.072, 0.990, 0.105)

U64 = np.uint64
MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


class SpcnError(RuntimeError):
    """Raised where the method has no defined result (no tissue, degenerate
    basis, invalid argument)."""

    def __init__(self, kind: str, msg: str):
        super().__init__(f"{kind}: {msg}")
        self.kind = kind


@dataclass
class Params:
    lam: float = LAMBDA
    white_thresh: int = WHITE_THRESH
    i0_pct: float = I0_PERCENTILE
    stain_pct: float = STAIN_PERCENTILE
    i0_max_samples: int = I0_MAX_SAMPLES
    sample_mode: str = "all"      # "all" | "hash" | "patches"
    sample_rate: float = 0.01
    n_patches: int = 200
    patch_size: int = 256
    max_iter: int = 200
    tol: float = 1e-6
    seed: int = 0
    i0_fixed_255: bool = False
    order: str = "red_blue"       # "red_blue" (§3.1 item 3) | "blue" (original)
    p99_patch_median: bool = False
    h_solve: str = "lasso"        # "lasso" (Eq. 2) | "pinv" (§2.1)


@dataclass
class Stats:
    W: np.ndarray                 # 3x2, column 0 = hematoxylin
    i0: np.ndarray                # (3,)
    p99: np.ndarray               # (2,)
    iters: int = 0
    objective: list = field(default_factory=list)
    n_sample: int = 0
    n_nonwhite: int = 0
    n_bright: int = 0


# --------------------------------------------------------------------------
# Counter-based randomness (reading R11)
# --------------------------------------------------------------------------
def mix64(z):
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=U64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> U64(30))) * U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> U64(27))) * U64(0x94D049BB133111EB)
        z = z ^ (z >> U64(31))
    return z


def splitmix64(seed: int, n):
    """The n-th (0-based) output of a SplitMix64 generator whose state starts
    at ``seed``: mix64(seed + (n + 1) * gamma) modulo 2**64."""
    n = np.asarray(n, dtype=U64)
    with np.errstate(over="ignore"):
        state = U64(seed & MASK64) + (n + U64(1)) * U64(GOLDEN_GAMMA)
    return mix64(state)


def mulhi64(a, b: int):
    """floor(a * b / 2**64) for uint64 array a and 0 <= b < 2**63, exactly,
    using 32-bit limbs."""
    a = np.asarray(a, dtype=U64)
    m32 = U64(0xFFFFFFFF)
    b = int(b)
    b_lo, b_hi = U64(b & 0xFFFFFFFF), U64(b >> 32)
    a_lo, a_hi = a & m32, a >> U64(32)
    with np.errstate(over="ignore"):
        ll = a_lo * b_lo
        lh = a_lo * b_hi
        hl = a_hi * b_lo
        hh = a_hi * b_hi
        mid = (ll >> U64(32)) + (lh & m32) + (hl & m32)
        return hh + (lh >> U64(32)) + (hl >> U64(32)) + (mid >> U64(32))


def rand_below(seed: int, n, bound: int):
    """Map SplitMix64 output n into [0, bound) by multiply-high."""
    return mulhi64(splitmix64(seed, n), bound)


# --------------------------------------------------------------------------
# Pixel classes (reading R1)
# --------------------------------------------------------------------------
def bright_mask(rgb: np.ndarray, thresh: int = WHITE_THRESH) -> np.ndarray:
    """§3.1 item 1: pixels with intensity above the threshold (all channels)."""
    return np.all(rgb.astype(np.int64) > thresh, axis=-1)


def nonwhite_mask(rgb: np.ndarray, thresh: int = WHITE_THRESH) -> np.ndarray:
    """§3.1 item 2: non-white pixels, the complement of ``bright_mask``."""
    return ~bright_mask(rgb, thresh)


# --------------------------------------------------------------------------
# Percentile (reading R2)
# --------------------------------------------------------------------------
def percentile(values, p: float) -> float:
    """Type-7 percentile of a 1-D array: sort ascending, take the element at
    position p/100 * (n - 1) with linear interpolation between neighbours."""
    a = np.sort(np.asarray(values, dtype=np.float64).ravel())
    n = a.size
    if n == 0:
        raise SpcnError("INVALID_ARG", "percentile of an empty set")
    pos = (n - 1) * (p / 100.0)
    k = int(math.floor(pos))
    t = pos - k
    if k + 1 >= n:
        return float(a[n - 1])
    lo, hi = float(a[k]), float(a[k + 1])
    return lo + t * (hi - lo)


def percentile_ranks(n: int, p: float):
    """(k, t): the 0-based lower rank and the interpolation weight used by
    ``percentile`` for n values."""
    pos = (n - 1) * (p / 100.0)
    k = int(math.floor(pos))
    return k, pos - k


# --------------------------------------------------------------------------
# Sampling for the basis and for i0 (§3.1 items 1-2, §3.2 item 2)
# --------------------------------------------------------------------------
def patch_origins(width: int, height: int, params: Params):
    """Candidate patch origins k = 0 .. 4*n_patches-1 (top-left corners)."""
    P = params.patch_size
    if P > width or P > height:
        raise SpcnError("INVALID_ARG", "patch larger than the image")
    k = np.arange(4 * params.n_patches, dtype=np.uint64)
    x0 = rand_below(params.seed, U64(2) * k, width - P + 1).astype(np.int64)
    y0 = rand_below(params.seed, U64(2) * k + U64(1), height - P + 1).astype(np.int64)
    return x0, y0


def select_sample(img: np.ndarray, params: Params) -> np.ndarray:
    """Sample pixels (n x 3 uint8, in sample order) from which i0 and the basis
    are estimated.

    * ``all``:     every pixel in raster order.
    * ``hash``:    m = round(rate * N) draws with replacement; draw k is pixel
                   rand_below(seed, k, N) of the raster order.
    * ``patches``: candidate P x P patches (see ``patch_origins``) are kept in
                   candidate order while at least half of their pixels are
                   non-white, up to n_patches; the sample is the kept patches'
                   pixels, patch after patch, raster order inside a patch.
    """
    h, w, _ = img.shape
    flat = img.reshape(-1, 3)
    mode = params.sample_mode
    if mode == "all":
        return flat.copy()
    if mode == "hash":
        n = h * w
        m = int(math.floor(params.sample_rate * n + 0.5))
        if m <= 0:
            raise SpcnError("INVALID_ARG", "empty hash sample")
        idx = rand_below(params.seed, np.arange(m, dtype=np.uint64), n).astype(np.int64)
        return flat[idx]
    if mode == "patches":
        return np.concatenate(select_patches(img, params), axis=0)
    raise SpcnError("INVALID_ARG", f"unknown sample mode {mode!r}")


def select_patches(img: np.ndarray, params: Params) -> list:
    """The kept patches of the ``patches`` sample, each P*P x 3 in raster
    order, in candidate order."""
    h, w, _ = img.shape
    P = params.patch_size
    x0, y0 = patch_origins(w, h, params)
    kept = []
    for k in range(x0.size):
        patch = img[y0[k]:y0[k] + P, x0[k]:x0[k] + P]
        nw = int(np.count_nonzero(nonwhite_mask(patch, params.white_thresh)))
        if 2 * nw >= P * P:
            kept.append(patch.reshape(-1, 3))
            if len(kept) == params.n_patches:
                break
    if not kept:
        raise SpcnError("NO_TISSUE", "no patch is at least half non-white")
    return kept


def estimate_i0(sample: np.ndarray, params: Params) -> np.ndarray:
    """§3.1 item 1: per channel, the 80th percentile of at most 100,000 sample
    pixels brighter than the threshold (reading R9 for the cap).  With
    ``i0_fixed_255``, §2.1's original i0 = 255."""
    if params.i0_fixed_255:
        return np.full(3, 255.0)
    bright = sample[bright_mask(sample, params.white_thresh)]
    nb = bright.shape[0]
    if nb == 0:
        return np.full(3, 255.0)
    cap = params.i0_max_samples
    stride = (nb + cap - 1) // cap
    kept = bright[::stride].astype(np.float64)
    return np.array([percentile(kept[:, c], params.i0_pct) for c in range(3)])


# --------------------------------------------------------------------------
# Eq. 1 -- optical density
# --------------------------------------------------------------------------
def optical_density(rgb: np.ndarray, i0) -> np.ndarray:
    """§2.1 Eq. 1 with i0 per channel (§3.1 item 1): v = log(i0 / i), the
    intensity clamped at 1 (reading R4).  rgb: (..., 3) -> (..., 3) float64."""
    i = np.maximum(np.asarray(rgb, dtype=np.float64), 1.0)
    return np.log(np.asarray(i0, dtype=np.float64) / i)


# --------------------------------------------------------------------------
# Eq. 2 -- H-step: the non-negative two-atom lasso
# --------------------------------------------------------------------------
def gram(W: np.ndarray):
    G = W.T @ W
    det = G[0, 0] * G[1, 1] - G[0, 1] * G[1, 0]
    if not det > 1e-12:
        raise SpcnError("DEGENERATE_BASIS", "stain vectors are (nearly) parallel")
    return G, det


def lasso2(V: np.ndarray, W: np.ndarray, lam: float) -> np.ndarray:
    """For every column v of V (3 x n), the exact minimiser over h >= 0 of
    1/2 ||v - W h||^2 + lam (h1 + h2), i.e. 1/2 h'Gh - c'h + lam 1'h with
    G = W'W, c = W'v.  The objective is strictly convex, so exactly one of the
    four active sets satisfies the KKT conditions; they are checked in the
    order {1,2}, {1}, {2}, {} and the first that holds is taken."""
    G, det = gram(W)
    C = W.T @ V                        # 2 x n
    d1 = C[0] - lam
    d2 = C[1] - lam
    # both stains active: G h = d
    hb1 = (G[1, 1] * d1 - G[0, 1] * d2) / det
    hb2 = (G[0, 0] * d2 - G[1, 0] * d1) / det
    both = (hb1 > 0) & (hb2 > 0)
    # only stain 1: h1 = d1/G11 > 0 and the stain-2 gradient G21 h1 - d2 >= 0
    a1 = d1 / G[0, 0]
    one1 = (a1 > 0) & (G[1, 0] * a1 - d2 >= 0)
    # only stain 2
    a2 = d2 / G[1, 1]
    one2 = (a2 > 0) & (G[0, 1] * a2 - d1 >= 0)
    H = np.zeros((2, V.shape[1]))
    sel1 = ~both & one1
    sel2 = ~both & ~one1 & one2
    H[0] = np.where(both, hb1, np.where(sel1, a1, 0.0))
    H[1] = np.where(both, hb2, np.where(sel2, a2, 0.0))
    return H


def pinv_densities(V: np.ndarray, W: np.ndarray) -> np.ndarray:
    """§2.1: H = pinv(W) V, the least-squares densities without sign or
    sparsity constraint (2 x n)."""
    gram(W)
    return np.linalg.pinv(np.asarray(W, dtype=np.float64)) @ V


def solve_h(V: np.ndarray, W: np.ndarray, params: "Params") -> np.ndarray:
    """The densities that are scaled and reconstructed: Eq. 2's lasso, or the
    pseudo-inverse variant."""
    if params.h_solve == "pinv":
        return pinv_densities(V, W)
    if params.h_solve != "lasso":
        raise SpcnError("INVALID_ARG", f"unknown H solve {params.h_solve!r}")
    return lasso2(V, W, params.lam)


def lasso_objective(V: np.ndarray, W: np.ndarray, H: np.ndarray, lam: float) -> float:
    """Eq. 2 with the 1/2 of reading R3."""
    R = V - W @ H
    return 0.5 * float(np.sum(R * R)) + lam * float(np.sum(H))


# --------------------------------------------------------------------------
# Eq. 2 -- dictionary learning of W
# --------------------------------------------------------------------------
def ruifrok_init() -> np.ndarray:
    W = np.array([RUIFROK_H, RUIFROK_E], dtype=np.float64).T
    return W / np.linalg.norm(W, axis=0, keepdims=True)


def snmf(V: np.ndarray, lam: float, max_iter: int, tol: float, W0=None):
    """Alternating minimisation of Eq. 2 (reading R5).

    Each iteration: H = lasso2(V, W) (exact); A = H H', B = V H'; then for
    j = 1, 2 in turn u = w_j + (b_j - W a_j) / A_jj, w_j = max(u,0)/||max(u,0)||
    (skipped when A_jj = 0).  With ||w_j|| = 1 this is the exact minimiser of
    Eq. 2 over column j on the feasible set, so the objective never rises.
    Returns (W, iterations, objective after each H-step)."""
    W = ruifrok_init() if W0 is None else np.array(W0, dtype=np.float64)
    objective = []
    it = 0
    for it in range(1, max_iter + 1):
        H = lasso2(V, W, lam)
        objective.append(lasso_objective(V, W, H, lam))
        A = H @ H.T
        B = V @ H.T
        W_prev = W.copy()
        for j in range(2):
            if A[j, j] <= 0:
                continue
            u = W[:, j] + (B[:, j] - W @ A[:, j]) / A[j, j]
            u = np.maximum(u, 0.0)
            nu = np.linalg.norm(u)
            if nu == 0:
                raise SpcnError("DEGENERATE_BASIS", "a stain column vanished")
            W[:, j] = u / nu
        gram(W)
        if np.max(np.abs(W - W_prev)) < tol:
            break
    return W, it, objective


def order_stains(W: np.ndarray, rule: str = "red_blue") -> np.ndarray:
    """§3.1 item 3 (reading R6): column 0 is hematoxylin, the stain whose OD
    red minus OD blue is larger; ties keep the order.  rule="blue" is the
    original heuristic the paper replaces (reading R14): the column with the
    larger blue OD is hematoxylin."""
    if rule == "red_blue":
        d0 = W[0, 0] - W[2, 0]
        d1 = W[0, 1] - W[2, 1]
    elif rule == "blue":
        d0, d1 = W[2, 0], W[2, 1]
    else:
        raise SpcnError("INVALID_ARG", f"unknown ordering rule {rule!r}")
    return W[:, ::-1].copy() if d1 > d0 else W.copy()


# --------------------------------------------------------------------------
# Basis estimation (§3.1, §3.2)
# --------------------------------------------------------------------------
def estimate_basis(img: np.ndarray, params: Params | None = None) -> Stats:
    """Sample -> i0 -> OD -> SNMF -> ordering -> P99 of the sampled non-white
    pixels' densities (§3.1 item 2's sub-sampled percentile), or with
    ``p99_patch_median`` the median over the kept patches of each patch's
    non-white P99 (§3.2 item 4)."""
    params = params or Params()
    if params.p99_patch_median and params.sample_mode != "patches":
        raise SpcnError("INVALID_ARG", "the patch median needs patches sampling")
    sample = select_sample(img, params)
    i0 = estimate_i0(sample, params)
    nw = sample[nonwhite_mask(sample, params.white_thresh)]
    if nw.shape[0] == 0:
        raise SpcnError("NO_TISSUE", "no non-white sample pixel")
    V = optical_density(nw, i0).T                       # 3 x m
    W, iters, obj = snmf(V, params.lam, params.max_iter, params.tol)
    W = order_stains(W, params.order)
    if params.p99_patch_median:
        per_patch = []
        for patch in select_patches(img, params):
            pnw = patch[nonwhite_mask(patch, params.white_thresh)]
            Hp = solve_h(optical_density(pnw, i0).T, W, params)
            per_patch.append([percentile(Hp[j], params.stain_pct) for j in range(2)])
        per_patch = np.array(per_patch)
        p99 = np.array([percentile(per_patch[:, j], 50.0) for j in range(2)])
    else:
        H = solve_h(V, W, params)
        p99 = np.array([percentile(H[j], params.stain_pct) for j in range(2)])
    return Stats(W=W, i0=i0, p99=p99, iters=iters, objective=obj,
                 n_sample=sample.shape[0], n_nonwhite=nw.shape[0],
                 n_bright=int(np.count_nonzero(bright_mask(sample, params.white_thresh))))


# --------------------------------------------------------------------------
# Full-image stain densities and their percentile
# --------------------------------------------------------------------------
def stain_densities(img: np.ndarray, W, i0, lam: float = LAMBDA,
                    h_solve: str = "lasso") -> np.ndarray:
    """H (2 x N, raster order) of every pixel for a given basis and i0."""
    V = optical_density(img.reshape(-1, 3), i0).T
    W = np.asarray(W, dtype=np.float64)
    return pinv_densities(V, W) if h_solve == "pinv" else lasso2(V, W, lam)


def stain_percentile(img: np.ndarray, W, i0, params: Params | None = None,
                     H: np.ndarray | None = None) -> np.ndarray:
    """§2.1 Eq. 3's P99 per stain, over the non-white pixels of the whole
    image (§3.1 item 2; reading R7)."""
    params = params or Params()
    if H is None:
        H = stain_densities(img, W, i0, params.lam, params.h_solve)
    nw = nonwhite_mask(img.reshape(-1, 3), params.white_thresh)
    if not np.any(nw):
        raise SpcnError("NO_TISSUE", "no non-white pixel")
    return np.array([percentile(H[j][nw], params.stain_pct) for j in range(2)])


def stain_scale(p99_src, p99_tgt) -> np.ndarray:
    """Eq. 3's per-stain factor P99(H_target) / P99(H_source); 1 where the
    source percentile is 0 (reading R7)."""
    s = np.ones(2)
    for j in range(2):
        if p99_src[j] != 0:
            s[j] = p99_tgt[j] / p99_src[j]
    return s


def normalize_float(img: np.ndarray, src_W, src_i0, src_p99, tgt_W, tgt_i0,
                    tgt_p99, lam: float = LAMBDA, h_solve: str = "lasso",
                    i0_out_255: bool = False) -> np.ndarray:
    """Eq. 3 then Eq. 4 (reading R8) for every pixel; H x W x 3 float64.
    With i0_out_255 Eq. 4 uses 255 for every channel instead of tgt_i0."""
    if i0_out_255:
        tgt_i0 = np.full(3, 255.0)
    h, w, _ = img.shape
    H = stain_densities(img, src_W, src_i0, lam, h_solve)
    s = stain_scale(src_p99, tgt_p99)
    Vn = np.asarray(tgt_W, dtype=np.float64) @ (s[:, None] * H)   # 3 x N
    I = np.asarray(tgt_i0, dtype=np.float64)[:, None] * np.exp(-Vn)
    return I.T.reshape(h, w, 3)


def to_uint8(I: np.ndarray) -> np.ndarray:
    """Reading R10: round half to even, clamp to [0, 255]."""
    return np.clip(np.rint(I), 0, 255).astype(np.uint8)


def normalize(img: np.ndarray, src: Stats, tgt: Stats, lam: float = LAMBDA,
              h_solve: str = "lasso", i0_out_255: bool = False) -> np.ndarray:
    """The full per-pixel path on a uint8 image with the source's P99 as
    src.p99 holds it (the exact one for the method; the sampled one of
    ``estimate_basis`` for the one-pass variant) and the target's
    statistics."""
    return to_uint8(normalize_float(img, src.W, src.i0, src.p99,
                                    tgt.W, tgt.i0, tgt.p99, lam, h_solve, i0_out_255))


def full_stats(img: np.ndarray, params: Params | None = None) -> Stats:
    """Basis and i0 from the sample, then the exact whole-image P99."""
    params = params or Params()
    st = estimate_basis(img, params)
    st.p99 = stain_percentile(img, st.W, st.i0, params)
    return st


# --------------------------------------------------------------------------
# Derivative of Eq. 1-4 (float intensities; percentile scale held fixed)
# --------------------------------------------------------------------------
def normalize_float_pixels(X: np.ndarray, src_W, src_i0, scale, tgt_W, tgt_i0,
                           lam: float = LAMBDA):
    """Eq. 1-4 on a 3 x N array of float intensities with a given per-stain
    scale (Eq. 3's percentile ratio).  Returns (Y, H), both float64."""
    V = optical_density(X.T, src_i0).T
    H = lasso2(V, np.asarray(src_W, dtype=np.float64), lam)
    Vn = np.asarray(tgt_W, dtype=np.float64) @ (np.asarray(scale, dtype=np.float64)[:, None] * H)
    Y = np.asarray(tgt_i0, dtype=np.float64)[:, None] * np.exp(-Vn)
    return Y, H


def normalize_grad(X: np.ndarray, GY: np.ndarray, src_W, src_i0, scale, tgt_W, tgt_i0,
                   lam: float = LAMBDA):
    """Gradient of L = sum(GY * Y) for Y = normalize_float_pixels(X, ...).

    Chain of Eq. 4, Eq. 3, the lasso of Eq. 2 and Eq. 1:
      dY_c/dV'_c = -Y_c;  dV'_c/dh_j = Wt[c,j] s_j;  dV'_c/dWt[c,j] = s_j h_j;
      on the active set A of each pixel h_A = G_AA^-1 (c_A - lambda), so
      dh_A/dc_A = G_AA^-1 and inactive densities have zero derivative;
      dc_j/dv_c = Ws[c,j];  dv_c/dx_c = -1/x_c where x_c > 1 (0 where Eq. 1's
      clamp at 1 is active).
    Returns (dL/dX (3 x N), dL/dWt (3 x 2))."""
    Ws = np.asarray(src_W, dtype=np.float64)
    Wt = np.asarray(tgt_W, dtype=np.float64)
    s = np.asarray(scale, dtype=np.float64)
    Y, H = normalize_float_pixels(X, Ws, src_i0, s, Wt, tgt_i0, lam)
    GV = -GY * Y                                   # dL/dV'
    gWt = (GV @ (s[:, None] * H).T)                # 3 x 2
    GH = s[:, None] * (Wt.T @ GV)                  # 2 x N
    G, det = gram(Ws)
    a1, a2 = H[0] > 0, H[1] > 0
    GC = np.zeros_like(GH)
    both = a1 & a2
    Ginv = np.array([[G[1, 1], -G[0, 1]], [-G[1, 0], G[0, 0]]]) / det
    GC[:, both] = Ginv @ GH[:, both]
    only1 = a1 & ~a2
    GC[0, only1] = GH[0, only1] / G[0, 0]
    only2 = a2 & ~a1
    GC[1, only2] = GH[1, only2] / G[1, 1]
    GVs = Ws @ GC                                  # dL/dv
    Xf = np.asarray(X, dtype=np.float64)
    GX = np.where(Xf > 1.0, -GVs / np.maximum(Xf, 1.0), 0.0)
    return GX, gWt
