"""Python binding of the SPCN C ABI (include/spcn.h) over ctypes.

Argument marshalling only: every step of the method runs in the CUDA library
``libspcn.so`` built beside this file.  Torch tensors supply device memory and
the current CUDA stream.  If the library is missing this module raises at
import time; there is no other implementation to fall back on.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SPCN_LIBRARY=checked selects the bounds-checked build (device index checks
# that report SPCN_ERR_INVALID_ARG); the default is the normal build.
LIB_PATH = os.path.join(HERE, "libspcn_checked.so" if os.environ.get("SPCN_LIBRARY") == "checked"
                        else "libspcn.so")

SPCN_OK = 0
STATUS_NAMES = {
    0: "OK", -1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "NO_TISSUE",
    -5: "DEGENERATE_BASIS", -6: "TIMEOUT", -7: "SCRATCH_LIMIT",
}
SAMPLE_MODES = {"all": 0, "hash": 1, "patches": 2}

# spcn_params.flags bits (include/spcn.h): the paper's earlier choices
FLAG_I0_255 = 0x1
FLAG_ORDER_BLUE = 0x2
FLAG_P99_SAMPLED = 0x4
FLAG_P99_PATCH_MEDIAN = 0x8
FLAG_H_PINV = 0x10
FLAG_I0_OUT_255 = 0x20


class SpcnError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.kind = STATUS_NAMES.get(status, str(status))
        msg = _lib.spcn_strerror(status).decode() if _lib is not None else self.kind
        super().__init__(f"{where}: {self.kind} ({msg})")


class Image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("pitch_bytes", ctypes.c_int64)]


class Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_float), ("white_thresh", ctypes.c_int32),
                ("i0_pct", ctypes.c_float), ("stain_pct", ctypes.c_float),
                ("i0_max_samples", ctypes.c_int32), ("sample_mode", ctypes.c_int32),
                ("sample_rate", ctypes.c_float), ("n_patches", ctypes.c_int32),
                ("patch_size", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("tol", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("W", ctypes.c_float * 6), ("i0", ctypes.c_float * 3),
                ("p99", ctypes.c_double * 2), ("iters", ctypes.c_int32),
                ("status", ctypes.c_int32), ("n_sample", ctypes.c_int64),
                ("n_nonwhite", ctypes.c_int64), ("n_bright", ctypes.c_int64),
                ("objective", ctypes.c_double)]

    @property
    def basis(self):
        """W as a 3x2 nested list (rows R, G, B; columns hematoxylin, eosin)."""
        return [[self.W[c], self.W[3 + c]] for c in range(3)]

    @staticmethod
    def from_values(W, i0, p99=(0.0, 0.0)) -> "Stats":
        """Record from a 3x2 basis (rows R,G,B), i0 (3) and p99 (2)."""
        s = Stats()
        for c in range(3):
            s.W[c] = float(W[c][0])
            s.W[3 + c] = float(W[c][1])
            s.i0[c] = float(i0[c])
        s.p99[0], s.p99[1] = float(p99[0]), float(p99[1])
        return s

    def copy(self) -> "Stats":
        s = Stats()
        ctypes.memmove(ctypes.byref(s), ctypes.byref(self), ctypes.sizeof(Stats))
        return s


class BatchConfig(ctypes.Structure):
    _fields_ = [("item_chunks", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("group_px", ctypes.c_int64), ("ms", ctypes.c_float), ("pad", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"item_chunks": int(self.item_chunks),
                "schedule": SCHEDULES_INV.get(int(self.schedule), int(self.schedule)),
                "group_px": int(self.group_px), "ms": float(self.ms)}


SCHEDULES = {"phased": 0, "interleaved": 1, "staged": 2, "persistent": 3}
SCHEDULES_INV = {v: k for k, v in SCHEDULES.items()}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1901_03088_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "spcn_params_default": (None, [P(Params)]),
        "spcn_context_create": (ctypes.c_int, [P(vp), ctypes.c_int]),
        "spcn_context_destroy": (ctypes.c_int, [vp]),
        "spcn_estimate_basis": (ctypes.c_int, [vp, P(Image), P(Params), P(Stats), vp]),
        "spcn_stain_percentile": (ctypes.c_int, [vp, P(Image), P(Stats), P(Params),
                                                 P(ctypes.c_double), vp]),
        "spcn_stain_densities": (ctypes.c_int, [vp, P(Image), P(Stats), P(Params), vp, i64, vp]),
        "spcn_stain_densities_estimated": (ctypes.c_int, [vp, P(Image), P(Params), vp, i64,
                                                          P(Stats), vp]),
        "spcn_normalize": (ctypes.c_int, [vp, P(Image), P(Stats), P(Stats), P(Params), vp, i64,
                                          P(ctypes.c_double), vp]),
        "spcn_normalize_estimated": (ctypes.c_int, [vp, P(Image), P(Stats), P(Params), vp, i64,
                                                    P(Stats), vp]),
        "spcn_synchronize": (ctypes.c_int, [vp, vp]),
        "spcn_launch_count": (i64, [vp]),
        "spcn_exact_fallbacks": (ctypes.c_int, [vp, P(i64)]),
        "spcn_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "spcn_debug_barrier_timeout": (ctypes.c_int, [vp, i32, i64, vp]),
        "spcn_kernel_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "spcn_estimate_basis_noalloc": (ctypes.c_int, [P(Image), P(Params), P(Stats), vp]),
        "spcn_normalize_f32": (ctypes.c_int, [vp, vp, i32, i32, i32, P(Stats), P(Stats), vp,
                                              P(Params), vp, vp]),
        "spcn_normalize_f32_backward": (ctypes.c_int, [vp, vp, vp, i32, i32, i32, P(Stats),
                                                       P(Stats), vp, P(Params), vp, vp, vp]),
        "spcn_kernel_times": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_double), P(i64)]),
        "spcn_batch_create": (ctypes.c_int, [vp, i32, P(Image), P(Stats), P(Stats), P(Params),
                                             P(vp), P(i64), P(vp)]),
        "spcn_batch_run": (ctypes.c_int, [vp, vp]),
        "spcn_batch_results": (ctypes.c_int, [vp, P(ctypes.c_double), P(i32), P(i32), vp]),
        "spcn_batch_get_config": (ctypes.c_int, [vp, P(BatchConfig)]),
        "spcn_batch_set_config": (ctypes.c_int, [vp, P(BatchConfig)]),
        "spcn_batch_tune": (ctypes.c_int, [vp, i32, P(BatchConfig), i32, P(i32), vp]),
        "spcn_batch_destroy": (ctypes.c_int, [vp]),
        "spcn_normalize_batched": (ctypes.c_int, [vp, i32, P(Image), P(Stats), P(Stats),
                                                  P(Params), P(vp), P(i64), P(ctypes.c_double),
                                                  P(i32), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None
_lib = _load()
lib = _lib

# Every name the header declares, for the export check.
EXPORTED = ("spcn_params_default", "spcn_context_create", "spcn_context_destroy",
            "spcn_estimate_basis", "spcn_stain_percentile", "spcn_stain_densities",
            "spcn_normalize", "spcn_normalize_estimated", "spcn_synchronize", "spcn_launch_count",
            "spcn_exact_fallbacks", "spcn_strerror",
            "spcn_debug_barrier_timeout", "spcn_kernel_timing", "spcn_kernel_times",
            "spcn_estimate_basis_noalloc", "spcn_normalize_f32", "spcn_normalize_f32_backward",
            "spcn_batch_create", "spcn_batch_run", "spcn_batch_results", "spcn_batch_get_config",
            "spcn_batch_set_config", "spcn_batch_tune", "spcn_batch_destroy",
            "spcn_normalize_batched", "spcn_stain_densities_estimated")
KERNELS = {"pass1": 0, "select": 1, "pass2": 2, "density": 3, "f32_fwd": 4, "f32_bwd": 5,
           "batch": 6, "ladder": 7}


def params(**kw) -> Params:
    """The paper's constants (spcn_params_default) with keyword overrides;
    ``lam`` sets lambda and ``sample_mode`` accepts 'all', 'hash', 'patches'."""
    p = Params()
    _lib.spcn_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("lam", "lambda_"):
            p.lambda_ = float(v)
        elif k == "sample_mode" and isinstance(v, str):
            p.sample_mode = SAMPLE_MODES[v]
        else:
            setattr(p, k, v)
    return p


def _check(rc: int, where: str):
    if rc != SPCN_OK:
        raise SpcnError(rc, where)


def image_of(t) -> Image:
    """spcn_image view of an (H, W, 3) uint8 CUDA tensor whose pixels are
    interleaved (channel stride 1, pixel stride 3); rows may be pitched."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.uint8 or t.dim() != 3 or t.shape[2] != 3:
        raise ValueError("expected an (H, W, 3) uint8 tensor")
    if not t.is_cuda:
        raise ValueError("image must be in device memory")
    if t.stride(2) != 1 or t.stride(1) != 3:
        raise ValueError("pixels must be interleaved RGB (strides (pitch, 3, 1))")
    return Image(t.data_ptr(), t.shape[1], t.shape[0], t.stride(0))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def estimate_basis_noalloc(img, p: Params | None = None, stream=None) -> Stats:
    """Basis estimation that allocates no device memory (for hosts that cannot
    call the CUDA allocator): same result as Context.estimate_basis, scratch
    from a fixed array inside the library, at most 524288 sample pixels.
    Runs on the current CUDA device; concurrent calls race."""
    st = Stats()
    im = image_of(img)
    p = p or params()
    rc = _lib.spcn_estimate_basis_noalloc(ctypes.byref(im), ctypes.byref(p), ctypes.byref(st),
                                          _stream(stream))
    _check(rc, "spcn_estimate_basis_noalloc")
    return st


class Context:
    """A library context on one CUDA device (owns the device scratch)."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(_lib.spcn_context_create(ctypes.byref(h), int(device)), "spcn_context_create")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            _lib.spcn_context_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def launches(self) -> int:
        return int(_lib.spcn_launch_count(self._h))

    @property
    def exact_fallbacks(self) -> int:
        """Whole-image percentiles resolved by the exact radix select (a rank
        outside pass 1's window) since the context was created."""
        n = ctypes.c_int64()
        _check(_lib.spcn_exact_fallbacks(self._h, ctypes.byref(n)), "spcn_exact_fallbacks")
        return int(n.value)

    def estimate_basis(self, img, p: Params | None = None, stream=None) -> Stats:
        st = Stats()
        im = image_of(img)
        p = p or params()
        rc = _lib.spcn_estimate_basis(self._h, ctypes.byref(im), ctypes.byref(p),
                                      ctypes.byref(st), _stream(stream))
        _check(rc, "spcn_estimate_basis")
        return st

    def stain_percentile(self, img, stats: Stats, p: Params | None = None, stream=None):
        out = (ctypes.c_double * 2)()
        im = image_of(img)
        p = p or params()
        rc = _lib.spcn_stain_percentile(self._h, ctypes.byref(im), ctypes.byref(stats),
                                        ctypes.byref(p), out, _stream(stream))
        _check(rc, "spcn_stain_percentile")
        return float(out[0]), float(out[1])

    def stain_densities(self, img, stats: Stats, p: Params | None = None, out=None, stream=None):
        import torch
        im = image_of(img)
        n = im.width * im.height
        if out is None:
            out = torch.empty((2, n), dtype=torch.float32, device=img.device)
        if out.dtype != torch.float32 or out.dim() != 2 or out.shape[0] != 2 or out.stride(1) != 1:
            raise ValueError("out must be a (2, >=H*W) float32 tensor with unit inner stride")
        p = p or params()
        rc = _lib.spcn_stain_densities(self._h, ctypes.byref(im), ctypes.byref(stats),
                                       ctypes.byref(p), ctypes.c_void_p(out.data_ptr()),
                                       out.stride(0), _stream(stream))
        _check(rc, "spcn_stain_densities")
        return out

    def stain_densities_estimated(self, img, p: Params | None = None, out=None,
                                  return_stats: bool = False, stream=None):
        """Basis estimation and the densities of every pixel in one call; with
        return_stats the call waits and also returns the estimated Stats."""
        import torch
        im = image_of(img)
        n = im.width * im.height
        if out is None:
            out = torch.empty((2, n), dtype=torch.float32, device=img.device)
        if out.dtype != torch.float32 or out.dim() != 2 or out.shape[0] != 2 or out.stride(1) != 1:
            raise ValueError("out must be a (2, >=H*W) float32 tensor with unit inner stride")
        p = p or params()
        st = Stats() if return_stats else None
        rc = _lib.spcn_stain_densities_estimated(self._h, ctypes.byref(im), ctypes.byref(p),
                                                 ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                                 ctypes.byref(st) if st is not None else None,
                                                 _stream(stream))
        _check(rc, "spcn_stain_densities_estimated")
        return (out, st) if return_stats else out

    def normalize(self, src, src_stats: Stats, tgt_stats: Stats, p: Params | None = None,
                  out=None, return_p99: bool = False, stream=None):
        import torch
        im = image_of(src)
        if out is None:
            out = torch.empty_like(src, memory_format=torch.contiguous_format)
        if out.shape != src.shape or out.dtype != torch.uint8 or out.stride(2) != 1 or out.stride(1) != 3:
            raise ValueError("out must be an (H, W, 3) uint8 interleaved tensor")
        p = p or params()
        p99 = (ctypes.c_double * 2)() if return_p99 else None
        rc = _lib.spcn_normalize(self._h, ctypes.byref(im), ctypes.byref(src_stats),
                                 ctypes.byref(tgt_stats), ctypes.byref(p),
                                 ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                 p99, _stream(stream))
        _check(rc, "spcn_normalize")
        if return_p99:
            return out, (float(p99[0]), float(p99[1]))
        return out

    def normalize_estimated(self, src, tgt_stats: Stats, p: Params | None = None, out=None,
                            return_stats: bool = False, stream=None):
        """Estimate the source's statistics and normalise it in one
        stream-ordered call (no host round trip in between).  With
        return_stats the call waits and also returns the source Stats (p99 =
        the exact percentile of the whole source)."""
        import torch
        im = image_of(src)
        if out is None:
            out = torch.empty_like(src, memory_format=torch.contiguous_format)
        if out.shape != src.shape or out.dtype != torch.uint8 or out.stride(2) != 1 or out.stride(1) != 3:
            raise ValueError("out must be an (H, W, 3) uint8 interleaved tensor")
        p = p or params()
        st = Stats() if return_stats else None
        rc = _lib.spcn_normalize_estimated(self._h, ctypes.byref(im), ctypes.byref(tgt_stats),
                                           ctypes.byref(p), ctypes.c_void_p(out.data_ptr()),
                                           out.stride(0), ctypes.byref(st) if st is not None else None,
                                           _stream(stream))
        _check(rc, "spcn_normalize_estimated")
        return (out, st) if return_stats else out

    def kernel_timing(self, enable: bool):
        """Start (and reset) or stop CUDA-event timing of the pixel kernels."""
        _check(_lib.spcn_kernel_timing(self._h, 1 if enable else 0), "spcn_kernel_timing")

    def kernel_times(self, name: str):
        """(total ms, launches) of a timed kernel: pass1, select, pass2, density."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(_lib.spcn_kernel_times(self._h, KERNELS[name], ctypes.byref(ms), ctypes.byref(n)),
               "spcn_kernel_times")
        return float(ms.value), int(n.value)

    def synchronize(self, stream=None):
        _check(_lib.spcn_synchronize(self._h, _stream(stream)), "spcn_synchronize")

    def debug_barrier_timeout(self, extra_arrivals: int, timeout_ns: int, stream=None) -> int:
        """Status of the failure-detection hook (see the header)."""
        return int(_lib.spcn_debug_barrier_timeout(self._h, int(extra_arrivals),
                                                   int(timeout_ns), _stream(stream)))


# ---------------------------------------------------------------------------
# Differentiable normalisation of float images
# ---------------------------------------------------------------------------
def stats_array(stats):
    """Contiguous C array of Stats records (build once, pass to normalize_f32)."""
    if isinstance(stats, ctypes.Array):
        return stats
    arr = (Stats * len(stats))()
    for i, st in enumerate(stats):
        ctypes.memmove(ctypes.byref(arr[i]), ctypes.byref(st), ctypes.sizeof(Stats))
    return arr


def _check_f32(x):
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and
            x.dim() == 4 and x.shape[1] == 3 and x.is_contiguous()):
        raise ValueError("expected a contiguous (B, 3, H, W) float32 CUDA tensor")


def _wt_colmajor(Wt):
    import torch
    if not (isinstance(Wt, torch.Tensor) and Wt.is_cuda and Wt.dtype == torch.float32 and
            tuple(Wt.shape) == (3, 2)):
        raise ValueError("W_target must be a (3, 2) float32 CUDA tensor (rows R, G, B)")
    return Wt.detach().t().contiguous()      # (2, 3): column-major 3x2


def _make_function():
    import torch

    class NormalizeF32(torch.autograd.Function):
        """y = Eq. 1-4 of x (no rounding); differentiable in x and W_target."""

        @staticmethod
        def forward(fctx, x, Wt, handle, src_arr, tgt, p):
            _check_f32(x)
            B, _, H, W = x.shape
            wt = _wt_colmajor(Wt)
            y = torch.empty_like(x)
            rc = _lib.spcn_normalize_f32(handle, ctypes.c_void_p(x.data_ptr()), B, H, W, src_arr,
                                         ctypes.byref(tgt), ctypes.c_void_p(wt.data_ptr()),
                                         ctypes.byref(p), ctypes.c_void_p(y.data_ptr()),
                                         _stream(None))
            _check(rc, "spcn_normalize_f32")
            fctx.save_for_backward(x, wt)
            fctx.handle, fctx.src_arr, fctx.tgt, fctx.p = handle, src_arr, tgt, p
            return y

        @staticmethod
        def backward(fctx, gy):
            x, wt = fctx.saved_tensors
            gy = gy.contiguous()
            B, _, H, W = x.shape
            gx = torch.empty_like(x)
            gwt = torch.empty(6, dtype=torch.float32, device=x.device)
            rc = _lib.spcn_normalize_f32_backward(
                fctx.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(gy.data_ptr()), B, H, W,
                fctx.src_arr, ctypes.byref(fctx.tgt), ctypes.c_void_p(wt.data_ptr()),
                ctypes.byref(fctx.p), ctypes.c_void_p(gx.data_ptr()),
                ctypes.c_void_p(gwt.data_ptr()), _stream(None))
            _check(rc, "spcn_normalize_f32_backward")
            return gx, gwt.view(2, 3).t(), None, None, None, None

    return NormalizeF32


_NormalizeF32Fn = None


def normalize_f32(ctx: "Context", x, W_target, src_stats, tgt_stats: Stats, p: Params | None = None):
    """Differentiable Eq. 1-4 for a (B, 3, H, W) float32 batch in [0, 255].

    src_stats: one Stats per image (W, i0 and the image's exact p99), as a
    list or as a prebuilt ``stats_array``.
    W_target: (3, 2) float32 CUDA tensor (rows R, G, B; may require grad);
    tgt_stats supplies the target i0 and p99.  Gradients flow to x and
    W_target; the percentile scale and source statistics are constants."""
    global _NormalizeF32Fn
    if _NormalizeF32Fn is None:
        _NormalizeF32Fn = _make_function()
    if len(src_stats) != x.shape[0]:
        raise ValueError("one source Stats per image")
    return _NormalizeF32Fn.apply(x, W_target, ctx.handle, stats_array(src_stats), tgt_stats,
                                 p or params())


# ---------------------------------------------------------------------------
# Batches: many tiles, one target, one persistent launch
# ---------------------------------------------------------------------------
def _batch_arrays(tiles, tile_stats, outs):
    n = len(tiles)
    if n < 1 or len(tile_stats) != n or len(outs) != n:
        raise ValueError("one source Stats and one output per tile")
    imgs = (Image * n)()
    out_p = (ctypes.c_void_p * n)()
    pitches = (ctypes.c_int64 * n)()
    for i, (t, o) in enumerate(zip(tiles, outs)):
        imgs[i] = image_of(t)
        if (tuple(o.shape) != tuple(t.shape) or o.dtype != t.dtype or o.stride(2) != 1 or
                o.stride(1) != 3 or not o.is_cuda):
            raise ValueError("each output must be an (H, W, 3) uint8 interleaved CUDA tensor "
                             "of its tile's size")
        out_p[i] = o.data_ptr()
        pitches[i] = o.stride(0)
    return imgs, stats_array(tile_stats), out_p, pitches


class Batch:
    """A fixed table of tiles (each with its own source Stats) normalised to
    one target by one cooperative persistent launch (spcn_batch_*).

    ``run`` is asynchronous and allocation-free, so it can be captured into a
    CUDA graph; the tiles and outputs must stay allocated while the batch is
    used (this object keeps references to them)."""

    def __init__(self, ctx: "Context", tiles, tile_stats, tgt_stats: Stats, outs,
                 p: Params | None = None):
        imgs, st, out_p, pitches = _batch_arrays(tiles, tile_stats, outs)
        self.p = p or params()
        self.tgt = tgt_stats.copy()
        h = ctypes.c_void_p()
        rc = _lib.spcn_batch_create(ctx.handle, len(tiles), imgs, st, ctypes.byref(self.tgt),
                                    ctypes.byref(self.p), out_p, pitches, ctypes.byref(h))
        _check(rc, "spcn_batch_create")
        self._h = h
        self.n = len(tiles)
        self._keep = (ctx, list(tiles), list(outs), imgs, st, out_p, pitches)

    def close(self):
        if getattr(self, "_h", None):
            _lib.spcn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, stream=None):
        _check(_lib.spcn_batch_run(self._h, _stream(stream)), "spcn_batch_run")

    def results(self, stream=None, fallback: bool = False):
        """(p99 as a list of (p0, p1) per tile, status per tile[, fallback
        flag per tile]); waits."""
        p99 = (ctypes.c_double * (2 * self.n))()
        status = (ctypes.c_int32 * self.n)()
        fb = (ctypes.c_int32 * self.n)()
        _check(_lib.spcn_batch_results(self._h, p99, status, fb, _stream(stream)),
               "spcn_batch_results")
        out = ([(p99[2 * i], p99[2 * i + 1]) for i in range(self.n)], list(status))
        return out + (list(fb),) if fallback else out

    @property
    def config(self) -> dict:
        c = BatchConfig()
        _check(_lib.spcn_batch_get_config(self._h, ctypes.byref(c)), "spcn_batch_get_config")
        return c.as_dict()

    def set_config(self, item_chunks: int, schedule: str = "phased", group_px: int = 0):
        c = BatchConfig(int(item_chunks), SCHEDULES[schedule], int(group_px), 0.0, 0)
        _check(_lib.spcn_batch_set_config(self._h, ctypes.byref(c)), "spcn_batch_set_config")

    def tune(self, reps: int = 3, stream=None):
        """Run the library's autotuner; returns every trial (dicts with the
        mean ms per run) and leaves the fastest schedule selected."""
        trials = (BatchConfig * 64)()
        n = ctypes.c_int32()
        _check(_lib.spcn_batch_tune(self._h, int(reps), trials, 64, ctypes.byref(n),
                                    _stream(stream)), "spcn_batch_tune")
        return [trials[i].as_dict() for i in range(n.value)]


def normalize_batched(ctx: "Context", tiles, tile_stats, tgt_stats: Stats, outs,
                      p: Params | None = None, stream=None):
    """One-shot batch (create, run, results, destroy); returns (p99, status)
    as in Batch.results.  Blocks."""
    imgs, st, out_p, pitches = _batch_arrays(tiles, tile_stats, outs)
    p = p or params()
    n = len(tiles)
    p99 = (ctypes.c_double * (2 * n))()
    status = (ctypes.c_int32 * n)()
    rc = _lib.spcn_normalize_batched(ctx.handle, n, imgs, st, ctypes.byref(tgt_stats),
                                     ctypes.byref(p), out_p, pitches, p99, status, _stream(stream))
    _check(rc, "spcn_normalize_batched")
    return [(p99[2 * i], p99[2 * i + 1]) for i in range(n)], list(status)
