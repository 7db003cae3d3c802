"""Thin Python binding over the C ABI of ``libatdct16.so`` (include/atdct16.h).

Argument marshalling only: every step of the transform runs in the CUDA
library.  Tensors are torch CUDA tensors; their ``data_ptr()`` and the current
torch stream are passed straight through.  If the library has not been built
the first call raises -- there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

U8, I16 = 0, 1
PLAN_ZIGZAG = 1  # ATDCT16_PLAN_ZIGZAG
PLAN_TEST_STALL_COPIES = 0x80000000  # ATDCT16_PLAN_TEST_STALL_COPIES (failure-path test hook)
PLAN_TEST_STALL_MMA = 0x40000000  # ATDCT16_PLAN_TEST_STALL_MMA (failure-path test hook)
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, EDEVICE = range(7)


class Atdct16Error(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class Image(C.Structure):
    """Mirror of ``atdct16_image``."""

    _fields_ = [
        ("src", C.c_void_p),
        ("dst", C.c_void_p),
        ("src_pitch", C.c_int64),
        ("dst_pitch", C.c_int64),
        ("width", C.c_int32),
        ("height", C.c_int32),
        ("r_or_qp", C.c_int32),
        ("reserved", C.c_int32),
    ]


class ServerConfig(C.Structure):
    """Mirror of ``atdct16_server_config``."""

    _fields_ = [
        ("memory_budget_bytes", C.c_size_t),
        ("max_batch", C.c_int32),
        ("compute_slots", C.c_int32),
        ("reserved", C.c_int32),
    ]


class Request(C.Structure):
    """Mirror of ``atdct16_request``."""

    _fields_ = [
        ("h_src", C.c_void_p),
        ("h_dst", C.c_void_p),
        ("src_pitch", C.c_int64),
        ("dst_pitch", C.c_int64),
        ("width", C.c_int32),
        ("height", C.c_int32),
        ("r", C.c_int32),
        ("reserved", C.c_int32),
    ]


class RequestTiming(C.Structure):
    """Mirror of ``atdct16_request_timing`` (seconds on the server clock)."""

    _fields_ = [(k, C.c_double) for k in ("arrival", "submit", "h2d_start", "h2d_end", "compute_start",
                                          "compute_end", "d2h_end", "done")]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "atdct16_version": (C.c_char_p, []),
    "atdct16_status_string": (C.c_char_p, [C.c_int]),
    "atdct16_plan_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int32, C.c_size_t, C.c_uint32]),
    "atdct16_plan_destroy": (C.c_int, [C.c_void_p]),
    "atdct16_forward": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "atdct16_inverse": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p]),
    "atdct16_forward_1d": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "atdct16_inverse_1d": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "atdct16_compress_zonal": (C.c_int, [C.c_void_p, C.POINTER(Image), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "atdct16_compress_quant": (C.c_int, [C.c_void_p, C.POINTER(Image), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "atdct16_psnr": (C.c_int, [C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "atdct16_last_device_status": (C.c_int, [C.c_void_p]),
    "atdct16_host_butterfly": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int32]),
    "atdct16_compress_zonal_noalloc": (C.c_int, [C.POINTER(Image), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "atdct16_noalloc_last_device_status": (C.c_int, [C.c_void_p]),
    "atdct16_batch_create": (C.c_int, [C.c_void_p, C.POINTER(Image), C.c_int32, C.c_void_p, C.c_void_p, C.c_uint32,
                                       C.c_void_p, C.POINTER(C.c_void_p)]),
    "atdct16_batch_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "atdct16_batch_last_device_status": (C.c_int, [C.c_void_p]),
    "atdct16_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_float)]),
    "atdct16_batch_destroy": (C.c_int, [C.c_void_p]),
    "atdct16_server_create": (C.c_int, [C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]),
    "atdct16_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "atdct16_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.c_int64]),
    "atdct16_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_size_t)]),
    "atdct16_server_destroy": (C.c_int, [C.c_void_p]),
    "atdct16_server_clock": (C.c_double, []),
    "atdct16_server_submit_at": (C.c_int, [C.c_void_p, C.POINTER(Request), C.c_double, C.POINTER(C.c_uint64)]),
    "atdct16_server_wait_timing": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_double), C.c_void_p, C.c_int64]),
    "atdct16_ssim_batch": (C.c_int, [C.c_void_p, C.POINTER(Image), C.c_int32, C.c_void_p, C.c_void_p]),
    "atdct16_compress_zonal_dct": (C.c_int, [C.c_void_p, C.POINTER(Image), C.c_int32, C.c_void_p, C.c_void_p,
                                            C.c_void_p]),
    "atdct16_batch_tuning": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "atdct16_plan_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "atdct16_plan_profile": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
}


def library_path() -> str:
    return _build.LIB_PATH


def lib() -> C.CDLL:
    """Load ``libatdct16.so`` (raises if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"atdct16 CUDA library missing at {path}; build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().atdct16_status_string(status).decode()
    except RuntimeError:
        return "library not loaded"


def _check(status: int, what: str):
    if status != OK:
        raise Atdct16Error(status, what)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def host_butterfly(values, inverse=False):
    """Run the library's 1-D butterfly on the host (16 int32 values)."""
    a = (C.c_int32 * 16)(*[int(v) for v in values])
    o = (C.c_int32 * 16)()
    _check(lib().atdct16_host_butterfly(a, o, 1 if inverse else 0), "host_butterfly")
    return list(o)


def descriptors(images):
    """A reusable C array of Image descriptors.  Building the array costs
    about 0.2 us per image on the host; a caller that compresses the same
    set of buffers repeatedly builds it once and passes it instead of a
    list."""
    return (Image * len(images))(*images)


def _as_array(images):
    return images if isinstance(images, C.Array) else descriptors(images)


def image(src, dst, param, width=None, height=None):
    """Descriptor for a 2-D (H, W) torch tensor pair (row pitch from strides)."""
    h, w = src.shape[-2], src.shape[-1]
    es = src.element_size()
    return Image(src.data_ptr(), 0 if dst is None else dst.data_ptr(), src.stride(-2) * es,
                 0 if dst is None else dst.stride(-2) * dst.element_size(),
                 w if width is None else width, h if height is None else height, int(param), 0)


class Plan:
    """Owns an ``atdct16_plan_t`` (device workspace)."""

    def __init__(self, dtype=U8, max_images=64, workspace_bytes=0, zigzag=False, flags=None):
        """``zigzag``: block coefficients (forward / inverse) and quantisation
        levels in the zig-zag scan order; ``flags`` overrides it with raw
        ``atdct16_plan_create`` flags."""
        self._h = C.c_void_p()
        fl = (PLAN_ZIGZAG if zigzag else 0) if flags is None else flags
        _check(lib().atdct16_plan_create(C.byref(self._h), dtype, max_images, workspace_bytes, fl), "plan_create")
        self.dtype = dtype
        self.max_images = max_images
        self.zigzag = bool(fl & PLAN_ZIGZAG)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().atdct16_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, img, coef, dtype=U8, stream=None):
        h, w = img.shape[-2], img.shape[-1]
        _check(lib().atdct16_forward(self._h, dtype, _ptr(img), img.stride(-2) * img.element_size(), w, h,
                                     _ptr(coef), _stream(stream)), "forward")

    def inverse(self, coef, out, dtype=U8, stream=None):
        h, w = out.shape[-2], out.shape[-1]
        _check(lib().atdct16_inverse(self._h, dtype, _ptr(coef), w, h, _ptr(out),
                                     out.stride(-2) * out.element_size(), _stream(stream)), "inverse")

    def forward_1d(self, x, coef, count=None, dtype=U8, stream=None):
        """``x``: 16 * count samples (contiguous), ``coef``: 16 * count int32."""
        n = x.numel() // 16 if count is None else count
        _check(lib().atdct16_forward_1d(self._h, dtype, _ptr(x), n, _ptr(coef), _stream(stream)), "forward_1d")

    def inverse_1d(self, coef, out, count=None, dtype=U8, stream=None):
        n = coef.numel() // 16 if count is None else count
        _check(lib().atdct16_inverse_1d(self._h, dtype, _ptr(coef), n, _ptr(out), _stream(stream)), "inverse_1d")

    def compress_zonal(self, images, psnr, sse=None, stream=None):
        """``images``: list of Image descriptors (param = r), or an array from
        ``descriptors``."""
        arr = _as_array(images)
        _check(lib().atdct16_compress_zonal(self._h, arr, len(images), _ptr(psnr), _ptr(sse), _stream(stream)),
               "compress_zonal")

    def compress_quant(self, images, psnr, levels=None, sse=None, stream=None):
        arr = _as_array(images)
        _check(lib().atdct16_compress_quant(self._h, arr, len(images), _ptr(levels), _ptr(psnr), _ptr(sse),
                                            _stream(stream)), "compress_quant")

    def compress_zonal_dct(self, images, psnr, sse=None, stream=None):
        """The exact-DCT baseline of ``compress_zonal`` (FP32 dense DCT-II)."""
        arr = _as_array(images)
        _check(lib().atdct16_compress_zonal_dct(self._h, arr, len(images), _ptr(psnr), _ptr(sse), _stream(stream)),
               "compress_zonal_dct")

    def ssim(self, images, out, stream=None):
        """Mean SSIM of each (src, dst) u8 pair of ``images`` into ``out``
        (float64, one per image)."""
        arr = _as_array(images)
        _check(lib().atdct16_ssim_batch(self._h, arr, len(images), _ptr(out), _stream(stream)), "ssim_batch")

    def set_profiling(self, on=True, every=1):
        """Bracket the first fused launch and then every `every`-th one with CUDA events."""
        _check(lib().atdct16_plan_set_profiling(self._h, int(every) if on else 0), "set_profiling")

    def profile(self):
        """(timed kernel launches, summed kernel milliseconds) since the last call."""
        n, ms = C.c_int64(), C.c_double()
        _check(lib().atdct16_plan_profile(self._h, C.byref(n), C.byref(ms)), "profile")
        return n.value, ms.value

    def last_device_status(self) -> int:
        return lib().atdct16_last_device_status(self._h)


BATCH_AUTOTUNE, BATCH_GRAPH = 1, 2
ZONAL_VARIANTS = ("f32", "swar", "mma", "tc")


def batch_variant(v):
    """Flag that pins the zonal kernel variant of a Batch (0, 1, 2 or 3)."""
    return (v + 1) << 8


def batch_shape(tiles_per_cta, staging_depth, vector_bytes):
    """Flag that pins the launch shape of a Batch's kernels for r <= 36."""
    w = {2: 1, 4: 2, 8: 3}[tiles_per_cta]
    v = {8: 1, 16: 2}[vector_bytes]
    return (w | (staging_depth << 2) | (v << 4)) << 12


class TunePoint(C.Structure):
    """``atdct16_tune_point``: one launch shape of a batch and its median time."""

    _fields_ = [("phase", C.c_int32), ("variant", C.c_int32), ("general_ctas", C.c_int32), ("tiles_per_cta", C.c_int32),
                ("staging_depth", C.c_int32), ("vector_bytes", C.c_int32), ("box_ctas", C.c_int32),
                ("ms", C.c_float)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["variant"] = ZONAL_VARIANTS[self.variant]
        return d


class Batch:
    """A resident zonal batch (``atdct16_batch_*``): descriptors on the device,
    optional autotuned launch shape and CUDA-graph capture."""

    def __init__(self, plan, images, psnr, sse=None, flags=BATCH_AUTOTUNE | BATCH_GRAPH, stream=None):
        self._h = C.c_void_p()
        self.plan = plan  # keeps the plan alive
        arr = _as_array(images)
        _check(lib().atdct16_batch_create(plan.handle, arr, len(images), _ptr(psnr), _ptr(sse), flags,
                                          _stream(stream), C.byref(self._h)), "batch_create")

    def launch(self, stream=None):
        _check(lib().atdct16_batch_launch(self._h, _stream(stream)), "batch_launch")

    def last_device_status(self) -> int:
        """Sticky device status of this batch's launches (waits for the last one)."""
        return lib().atdct16_batch_last_device_status(self._h)

    def info(self):
        v, w, p, g = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        t, ms = C.c_int64(), C.c_float()
        _check(lib().atdct16_batch_info(self._h, C.byref(v), C.byref(w), C.byref(p), C.byref(g), C.byref(t),
                                        C.byref(ms)), "batch_info")
        return {"variant": ZONAL_VARIANTS[v.value], "warps": w.value, "prefetch": p.value, "grid": g.value,
                "tiles": t.value, "tuned_ms": ms.value}

    def tuning(self):
        """The chosen launch shape and every candidate the autotuner timed."""
        n = C.c_int32()
        chosen = TunePoint()
        _check(lib().atdct16_batch_tuning(self._h, C.byref(chosen), None, 0, C.byref(n)), "batch_tuning")
        cands = (TunePoint * max(1, n.value))()
        _check(lib().atdct16_batch_tuning(self._h, None, cands, n.value, C.byref(n)), "batch_tuning")
        return {"chosen": chosen.as_dict(), "candidates": [cands[i].as_dict() for i in range(n.value)]}

    def close(self):
        if self._h:
            lib().atdct16_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(a):
    """Address of a host buffer: a CPU torch tensor or a numpy array."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), a.stride(-2) * a.element_size()
    return a.ctypes.data, a.strides[-2]


class Server:
    """Continuous-batching compression server (``atdct16_server_*``)."""

    def __init__(self, memory_budget_bytes=1 << 30, max_batch=64, compute_slots=2):
        self._h = C.c_void_p()
        cfg = ServerConfig(memory_budget_bytes, max_batch, compute_slots, 0)
        _check(lib().atdct16_server_create(C.byref(cfg), C.byref(self._h)), "server_create")

    def submit(self, src, dst, r, arrival=None):
        """Queue ``src`` (H, W uint8, host) -> ``dst`` (host); returns a ticket.
        ``arrival``: the request's arrival time on :func:`server_clock`
        (latency is measured from it; default: now)."""
        sp, spitch = _host_ptr(src)
        dp, dpitch = _host_ptr(dst)
        h, w = src.shape[-2], src.shape[-1]
        req = Request(sp, dp, spitch, dpitch, w, h, int(r), 0)
        t = C.c_uint64()
        if arrival is None:
            _check(lib().atdct16_server_submit(self._h, C.byref(req), C.byref(t)), "server_submit")
        else:
            _check(lib().atdct16_server_submit_at(self._h, C.byref(req), float(arrival), C.byref(t)),
                   "server_submit_at")
        return t.value

    def wait_timing(self, ticket, timeout_us=-1):
        """(PSNR, stage timestamps on the server clock) of a request; forgets the ticket."""
        p, tm = C.c_double(), RequestTiming()
        _check(lib().atdct16_server_wait_timing(self._h, ticket, C.byref(p), C.byref(tm), timeout_us),
               "server_wait_timing")
        return p.value, {k: getattr(tm, k) for k, _ in RequestTiming._fields_}

    def wait(self, ticket, timeout_us=-1):
        """(PSNR, latency in seconds) of a request; forgets the ticket."""
        p, lat = C.c_double(), C.c_double()
        _check(lib().atdct16_server_wait(self._h, ticket, C.byref(p), C.byref(lat), timeout_us), "server_wait")
        return p.value, lat.value

    def stats(self):
        c, l, px, b, a = C.c_uint64(), C.c_uint64(), C.c_double(), C.c_double(), C.c_size_t()
        _check(lib().atdct16_server_stats(self._h, C.byref(c), C.byref(l), C.byref(px), C.byref(b), C.byref(a)),
               "server_stats")
        return {"completed": c.value, "launches": l.value, "pixels": px.value, "busy_s": b.value,
                "arena_used": a.value}

    def close(self):
        if self._h:
            lib().atdct16_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_clock() -> float:
    """Seconds on the server's steady clock."""
    return float(lib().atdct16_server_clock())


def compress_zonal_noalloc(images, psnr, sse=None, stream=None):
    """Zonal compression through the entry point that allocates nothing (no
    plan; at most 64 images and 131072 tiles per call)."""
    arr = _as_array(images)
    _check(lib().atdct16_compress_zonal_noalloc(arr, len(images), _ptr(psnr), _ptr(sse), _stream(stream)),
           "compress_zonal_noalloc")


def noalloc_last_device_status(stream=None) -> int:
    """Device-side status of the last no-allocation call on the current
    device (synchronises ``stream``)."""
    return int(lib().atdct16_noalloc_last_device_status(_stream(stream)))


def psnr(a, b, out, dtype=U8, stream=None):
    h, w = a.shape[-2], a.shape[-1]
    _check(lib().atdct16_psnr(dtype, _ptr(a), a.stride(-2) * a.element_size(), _ptr(b),
                              b.stride(-2) * b.element_size(), w, h, _ptr(out), _stream(stream)), "psnr")
