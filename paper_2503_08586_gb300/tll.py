"""Python binding of libtll.so (ctypes).  Argument marshalling only: every
step of the likelihood runs in the library's CUDA kernels.  There is no
fallback -- if the library is missing or no GPU is usable, calls raise.

Device tensors are torch tensors (torch provides memory and streams);
host arrays are numpy arrays or CPU tensors (pinned ones copy faster).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtll.so")

NPARAM = 21
NPARAM_EPL = 22
MASS_EPL = 0x400
AMP_LINEAR = 0
AMP_FIXED = 1
FLAG_DIRECT_CONV = 0x100
FLAG_BATCH_ONLY = 0x200
NOALLOC_MAX_B = 16384

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY = range(6)
_CODES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUSY"}

# Every entry point include/tll.h declares (checked by the ABI test).
SYMBOLS = ("tll_create_lens", "tll_loglike_batch", "tll_loglike_batch_host",
           "tll_loglike_batch_noalloc", "tll_batcher_create", "tll_batcher_run",
           "tll_batcher_destroy", "tll_lens_footprint", "tll_server_create",
           "tll_server_open_job", "tll_server_close_job", "tll_server_submit",
           "tll_server_poll", "tll_server_wait", "tll_server_stats",
           "tll_server_destroy", "tll_server_last_error",
           "tll_model_image", "tll_model_columns", "tll_lens_info",
           "tll_profile_enable", "tll_profile_last", "tll_lens_shape", "tll_set_shape",
           "tll_autotune", "tll_set_conv", "tll_conv_check", "tll_lens_nparam",
           "tll_destroy_lens", "tll_last_error", "tll_version", "tll_set_light",
           "tll_lens_ncols", "tll_model_columns_n", "tll_lens_ntrace",
           "tll_sampler_create", "tll_sampler_set_walkers", "tll_sampler_run",
           "tll_sampler_state", "tll_sampler_destroy", "tll_server_set_light",
           "tll_autotune_save", "tll_autotune_load", "tll_autotune_clear")

# Multi-component light (tll_set_light).
MAX_COMPS = 32
COMP_SERSIC, COMP_GAUSSIAN = 0, 1
PLANE_LENS, PLANE_SOURCE = 0, 1
COMP_FREE_SCALE, COMP_FREE_INDEX = 1, 2
MULTI_HEAD = 15


class TLLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("pixel_scale", ctypes.c_float), ("sub", ctypes.c_int),
                ("x0", ctypes.c_float), ("y0", ctypes.c_float)]


class Comp(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("plane", ctypes.c_int),
                ("flags", ctypes.c_int), ("scale", ctypes.c_float),
                ("index", ctypes.c_float)]


def comp(type: str, plane: str, free_scale: bool = True, free_index: bool = False,
         scale: float = 1.0, index: float = 1.0) -> Comp:
    """One light component: type "sersic" | "gauss", plane "lens" | "source"."""
    t = {"sersic": COMP_SERSIC, "gauss": COMP_GAUSSIAN}[type]
    pl = {"lens": PLANE_LENS, "source": PLANE_SOURCE}[plane]
    fl = (COMP_FREE_SCALE if free_scale else 0) | (
        COMP_FREE_INDEX if free_index and t == COMP_SERSIC else 0)
    return Comp(t, pl, fl, float(scale), float(index))


PLACEMENTS = {0: "global", 1: "smem", 2: "padded", 3: "banded"}
CONV_FUSED, CONV_SPLIT_DIRECT, CONV_SPLIT_TOEPLITZ_TC, CONV_SPLIT_TOEPLITZ_BF16 = 0, 1, 2, 3


class Shape(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("placement", ctypes.c_int), ("band_rows", ctypes.c_int),
                ("smem_bytes", ctypes.c_size_t), ("ms", ctypes.c_float),
                ("tuned", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"threads": self.threads, "ctas_per_sm": self.ctas_per_sm,
                "placement": PLACEMENTS.get(self.placement, self.placement),
                "band_rows": self.band_rows, "smem_bytes": int(self.smem_bytes),
                "ms": float(self.ms), "tuned": bool(self.tuned)}


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_jobs", ctypes.c_int),
                ("max_vectors_per_launch", ctypes.c_int), ("max_inflight", ctypes.c_int),
                ("coalesce", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("autotune", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("vectors", ctypes.c_longlong),
                ("requests", ctypes.c_longlong), ("admissions_refused", ctypes.c_longlong),
                ("pending", ctypes.c_longlong), ("inflight", ctypes.c_longlong),
                ("hbm_used_bytes", ctypes.c_size_t), ("open_jobs", ctypes.c_int),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_max_ms", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Load libtll.so (built in-tree by paper_2503_08586_gb300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with "
                           "`python -m paper_2503_08586_gb300.build`")
    lib = ctypes.CDLL(p)
    vp, i, fp, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
    lib.tll_create_lens.argtypes = [fp, fp, fp, i, ctypes.POINTER(Grid), i,
                                    ctypes.POINTER(vp)]
    lib.tll_create_lens.restype = i
    lib.tll_loglike_batch.argtypes = [vp, fp, i, dp, vp]
    lib.tll_loglike_batch.restype = i
    lib.tll_loglike_batch_host.argtypes = [vp, fp, i, dp, vp]
    lib.tll_loglike_batch_host.restype = i
    lib.tll_loglike_batch_noalloc.argtypes = [vp, fp, i, dp, vp]
    lib.tll_loglike_batch_noalloc.restype = i
    lib.tll_model_image.argtypes = [vp, fp, fp, fp, dp]
    lib.tll_model_image.restype = i
    lib.tll_model_columns.argtypes = [vp, fp, fp, fp, i]
    lib.tll_model_columns.restype = i
    ip = ctypes.POINTER(ctypes.c_int)
    lib.tll_lens_info.argtypes = [vp, ip, ip, ip, ip, ip, ip]
    lib.tll_lens_info.restype = i
    lib.tll_profile_enable.argtypes = [vp, i]
    lib.tll_profile_enable.restype = i
    lib.tll_profile_last.argtypes = [vp, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_float)]
    lib.tll_profile_last.restype = i
    lib.tll_lens_shape.argtypes = [vp, ctypes.POINTER(Shape)]
    lib.tll_lens_shape.restype = i
    lib.tll_lens_nparam.argtypes = [vp]
    lib.tll_lens_nparam.restype = i
    lib.tll_set_conv.argtypes = [vp, i, i]
    lib.tll_set_conv.restype = i
    lib.tll_conv_check.argtypes = [vp]
    lib.tll_conv_check.restype = i
    lib.tll_set_shape.argtypes = [vp, i, i]
    lib.tll_set_shape.restype = i
    lib.tll_autotune.argtypes = [vp, fp, i, vp, ctypes.POINTER(Shape), ctypes.POINTER(Shape), i,
                                 ctypes.POINTER(ctypes.c_int)]
    lib.tll_autotune.restype = i
    lib.tll_batcher_create.argtypes = [i, ctypes.POINTER(vp)]
    lib.tll_batcher_create.restype = i
    lib.tll_batcher_run.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp),
                                    i, vp]
    lib.tll_batcher_run.restype = i
    lib.tll_batcher_destroy.argtypes = [vp]
    lib.tll_batcher_destroy.restype = None
    sz = ctypes.c_size_t
    lib.tll_lens_footprint.argtypes = [vp, ctypes.POINTER(sz)]
    lib.tll_lens_footprint.restype = i
    lib.tll_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.tll_server_create.restype = i
    lib.tll_server_open_job.argtypes = [vp, fp, fp, fp, i, ctypes.POINTER(Grid), i,
                                        ctypes.POINTER(ctypes.c_int)]
    lib.tll_server_open_job.restype = i
    lib.tll_server_close_job.argtypes = [vp, i]
    lib.tll_server_close_job.restype = i
    lib.tll_server_submit.argtypes = [vp, i, fp, i, dp, ctypes.POINTER(ctypes.c_longlong)]
    lib.tll_server_submit.restype = i
    lib.tll_server_poll.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
    lib.tll_server_poll.restype = i
    lib.tll_server_wait.argtypes = [vp, ctypes.c_longlong, i, ctypes.POINTER(ctypes.c_double)]
    lib.tll_server_wait.restype = i
    lib.tll_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.tll_server_stats.restype = i
    lib.tll_server_destroy.argtypes = [vp]
    lib.tll_server_destroy.restype = None
    lib.tll_server_last_error.argtypes = []
    lib.tll_server_last_error.restype = ctypes.c_char_p
    lib.tll_destroy_lens.argtypes = [vp]
    lib.tll_destroy_lens.restype = None
    lib.tll_last_error.argtypes = []
    lib.tll_last_error.restype = ctypes.c_char_p
    lib.tll_version.argtypes = []
    lib.tll_version.restype = i
    lib.tll_set_light.argtypes = [vp, ctypes.POINTER(Comp), i]
    lib.tll_set_light.restype = i
    lib.tll_lens_ncols.argtypes = [vp]
    lib.tll_lens_ncols.restype = i
    lib.tll_lens_ntrace.argtypes = [vp]
    lib.tll_lens_ntrace.restype = i
    lib.tll_sampler_create.argtypes = [vp, i, fp, fp, ctypes.c_double, i, ctypes.c_ulonglong,
                                       ctypes.POINTER(vp)]
    lib.tll_sampler_create.restype = i
    lib.tll_sampler_set_walkers.argtypes = [vp, fp, vp]
    lib.tll_sampler_set_walkers.restype = i
    lib.tll_sampler_run.argtypes = [vp, i, fp, dp, dp, vp]
    lib.tll_sampler_run.restype = i
    ll = ctypes.POINTER(ctypes.c_longlong)
    lib.tll_sampler_state.argtypes = [vp, fp, dp, ll, ll, ll, vp]
    lib.tll_sampler_state.restype = i
    lib.tll_sampler_destroy.argtypes = [vp]
    lib.tll_sampler_destroy.restype = None
    lib.tll_server_set_light.argtypes = [vp, i, ctypes.POINTER(Comp), i]
    lib.tll_server_set_light.restype = i
    lib.tll_autotune_save.argtypes = [ctypes.c_char_p]
    lib.tll_autotune_save.restype = i
    lib.tll_autotune_load.argtypes = [ctypes.c_char_p]
    lib.tll_autotune_load.restype = i
    lib.tll_autotune_clear.argtypes = []
    lib.tll_autotune_clear.restype = None
    lib.tll_model_columns_n.argtypes = [vp, fp, fp, i]
    lib.tll_model_columns_n.restype = i
    if path is None:
        _lib = lib
    return lib


def _check(rc: int):
    if rc != OK:
        raise TLLError(rc, load().tll_last_error().decode(errors="replace"))


def _host_ptr(a, dtype):
    """(pointer, keep-alive) for a contiguous host array of dtype."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda:
                raise ValueError("expected a host tensor")
            want = torch.float32 if dtype == np.float32 else torch.float64
            if a.dtype != want or not a.is_contiguous():
                raise ValueError(f"expected a contiguous {want} host tensor")
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Lens:
    """One observed lens resident on the current CUDA device."""

    def __init__(self, image, noise, psf, pixel_scale: float, sub: int,
                 x0: float | None = None, y0: float | None = None,
                 mode: int = AMP_LINEAR, direct_conv: bool = False,
                 batch_only: bool = False, mass: str = "sie"):
        """mass: "sie" (21 parameters per vector) or "epl" (the elliptical
        power law of Eq. 12, 22 parameters: the slope gamma last)."""
        lib = load()
        if mass not in ("sie", "epl"):
            raise ValueError("mass must be 'sie' or 'epl'")
        img = np.ascontiguousarray(image, dtype=np.float32)
        nse = np.ascontiguousarray(noise, dtype=np.float32)
        k = np.ascontiguousarray(psf, dtype=np.float32)
        if img.ndim != 2 or nse.shape != img.shape or k.ndim != 2 \
                or k.shape[0] != k.shape[1]:
            raise ValueError("image/noise must be [ny, nx], psf square")
        ny, nx = img.shape
        if x0 is None:
            x0 = -(nx - 1) * pixel_scale / 2.0
        if y0 is None:
            y0 = -(ny - 1) * pixel_scale / 2.0
        g = Grid(nx, ny, pixel_scale, sub, x0, y0)
        h = ctypes.c_void_p()
        flags = (mode | (FLAG_DIRECT_CONV if direct_conv else 0)
                 | (FLAG_BATCH_ONLY if batch_only else 0)
                 | (MASS_EPL if mass == "epl" else 0))
        _check(lib.tll_create_lens(img.ctypes.data, nse.ctypes.data,
                                   k.ctypes.data, k.shape[0], ctypes.byref(g),
                                   flags, ctypes.byref(h)))
        self._h = h
        self.ny, self.nx, self.sub, self.psf_size = ny, nx, sub, k.shape[0]
        self.mode = mode
        self.mass = mass
        self.nparam = lib.tll_lens_nparam(h)
        self.ncols = 2
        self.pixel_scale, self.x0, self.y0 = pixel_scale, x0, y0

    @property
    def handle(self):
        return self._h

    def ntrace(self) -> int:
        """Pixels the batched kernels trace per vector (fewer than ny * nx
        when masked pixels leave some out of the PSF's reach)."""
        return load().tll_lens_ntrace(self._h)

    def info(self) -> dict:
        v = [ctypes.c_int() for _ in range(6)]
        _check(load().tll_lens_info(self._h, *[ctypes.byref(x) for x in v]))
        keys = ("nx", "ny", "sub", "psf_size", "flags", "separable")
        return {k: x.value for k, x in zip(keys, v)}

    # -- device batch
    def loglike_batch(self, params, out=None, stream=None):
        """params: CUDA float32 tensor [B, 21]; returns CUDA float64 [B]
        (asynchronous on `stream`, default torch's current stream)."""
        import torch
        if not (params.is_cuda and params.dtype == torch.float32
                and params.dim() == 2 and params.shape[1] == self.nparam
                and params.is_contiguous()):
            raise ValueError(f"params must be a contiguous CUDA float32 [B, {self.nparam}]")
        B = params.shape[0]
        if out is None:
            out = torch.empty(B, dtype=torch.float64, device=params.device)
        elif not (out.is_cuda and out.dtype == torch.float64
                  and out.numel() >= B and out.is_contiguous()):
            raise ValueError("out must be a contiguous CUDA float64 [B]")
        _check(load().tll_loglike_batch(self._h, params.data_ptr(), B,
                                        out.data_ptr(), _stream_handle(stream)))
        return out

    def loglike_batch_noalloc(self, params, out, stream=None):
        """As loglike_batch, but the call allocates no device memory: the
        library's fixed scratch array is used (B <= NOALLOC_MAX_B; calls
        that overlap on the GPU race on that array).  `out` must be given,
        since creating it would allocate."""
        import torch
        if not (params.is_cuda and params.dtype == torch.float32
                and params.dim() == 2 and params.shape[1] == self.nparam
                and params.is_contiguous()):
            raise ValueError(f"params must be a contiguous CUDA float32 [B, {self.nparam}]")
        B = params.shape[0]
        if not (out.is_cuda and out.dtype == torch.float64
                and out.numel() >= B and out.is_contiguous()):
            raise ValueError("out must be a contiguous CUDA float64 [B]")
        _check(load().tll_loglike_batch_noalloc(self._h, params.data_ptr(), B,
                                                out.data_ptr(),
                                                _stream_handle(stream)))
        return out

    # -- host batch (copies inside the call)
    def loglike_batch_host(self, params, out=None, stream=None):
        """params: host float32 [B, nparam] (numpy or CPU tensor, pinned is
        best); returns host float64 [B] (numpy unless `out` is given)."""
        p, keep = _host_ptr(params, np.float32)
        B = int(np.prod(keep.shape)) // self.nparam
        if out is None:
            out = np.empty(B, dtype=np.float64)
        o, okeep = _host_ptr(out, np.float64)
        if okeep is not out:
            raise ValueError("out must be a contiguous float64 host array")
        _check(load().tll_loglike_batch_host(self._h, p, B, o,
                                             _stream_handle(stream)))
        return out

    # -- multi-component light
    def set_light(self, comps):
        """Give the lens a multi-component light model: a list of Comp
        (see comp()); [] returns it to the two-column model.  Updates
        self.nparam and self.ncols."""
        arr = (Comp * max(1, len(comps)))(*comps)
        _check(load().tll_set_light(self._h, arr, len(comps)))
        self.nparam = load().tll_lens_nparam(self._h)
        self.ncols = load().tll_lens_ncols(self._h)

    def model_columns_n(self, params, blurred: bool = True):
        """Every unit-amplitude column [ncols, ny, nx] float32."""
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(self.nparam)
        nc = load().tll_lens_ncols(self._h)
        out = np.empty((nc, self.ny, self.nx), dtype=np.float32)
        _check(load().tll_model_columns_n(self._h, p.ctypes.data, out.ctypes.data,
                                          1 if blurred else 0))
        return out

    # -- single vector
    def model_image(self, params):
        """(blurred model image [ny, nx] float32, amplitudes (ncols,), log L)."""
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(self.nparam)
        img = np.empty((self.ny, self.nx), dtype=np.float32)
        amps = np.empty(load().tll_lens_ncols(self._h), dtype=np.float32)
        ll = ctypes.c_double()
        _check(load().tll_model_image(self._h, p.ctypes.data, img.ctypes.data,
                                      amps.ctypes.data, ctypes.byref(ll)))
        return img, amps, ll.value

    def model_columns(self, params, blurred: bool = True):
        """Unit-amplitude (lens, source) columns [ny, nx] float32."""
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(self.nparam)
        a = np.empty((self.ny, self.nx), dtype=np.float32)
        b = np.empty((self.ny, self.nx), dtype=np.float32)
        _check(load().tll_model_columns(self._h, p.ctypes.data, a.ctypes.data,
                                        b.ctypes.data, 1 if blurred else 0))
        return a, b

    # -- launch shape
    def shape(self) -> dict:
        """The batched kernels' launch shape (CTA size, CTAs per SM,
        image placement, band rows, shared memory)."""
        sh = Shape()
        _check(load().tll_lens_shape(self._h, ctypes.byref(sh)))
        return sh.as_dict()

    def set_conv(self, variant: int, chunk: int = 0):
        """Convolution variant of the one-lens batched path: CONV_FUSED
        (default), CONV_SPLIT_DIRECT, CONV_SPLIT_TOEPLITZ_TC (3xTF32) or
        CONV_SPLIT_TOEPLITZ_BF16 (split-BF16) (split pipeline, chunk vectors
        per pass, 0: 1024)."""
        _check(load().tll_set_conv(self._h, int(variant), int(chunk)))

    def conv_check(self):
        """Raise TLLError(ETIMEOUT) if the tensor-core convolution's
        bounded waits ran out since the last check (waits for the device)."""
        _check(load().tll_conv_check(self._h))

    def set_shape(self, threads: int, ctas_per_sm: int) -> dict:
        """Use `threads`-thread CTAs, ctas_per_sm per SM; returns the shape."""
        _check(load().tll_set_shape(self._h, int(threads), int(ctas_per_sm)))
        return self.shape()

    def autotune(self, params=None, stream=None) -> dict:
        """Time the candidate launch shapes on the device and keep the
        fastest.  params: CUDA float32 [B, 21] to time with, or None for the
        library's built-in set.  Returns {"chosen": shape, "tried": [shapes]}
        (each with its mean time per tuning batch, ms)."""
        p, B = None, 0
        if params is not None:
            import torch
            if not (params.is_cuda and params.dtype == torch.float32
                    and params.dim() == 2 and params.shape[1] == self.nparam
                    and params.is_contiguous()):
                raise ValueError(f"params must be a contiguous CUDA float32 [B, {self.nparam}]")
            p, B = ctypes.c_void_p(params.data_ptr()), int(params.shape[0])
        chosen = Shape()
        tried = (Shape * 8)()
        n = ctypes.c_int()
        _check(load().tll_autotune(self._h, p, B, _stream_handle(stream), ctypes.byref(chosen),
                                   tried, 8, ctypes.byref(n)))
        return {"chosen": chosen.as_dict(), "tried": [tried[k].as_dict() for k in range(n.value)]}

    # -- profiling hook
    def profile(self, on: bool = True):
        """Record events around the two launches of each batch call."""
        _check(load().tll_profile_enable(self._h, 1 if on else 0))

    def profile_last(self):
        """(prologue ms, main-kernel ms) of the last batch call (waits)."""
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(load().tll_profile_last(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().tll_destroy_lens(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def autotune_save(path: str):
    """Write this process's tuned launch shapes to a cache file."""
    _check(load().tll_autotune_save(os.fsencode(path)))


def autotune_load(path: str):
    """Add a cache file's tuned shapes (for GPUs of the same name); lenses
    created afterwards start with them."""
    _check(load().tll_autotune_load(os.fsencode(path)))


def autotune_clear():
    """Forget every tuned launch shape of this process."""
    load().tll_autotune_clear()


class Sampler:
    """Device-side ensemble sampler (stretch move, Philox4x32-10) over one
    lens: proposals, likelihood, accept / reject and the chain stay on the
    GPU (see tll_sampler_* in tll.h)."""

    def __init__(self, lens: "Lens", nwalkers: int, lo, hi, a: float = 2.0, ndim: int = 0,
                 seed: int = 0):
        lo = np.ascontiguousarray(lo, np.float32)
        hi = np.ascontiguousarray(hi, np.float32)
        if lo.shape != (lens.nparam,) or hi.shape != (lens.nparam,):
            raise ValueError(f"lo, hi must have {lens.nparam} entries")
        h = ctypes.c_void_p()
        _check(load().tll_sampler_create(lens.handle, int(nwalkers), lo.ctypes.data,
                                         hi.ctypes.data, float(a), int(ndim), int(seed),
                                         ctypes.byref(h)))
        self._h = h
        self.lens, self.W, self.P = lens, int(nwalkers), lens.nparam

    def set_walkers(self, x0, stream=None):
        """x0: contiguous CUDA float32 [W, nparam]."""
        import torch
        if not (x0.is_cuda and x0.dtype == torch.float32 and x0.is_contiguous()
                and tuple(x0.shape) == (self.W, self.P)):
            raise ValueError(f"x0 must be a contiguous CUDA float32 [{self.W}, {self.P}]")
        _check(load().tll_sampler_set_walkers(self._h, x0.data_ptr(), _stream_handle(stream)))

    def run(self, nsteps: int, keep_chain: bool = True, keep_proposals: bool = False,
            stream=None):
        """Enqueue nsteps steps (asynchronous); returns (chain [n, W, P],
        lp [n, W], proposals' lp [n, W] or None) CUDA tensors, or Nones when
        keep_chain is False."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        chain = lpc = lpp = None
        if keep_chain:
            chain = torch.empty((nsteps, self.W, self.P), dtype=torch.float32, device=dev)
            lpc = torch.empty((nsteps, self.W), dtype=torch.float64, device=dev)
        if keep_proposals:
            lpp = torch.empty((nsteps, self.W), dtype=torch.float64, device=dev)
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(load().tll_sampler_run(self._h, int(nsteps), ptr(chain), ptr(lpc), ptr(lpp),
                                      _stream_handle(stream)))
        return chain, lpc, lpp

    def state(self, stream=None):
        """(walkers [W, P], lp [W] CUDA tensors, steps, accepted, proposed)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        x = torch.empty((self.W, self.P), dtype=torch.float32, device=dev)
        lp = torch.empty(self.W, dtype=torch.float64, device=dev)
        st, acc, pro = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().tll_sampler_state(self._h, x.data_ptr(), lp.data_ptr(), ctypes.byref(st),
                                        ctypes.byref(acc), ctypes.byref(pro),
                                        _stream_handle(stream)))
        return x, lp, st.value, acc.value, pro.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().tll_sampler_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Batcher:
    """One persistent launch over the parameter batches of several lenses
    (ragged sizes), optionally replayed as a CUDA graph."""

    def __init__(self, use_graph: bool = True):
        h = ctypes.c_void_p()
        _check(load().tll_batcher_create(1 if use_graph else 0, ctypes.byref(h)))
        self._h = h

    def run(self, lenses, params, outs=None, stream=None):
        """lenses: list of Lens; params: list of CUDA float32 [B_k, 21];
        returns the list of CUDA float64 [B_k] outputs (asynchronous)."""
        import torch
        n = len(lenses)
        if len(params) != n:
            raise ValueError("one params tensor per lens")
        if outs is None:
            outs = [torch.empty(p.shape[0], dtype=torch.float64, device=p.device)
                    for p in params]
        for L, p, o in zip(lenses, params, outs):
            if not (p.is_cuda and p.dtype == torch.float32 and p.is_contiguous()
                    and p.dim() == 2 and p.shape[1] == L.nparam):
                raise ValueError(f"params must be contiguous CUDA float32 [B, {L.nparam}]")
            if not (o.is_cuda and o.dtype == torch.float64 and o.is_contiguous()
                    and o.numel() >= p.shape[0]):
                raise ValueError("outs must be contiguous CUDA float64 [B]")
        arr_l = (ctypes.c_void_p * n)(*[L.handle.value for L in lenses])
        arr_p = (ctypes.c_void_p * n)(*[p.data_ptr() for p in params])
        arr_c = (ctypes.c_int * n)(*[p.shape[0] for p in params])
        arr_o = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        _check(load().tll_batcher_run(self._h, arr_l, arr_p, arr_c, arr_o, n,
                                      _stream_handle(stream)))
        return outs

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().tll_batcher_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def _scheck(rc: int):
    if rc != OK:
        raise TLLError(rc, load().tll_server_last_error().decode(errors="replace"))


class Server:
    """Continuous-batching server (see tll.h): jobs are lenses admitted by
    device-memory footprint; requests are host parameter batches merged
    across jobs into multi-lens launches."""

    def __init__(self, hbm_budget_bytes: int = 0, max_jobs: int = 256,
                 max_vectors_per_launch: int = 16384, max_inflight: int = 2,
                 coalesce: bool = True, use_graph: bool = True, autotune: bool = False):
        cfg = ServerConfig(hbm_budget_bytes, max_jobs, max_vectors_per_launch,
                           max_inflight, 1 if coalesce else 0, 1 if use_graph else 0,
                           1 if autotune else 0)
        h = ctypes.c_void_p()
        _scheck(load().tll_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}
        self._nparam = {}
        self._mass = {}
        self.max_vectors = max_vectors_per_launch

    def open_job(self, image, noise, psf, pixel_scale, sub, x0=None, y0=None,
                 mode=AMP_LINEAR, mass: str = "sie"):
        """Admit a lens; returns its job id, or None when it does not fit
        the budget / slots now (TLL_EBUSY)."""
        img = np.ascontiguousarray(image, dtype=np.float32)
        nse = np.ascontiguousarray(noise, dtype=np.float32)
        k = np.ascontiguousarray(psf, dtype=np.float32)
        ny, nx = img.shape
        x0 = -(nx - 1) * pixel_scale / 2.0 if x0 is None else x0
        y0 = -(ny - 1) * pixel_scale / 2.0 if y0 is None else y0
        g = Grid(nx, ny, pixel_scale, sub, x0, y0)
        jid = ctypes.c_int(-1)
        flags = mode | (MASS_EPL if mass == "epl" else 0)
        rc = load().tll_server_open_job(self._h, img.ctypes.data, nse.ctypes.data,
                                        k.ctypes.data, k.shape[0], ctypes.byref(g),
                                        flags, ctypes.byref(jid))
        if rc == EBUSY:
            return None
        _scheck(rc)
        self._nparam[jid.value] = NPARAM_EPL if mass == "epl" else NPARAM
        self._mass[jid.value] = mass
        return jid.value

    def set_light(self, job: int, comps):
        """Give the job's lens a multi-component light model (a list of
        Comp); its requests then take that model's parameter layout."""
        arr = (Comp * max(1, len(comps)))(*comps)
        _scheck(load().tll_server_set_light(self._h, int(job), arr, len(comps)))
        n = MULTI_HEAD + sum((1 if c.flags & COMP_FREE_SCALE else 0)
                             + (1 if c.flags & COMP_FREE_INDEX else 0) for c in comps)
        epl = self._nparam.get(job) == NPARAM_EPL or self._mass.get(job) == "epl"
        self._nparam[job] = n + (1 if epl else 0) if comps else (
            NPARAM_EPL if epl else NPARAM)

    def close_job(self, job: int) -> bool:
        """True when closed; False while it still has requests in flight."""
        rc = load().tll_server_close_job(self._h, job)
        if rc == EBUSY:
            return False
        _scheck(rc)
        return True

    def submit(self, job: int, params, out=None) -> int:
        """Queue a host batch; returns a request id.  params: float32
        [B, nparam] (numpy or pinned CPU tensor), kept alive until waited."""
        p, keep = _host_ptr(params, np.float32)
        B = int(np.prod(keep.shape)) // self._nparam.get(job, NPARAM)
        if out is None:
            out = np.empty(B, dtype=np.float64)
        o, okeep = _host_ptr(out, np.float64)
        rid = ctypes.c_longlong()
        _scheck(load().tll_server_submit(self._h, job, p, B, o, ctypes.byref(rid)))
        self._keep[rid.value] = (keep, okeep, out)
        return rid.value

    def poll(self, rid: int) -> bool:
        d = ctypes.c_int()
        _scheck(load().tll_server_poll(self._h, rid, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, rid: int, timeout_ms: int = -1):
        """(out array, latency ms); raises TLLError(ETIMEOUT) on timeout."""
        lat = ctypes.c_double()
        _scheck(load().tll_server_wait(self._h, rid, timeout_ms, ctypes.byref(lat)))
        keep = self._keep.pop(rid)
        return keep[2], lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _scheck(load().tll_server_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().tll_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def columns_renderer(pixel_scale, sub, psf, ny, nx, mass: str = "sie"):
    """Render function for the input generator backed by this library
    (blurred unit columns of the truth vector)."""
    dummy = np.zeros((ny, nx), dtype=np.float32)
    lens = Lens(dummy, np.ones((ny, nx), dtype=np.float32), psf, pixel_scale,
                sub, mass=mass)

    def render(params):
        return lens.model_columns(params, blurred=True)

    render.lens = lens
    return render
