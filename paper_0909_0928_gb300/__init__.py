"""GB300 demons deformable image registration: Python binding of libdir.so.

Thin ctypes layer over the C ABI declared in include/dir.h; it only marshals
arguments (numpy arrays for host memory, torch CUDA tensors for device memory,
torch streams), and every step of the registration runs in the library's CUDA
kernels.  There is no CPU fallback: if libdir.so is missing or fails to load,
importing this package raises.

Functions carry the C names: dir_params_default, dir_create, dir_load,
dir_register, dir_register_async, dir_sync, dir_get_field, dir_get_field_f64,
dir_get_history, dir_get_correlation, dir_warp, dir_destroy, dir_status_string, dir_last_error, dir_version,
dir_register_noalloc, dir_batch_create, dir_batch_run, dir_batch_grouped, dir_batch_destroy,
dir_autotune, dir_check_wait_timeout.
`Registration` wraps a context for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdir.so")

DIR_OK, DIR_EINVAL, DIR_ENOMEM, DIR_ECUDA, DIR_ESTATE, DIR_EUNSUPPORTED, DIR_ETIMEOUT = (
    0, -1, -2, -3, -4, -5, -6)
DIR_MAX_LEVELS = 8
(DIR_PASSIVE, DIR_EVOLVED_PASSIVE, DIR_ACTIVE, DIR_DOUBLE, DIR_ADJUSTED_DOUBLE,
 DIR_INVERSE_CONSISTENT) = range(6)
DIR_F32, DIR_I16, DIR_F16, DIR_BF16, DIR_F64 = range(5)
VARIANTS = {"passive": 0, "evolved_passive": 1, "active": 2, "double": 3, "adjusted_double": 4,
            "inverse_consistent": 5}

# every symbol the C header declares
EXPORTS = ["dir_params_default", "dir_create", "dir_load", "dir_register", "dir_register_async",
           "dir_sync", "dir_get_field", "dir_get_field_f64", "dir_get_history",
           "dir_get_correlation", "dir_warp", "dir_destroy",
           "dir_status_string", "dir_last_error", "dir_version", "dir_register_noalloc",
           "dir_batch_create", "dir_batch_run", "dir_batch_grouped", "dir_batch_destroy",
           "dir_autotune",
           "dir_check_wait_timeout"]


class DirParams(C.Structure):
    _fields_ = [("levels", C.c_int), ("iters", C.c_int * DIR_MAX_LEVELS), ("sigma", C.c_double),
                ("alpha", C.c_double), ("stop_mode", C.c_int), ("eps", C.c_double),
                ("stop_window", C.c_int), ("field_dtype", C.c_int),
                ("init_field", C.c_void_p), ("use_graph", C.c_int), ("timing", C.c_int),
                ("precision", C.c_int), ("fuse", C.c_int), ("plain_kernels", C.c_int),
                ("correlation", C.c_int), ("pdl", C.c_int)]


class DirStats(C.Structure):
    _fields_ = [("levels", C.c_int), ("iters_run", C.c_int * DIR_MAX_LEVELS),
                ("mse_first", C.c_double), ("mse_final", C.c_double),
                ("relnorm_final", C.c_double), ("ms_total", C.c_float),
                ("ms_force_finest", C.c_float), ("ms_smooth_finest", C.c_float),
                ("n_force_finest", C.c_int), ("n_smooth_finest", C.c_int),
                ("voxel_updates", C.c_longlong), ("kernel_launches", C.c_int),
                ("ms_fused_finest", C.c_float), ("n_fused_finest", C.c_int),
                ("schedule_finest", C.c_int)]

    def as_dict(self) -> dict:
        return {"levels": self.levels, "iters_run": list(self.iters_run[: self.levels]),
                "mse_first": self.mse_first, "mse_final": self.mse_final,
                "relnorm_final": self.relnorm_final, "ms_total": self.ms_total,
                "ms_force_finest": self.ms_force_finest,
                "ms_smooth_finest": self.ms_smooth_finest,
                "n_force_finest": self.n_force_finest, "n_smooth_finest": self.n_smooth_finest,
                "voxel_updates": self.voxel_updates, "kernel_launches": self.kernel_launches,
                "ms_fused_finest": self.ms_fused_finest, "n_fused_finest": self.n_fused_finest,
                "schedule_finest": self.schedule_finest}


class DirError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where} failed: {dir_status_string(code)} ({code}) {detail}".strip())


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libdir.so not built at {path}; run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, ip = C.c_void_p, C.c_int
    sig = {
        "dir_params_default": (ip, [C.POINTER(DirParams)]),
        "dir_create": (ip, [C.POINTER(vp), vp, vp, C.POINTER(C.c_int * 3),
                            C.POINTER(C.c_float * 3), ip, ip, ip, C.POINTER(DirParams), vp]),
        "dir_load": (ip, [vp, vp, vp, ip, ip]),
        "dir_register": (ip, [vp, C.POINTER(DirStats)]),
        "dir_register_async": (ip, [vp]),
        "dir_sync": (ip, [vp, C.POINTER(DirStats)]),
        "dir_get_field": (ip, [vp, vp, ip, ip]),
        "dir_get_field_f64": (ip, [vp, vp, ip, ip]),
        "dir_get_history": (ip, [vp, C.POINTER(C.c_double), ip]),
        "dir_get_correlation": (ip, [vp, C.POINTER(C.c_double), ip]),
        "dir_warp": (ip, [vp, vp, vp, ip, ip]),
        "dir_destroy": (None, [vp]),
        "dir_status_string": (C.c_char_p, [ip]),
        "dir_last_error": (C.c_char_p, [vp]),
        "dir_version": (C.c_char_p, []),
        "dir_register_noalloc": (ip, [vp, vp, C.POINTER(C.c_int * 3), ip, C.POINTER(DirParams),
                                      vp, vp, C.POINTER(DirStats)]),
        "dir_batch_create": (ip, [C.POINTER(vp), C.POINTER(vp), ip, ip, ip, vp]),
        "dir_batch_run": (ip, [vp, C.POINTER(C.c_float)]),
        "dir_batch_grouped": (ip, [vp]),
        "dir_batch_destroy": (None, [vp]),
        "dir_autotune": (ip, [vp, ip, C.POINTER(C.c_int)]),
        "dir_check_wait_timeout": (ip, [vp, C.c_double]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


# ------------------------------------------------------------------ helpers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, want_device: bool):
    """Raw pointer of a host numpy array or a contiguous torch tensor."""
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if bool(x.is_cuda) != want_device:
            raise ValueError("tensor on the wrong device for this call")
        return C.c_void_p(x.data_ptr())
    if want_device:
        raise ValueError("device call needs a torch CUDA tensor")
    a = np.asarray(x)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data)


_ITEMSIZE = {DIR_F32: 4, DIR_I16: 2, DIR_F16: 2, DIR_BF16: 2, DIR_F64: 8}


def _check_buffer(x, count: int, itemsize: int, name: str):
    """The library reads or writes exactly `count` elements of `itemsize`
    bytes through the pointer: refuse anything smaller or of another width."""
    if _is_torch(x):
        n, w = int(x.numel()), int(x.element_size())
    else:
        a = np.asarray(x)
        n, w = int(a.size), int(a.itemsize)
    if n != count or w != itemsize:
        raise ValueError(f"{name}: expected {count} elements of {itemsize} bytes, "
                         f"got {n} of {w}")


def _stream_handle(stream) -> C.c_void_p:
    if stream is None:
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(int(stream.cuda_stream))


def _check(code: int, where: str, ctx=None):
    if code < 0:
        glob = where in ("dir_create", "dir_batch_create", "dir_batch_run")
        detail = _lib.dir_last_error(ctx).decode() if ctx is not None or glob else ""
        raise DirError(code, where, detail)
    return code


# ----------------------------------------------------------- C ABI, by name

def dir_status_string(code: int) -> str:
    return _lib.dir_status_string(int(code)).decode()


def dir_version() -> str:
    return _lib.dir_version().decode()


def dir_last_error(ctx=None) -> str:
    return _lib.dir_last_error(ctx).decode()


def dir_params_default(**overrides) -> DirParams:
    p = DirParams()
    _check(_lib.dir_params_default(C.byref(p)), "dir_params_default")
    for k, v in overrides.items():
        if k == "iters":
            vals = list(v) + [0] * (DIR_MAX_LEVELS - len(v))
            p.iters = (C.c_int * DIR_MAX_LEVELS)(*vals)
        elif k == "init_field":
            p.init_field = None if v is None else int(v.data_ptr())
        else:
            setattr(p, k, v)
    return p


def dir_create(static_img, moving_img, dims, spacing_mm=(1.0, 1.0, 1.0), image_dtype=DIR_F32,
               inputs_on_device=False, variant=DIR_PASSIVE, params: DirParams | None = None,
               stream=None):
    """Returns an opaque context handle (c_void_p).  Images: (nz, ny, nx) float32,
    numpy on the host or torch CUDA tensors with inputs_on_device=True."""
    out = C.c_void_p()
    d = (C.c_int * 3)(*[int(x) for x in dims])
    s = (C.c_float * 3)(*[float(x) for x in spacing_mm])
    n = d[0] * d[1] * d[2]
    if n > 0 and int(image_dtype) in (DIR_F32, DIR_I16):  # the image storage types
        _check_buffer(static_img, n, _ITEMSIZE[int(image_dtype)], "static_img")
        _check_buffer(moving_img, n, _ITEMSIZE[int(image_dtype)], "moving_img")
    rc = _lib.dir_create(C.byref(out), _ptr(static_img, inputs_on_device),
                         _ptr(moving_img, inputs_on_device), C.byref(d), C.byref(s),
                         int(image_dtype), int(bool(inputs_on_device)), int(variant),
                         C.byref(params) if params is not None else None,
                         _stream_handle(stream))
    _check(rc, "dir_create")
    return out


def dir_load(ctx, static_img, moving_img, image_dtype=DIR_F32, on_device=False):
    _check(_lib.dir_load(ctx, _ptr(static_img, on_device), _ptr(moving_img, on_device),
                         int(image_dtype), int(bool(on_device))), "dir_load", ctx)


def dir_register(ctx) -> DirStats:
    st = DirStats()
    _check(_lib.dir_register(ctx, C.byref(st)), "dir_register", ctx)
    return st


def dir_register_async(ctx):
    _check(_lib.dir_register_async(ctx), "dir_register_async", ctx)


def dir_sync(ctx) -> DirStats:
    st = DirStats()
    _check(_lib.dir_sync(ctx, C.byref(st)), "dir_sync", ctx)
    return st


def dir_get_field(ctx, out, in_mm=False, out_on_device=False):
    """Fills `out` (3*N float32: numpy array, or torch CUDA tensor if out_on_device)."""
    _check(_lib.dir_get_field(ctx, _ptr(out, out_on_device), int(bool(in_mm)),
                              int(bool(out_on_device))), "dir_get_field", ctx)
    return out


def dir_get_field_f64(ctx, out, in_mm=False, out_on_device=False):
    """As dir_get_field with a float64 `out` (numpy or torch CUDA tensor)."""
    _check(_lib.dir_get_field_f64(ctx, _ptr(out, out_on_device), int(bool(in_mm)),
                                  int(bool(out_on_device))), "dir_get_field_f64", ctx)
    return out


def dir_get_history(ctx, max_iters: int) -> np.ndarray:
    buf = np.zeros((max(int(max_iters), 0), 3), dtype=np.float64)
    n = _check(_lib.dir_get_history(ctx, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                    int(max_iters)), "dir_get_history", ctx)
    return buf[:n]


def dir_get_correlation(ctx, max_iters: int) -> np.ndarray:
    """Per-iteration correlation coefficient of the warped image with S
    (contexts created with correlation = 1 or stop_mode = 2)."""
    buf = np.zeros(max(int(max_iters), 0), dtype=np.float64)
    n = _check(_lib.dir_get_correlation(ctx, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                        int(max_iters)), "dir_get_correlation", ctx)
    return buf[:n]


def dir_warp(ctx, img_in, img_out, dtype=DIR_F32, on_device=False):
    _check(_lib.dir_warp(ctx, _ptr(img_in, on_device), _ptr(img_out, on_device), int(dtype),
                         int(bool(on_device))), "dir_warp", ctx)
    return img_out


def dir_register_noalloc(static_img, moving_img, dims, variant=DIR_PASSIVE,
                         params: DirParams | None = None, field_out=None, stream=None) -> DirStats:
    """Registration without device allocation: float32 torch CUDA tensors of
    nx*ny*nz voxels in, the static-grid field (3*N float32, voxels) written
    into `field_out`, scratch from the library's static 48 MiB device array."""
    if field_out is None:
        raise ValueError("dir_register_noalloc: field_out (3*N float32 CUDA tensor) is required")
    st = DirStats()
    d = (C.c_int * 3)(*[int(x) for x in dims])
    n = d[0] * d[1] * d[2]
    _check_buffer(static_img, n, 4, "static_img")
    _check_buffer(moving_img, n, 4, "moving_img")
    _check_buffer(field_out, 3 * n, 4, "field_out")
    for name, t in (("static_img", static_img), ("moving_img", moving_img),
                    ("field_out", field_out)):
        if not _is_torch(t) or not str(t.dtype).endswith("float32"):
            raise ValueError(f"dir_register_noalloc: {name} must be a float32 torch CUDA tensor")
    rc = _lib.dir_register_noalloc(_ptr(static_img, True), _ptr(moving_img, True), C.byref(d),
                                   int(variant), C.byref(params) if params is not None else None,
                                   _ptr(field_out, True), _stream_handle(stream), C.byref(st))
    if rc < 0:
        raise DirError(rc, "dir_register_noalloc", _lib.dir_last_error(None).decode())
    return st


def dir_destroy(ctx):
    if ctx is not None:
        _lib.dir_destroy(ctx)


def dir_check_wait_timeout(stream=None, limit_ms: float = 100.0) -> int:
    """Runs the library's bounded device-side wait on a barrier that nothing
    completes and returns the status code (DIR_ETIMEOUT when the wait gave up
    as designed)."""
    return int(_lib.dir_check_wait_timeout(_stream_handle(stream), float(limit_ms)))


DIR_BATCH_BRANCHES = 1


def dir_batch_create(ctxs, branches: int = 8, stream=None, grouped: bool = True):
    """One captured CUDA graph that runs the registrations of `ctxs` (contexts
    from dir_create): grouped launches per iteration where the contexts allow
    it (and `grouped`), else each registration on one of `branches`
    concurrent branches."""
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    out = C.c_void_p()
    flags = 0 if grouped else DIR_BATCH_BRANCHES
    _check(_lib.dir_batch_create(C.byref(out), arr, len(ctxs), int(branches), flags,
                                 _stream_handle(stream)), "dir_batch_create")
    return out


def dir_batch_grouped(batch) -> bool:
    """True if the batch was captured in the grouped form."""
    return int(_lib.dir_batch_grouped(batch)) == 1


def dir_batch_run(batch) -> float:
    """Replay the batch and wait for it; returns its device time in ms."""
    ms = C.c_float()
    _check(_lib.dir_batch_run(batch, C.byref(ms)), "dir_batch_run")
    return float(ms.value)


def dir_batch_destroy(batch):
    if batch is not None:
        _lib.dir_batch_destroy(batch)


def dir_autotune(ctx, reps: int = 5, levels: int = DIR_MAX_LEVELS) -> list:
    """Pick per-level force brick depths and smoothing z chunks by timing them;
    returns [(depth, zchunk)] per level, finest first (zchunk 0 = one wave)."""
    shapes = (C.c_int * (2 * DIR_MAX_LEVELS))()
    _check(_lib.dir_autotune(ctx, int(reps), shapes), "dir_autotune", ctx)
    return [(shapes[2 * l], shapes[2 * l + 1]) for l in range(levels)]


# --------------------------------------------------------------- convenience

class Registration:
    """Owns one dir_ctx.  Host arrays in and out unless device tensors are given."""

    def __init__(self, static_img, moving_img, spacing_mm=(1.0, 1.0, 1.0), variant=DIR_PASSIVE,
                 params: DirParams | None = None, stream=None):
        on_dev = _is_torch(static_img) and bool(static_img.is_cuda)
        nz, ny, nx = static_img.shape
        self.dims = (nx, ny, nz)
        self.spacing = tuple(float(s) for s in spacing_mm)
        self.variant = int(variant)
        self.params = params if params is not None else dir_params_default()
        self.ctx = dir_create(static_img, moving_img, self.dims, spacing_mm, DIR_F32, on_dev,
                              variant, self.params, stream)
        self.stats = None

    def register(self) -> DirStats:
        self.stats = dir_register(self.ctx)
        return self.stats

    def field(self, in_mm=False, out=None, f64=False):
        nx, ny, nz = self.dims
        if out is None:
            out = np.empty((3, nz, ny, nx), dtype=np.float64 if f64 else np.float32)
        on_dev = _is_torch(out) and bool(out.is_cuda)
        is64 = (str(out.dtype).endswith("float64"))
        _check_buffer(out, 3 * nx * ny * nz, 8 if is64 else 4, "field out")
        (dir_get_field_f64 if is64 else dir_get_field)(self.ctx, out, in_mm, on_dev)
        return out

    def history(self) -> np.ndarray:
        return dir_get_history(self.ctx, sum(self.params.iters[: self.params.levels]))

    def correlation(self) -> np.ndarray:
        return dir_get_correlation(self.ctx, sum(self.params.iters[: self.params.levels]))

    def warp(self, img, out=None):
        on_dev = _is_torch(img) and bool(img.is_cuda)
        if out is None:
            out = np.empty_like(img) if not on_dev else img.new_empty(img.shape)
        nx, ny, nz = self.dims
        _check_buffer(img, nx * ny * nz, 4, "warp input")
        _check_buffer(out, nx * ny * nz, 4, "warp output")
        dir_warp(self.ctx, img, out, DIR_F32, on_dev)
        return out

    def close(self):
        if self.ctx is not None:
            dir_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
