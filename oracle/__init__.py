"""FP64 CPU oracle for demons registration -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never does, and shares no code with it.

The arithmetic lives in ``demons_oracle.c`` (plain C, doubles, written from the
paper's equations); this module only marshals numpy arrays through ctypes.
Volumes are numpy arrays of shape (nz, ny, nx), C order (x fastest); fields are
(3, nz, ny, nx), components (x, y, z), in voxel units.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build_mod

_LIBS: dict[bool, C.CDLL] = {}

PASSIVE, EVOLVED_PASSIVE, ACTIVE, DOUBLE, ADJUSTED_DOUBLE, INVERSE_CONSISTENT = range(6)
VARIANT_NAMES = ["passive", "evolved_passive", "active", "double", "adjusted_double",
                 "inverse_consistent"]

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def _lib(threaded: bool = False) -> C.CDLL:
    if threaded not in _LIBS:
        path = _build_mod.library_path(threaded)
        if not os.path.exists(path):
            _build_mod.build()
        lib = C.CDLL(path)
        lib.or_interp.restype = C.c_double
        lib.or_interp.argtypes = [_dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                  C.c_double]
        lib.or_interp_points.restype = None
        lib.or_interp_points.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp,
                                         C.c_int64]
        lib.or_grad.restype = None
        lib.or_grad.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
        lib.or_gauss_taps.restype = C.c_int
        lib.or_gauss_taps.argtypes = [C.c_double, _dp, C.c_int]
        lib.or_gauss3.restype = C.c_int
        lib.or_gauss3.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_int, C.c_double]
        lib.or_downsample.restype = C.c_int
        lib.or_downsample.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp]
        lib.or_upsample.restype = None
        lib.or_upsample.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp, C.c_int, C.c_int,
                                    C.c_int]
        lib.or_warp.restype = None
        lib.or_warp.argtypes = [_dp, _dp, _dp, _dp, C.c_int, C.c_int, C.c_int, C.c_double, _dp]
        lib.or_force_arrays.restype = None
        lib.or_force_arrays.argtypes = [C.c_int, C.c_double] + [_dp] * 8 + [_dp] * 3 + [C.c_int64]
        lib.or_iterate.restype = C.c_int
        lib.or_iterate.argtypes = ([C.c_int, C.c_double, C.c_double] + [_dp] * 6 + [_dp] * 3 +
                                   [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp])
        lib.or_correlation.restype = C.c_double
        lib.or_correlation.argtypes = [_dp, _dp, C.c_int64]
        lib.or_ic_field.restype = None
        lib.or_ic_field.argtypes = [_dp, _dp, _dp, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
        lib.or_register.restype = C.c_int
        lib.or_register.argtypes = ([_dp, _dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                     C.c_double, C.c_int, _ip, C.c_int, C.c_double, C.c_int, _dp,
                                     _dp, _dp, _ip, _dp, C.c_double, C.c_uint64, _dp])
        lib.or_num_threads.restype = C.c_int
        lib.or_num_threads.argtypes = []
        _LIBS[threaded] = lib
    return _LIBS[threaded]


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _dims(vol: np.ndarray) -> tuple[int, int, int]:
    nz, ny, nx = vol.shape
    return nx, ny, nz


def num_threads(threaded: bool = True) -> int:
    return int(_lib(threaded).or_num_threads())


def interp(vol, px, py, pz) -> np.ndarray:
    """Trilinear value of `vol` at continuous voxel points (arrays of equal shape)."""
    v = _f64(vol)
    px, py, pz = (_f64(np.broadcast_to(a, np.broadcast(px, py, pz).shape)) for a in (px, py, pz))
    out = np.empty(px.shape, dtype=np.float64)
    nx, ny, nz = _dims(v)
    _lib().or_interp_points(_p(v), nx, ny, nz, _p(px), _p(py), _p(pz), _p(out), out.size)
    return out


def grad(vol) -> np.ndarray:
    v = _f64(vol)
    g = np.empty((3,) + v.shape, dtype=np.float64)
    nx, ny, nz = _dims(v)
    _lib().or_grad(_p(v), nx, ny, nz, _p(g[0]), _p(g[1]), _p(g[2]))
    return g


def gauss_taps(sigma: float) -> np.ndarray:
    w = np.zeros(129, dtype=np.float64)
    r = _lib().or_gauss_taps(float(sigma), _p(w), 129)
    if r < 0:
        raise ValueError("bad sigma")
    return w[: 2 * r + 1].copy()


def gauss3(vol, sigma: float = 1.0, threaded: bool = False) -> np.ndarray:
    v = _f64(vol)
    out = np.empty_like(v)
    nx, ny, nz = _dims(v)
    if _lib(threaded).or_gauss3(_p(v), _p(out), nx, ny, nz, float(sigma)) != 0:
        raise ValueError("gauss3 failed")
    return out


def downsample(vol) -> np.ndarray:
    v = _f64(vol)
    nx, ny, nz = _dims(v)
    out = np.empty(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2), dtype=np.float64)
    if _lib().or_downsample(_p(v), nx, ny, nz, out.ctypes.data_as(_dp)) != 0:
        raise ValueError("downsample failed")
    return out


def upsample(coarse, fine_dims) -> np.ndarray:
    """Field or single component: coarse (..., cz, cy, cx) -> fine (..., nz, ny, nx)."""
    c = _f64(coarse)
    nx, ny, nz = fine_dims
    lead = c.shape[:-3]
    cz, cy, cx = c.shape[-3:]
    cf = c.reshape((-1, cz, cy, cx))
    out = np.empty((cf.shape[0], nz, ny, nx), dtype=np.float64)
    for q in range(cf.shape[0]):
        src = np.ascontiguousarray(cf[q])
        _lib().or_upsample(_p(src), cx, cy, cz, _p(out[q]), nx, ny, nz)
    return out.reshape(lead + (nz, ny, nx))


def warp(vol, u, sign: float = 1.0) -> np.ndarray:
    """W(x) = vol(x + sign * u(x))."""
    v = _f64(vol)
    u = _f64(u)
    out = np.empty_like(v)
    nx, ny, nz = _dims(v)
    _lib().or_warp(_p(v), _p(u[0]), _p(u[1]), _p(u[2]), nx, ny, nz, float(sign), _p(out))
    return out


def force(variant: int, d, gs, gm=None, b=None, alpha: float = 1.0) -> np.ndarray:
    """Demons force dr (3, ...) per voxel for intensity differences d (...),
    static gradient gs (3, ...), moving gradient gm (3, ...), |grad M| b (...)."""
    d = _f64(d)
    n = d.size
    gs = _f64(gs).reshape(3, n) if gs is not None else np.zeros((3, n))
    gm = _f64(gm).reshape(3, n) if gm is not None else np.zeros((3, n))
    gs = np.ascontiguousarray(gs)
    gm = np.ascontiguousarray(gm)
    bb = _f64(b).reshape(n) if b is not None else np.zeros(n)
    out = np.empty((3, n), dtype=np.float64)
    _lib().or_force_arrays(int(variant), float(alpha), _p(d.reshape(n)), _p(gs[0]), _p(gs[1]),
                           _p(gs[2]), _p(gm[0]), _p(gm[1]), _p(gm[2]), _p(bb), _p(out[0]),
                           _p(out[1]), _p(out[2]), n)
    return out.reshape((3,) + d.shape)


def correlation(a, b) -> float:
    """Pearson correlation coefficient of two images (NaN if one is constant)."""
    a = _f64(a).ravel()
    b = _f64(b).ravel()
    if a.size != b.size:
        raise ValueError("images of different sizes")
    return float(_lib().or_correlation(_p(a), _p(b), a.size))


def iterate(variant: int, S, M, u, sigma: float = 1.0, alpha: float = 1.0, corr: bool = False):
    """One iteration at one level.  Returns (new field, [sum d^2, sum|du|, sum|u|]),
    plus the correlation coefficient of the warped image(s) if corr."""
    S = _f64(S)
    M = _f64(M)
    u = _f64(u).copy()
    nx, ny, nz = _dims(S)
    gs = grad(S)
    bm = None
    if variant == EVOLVED_PASSIVE:
        bm = np.ascontiguousarray(np.sqrt(np.sum(grad(M) ** 2, axis=0)))
    work = np.empty((8,) + S.shape, dtype=np.float64)
    red = np.zeros(3, dtype=np.float64)
    rho = np.zeros(1, dtype=np.float64)
    rc = _lib().or_iterate(int(variant), float(alpha), float(sigma), _p(S), _p(M), _p(gs[0]),
                           _p(gs[1]), _p(gs[2]), _p(bm) if bm is not None else None, _p(u[0]),
                           _p(u[1]), _p(u[2]), nx, ny, nz, _p(work), _p(red),
                           _p(rho) if corr else None)
    if rc != 0:
        raise ValueError(f"or_iterate failed: {rc}")
    return (u, red, float(rho[0])) if corr else (u, red)


def ic_field(h) -> np.ndarray:
    h = _f64(h)
    nz, ny, nx = h.shape[1:]
    out = np.empty_like(h)
    _lib().or_ic_field(_p(h[0]), _p(h[1]), _p(h[2]), nx, ny, nz, _p(out[0]), _p(out[1]),
                       _p(out[2]))
    return out


ROUND32 = 0xFFFFFFFFFFFFFFFF  # probe_seed: single-precision storage of the state


def register(S, M, variant: int = PASSIVE, levels: int = 1, iters=(50,), sigma: float = 1.0,
             alpha: float = 0.4, stop_mode: int = 0, eps: float = 1e-4, stop_window: int = 10,
             init=None, threaded: bool = True, return_raw: bool = False,
             probe_rel: float = 0.0, probe_seed: int = 0, return_corr: bool = False):
    """Whole registration.  `iters` lists iterations per level, coarsest first.

    Returns dict(u=(3, nz, ny, nx) field in voxels, stats=(n, 3) per-iteration
    [MSE, sum|du|, sum|u|], iters_run=list per level[, raw=iterated field]
    [, corr=(n,) correlation coefficient of the warped image with S per
    iteration, before its update (Eq. 6: of the two warped images)]).
    stop_mode 2 stops a level on the correlation instead of the relative norm.
    probe_rel > 0 injects relative noise of that size into the warped images
    and the smoothed field every iteration (keyed by probe_seed): a probe of
    how strongly the iteration amplifies rounding, not part of the method.
    probe_seed = ROUND32 (with any probe_rel > 0) instead stores the state in
    single precision (pyramid images, the field before and after smoothing and
    after upsampling, the warped images relative to S).
    """
    S = _f64(S)
    M = _f64(M)
    nx, ny, nz = _dims(S)
    it = (C.c_int * 8)(*([int(x) for x in iters] + [0] * (8 - len(iters))))
    total = sum(int(x) for x in iters)
    stats = np.zeros((max(total, 1), 3), dtype=np.float64)
    run = (C.c_int * 8)()
    u = np.empty((3,) + S.shape, dtype=np.float64)
    raw = np.empty_like(u) if return_raw else None
    want_corr = return_corr or int(stop_mode) == 2
    corr = np.full(max(total, 1), np.nan) if want_corr else None
    ini = _f64(init) if init is not None else None
    rc = _lib(threaded).or_register(_p(S), _p(M), nx, ny, nz, int(variant), float(alpha),
                                    float(sigma), int(levels), it, int(stop_mode), float(eps),
                                    int(stop_window), _p(ini) if ini is not None else None,
                                    _p(u), _p(stats), run, _p(raw) if raw is not None else None,
                                    float(probe_rel), int(probe_seed) & 0xFFFFFFFFFFFFFFFF,
                                    _p(corr) if corr is not None else None)
    if rc != 0:
        raise ValueError(f"or_register failed: {rc}")
    runs = [int(run[i]) for i in range(levels)]
    out = {"u": u, "stats": stats[: sum(runs)], "iters_run": runs}
    if return_raw:
        out["raw"] = raw
    if want_corr:
        out["corr"] = corr[: sum(runs)]
    return out
