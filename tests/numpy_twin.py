"""Second, independent FP64 implementation of the demons iteration in NumPy.

Test infrastructure.  It exists only to cross-check the C oracle on tiny
volumes: it is written vectorised (padding and shifted slices instead of the C
code's per-voxel clamped loops), so a slip in either shows up as a mismatch.
Same readings of the paper as the C oracle: trilinear with clamped coordinates
(Sec. 2.5), central-difference gradient with replicated edges, normalised
Gaussian of radius ceil(3 sigma) applied x, y, z (Sec. 2.5), du = -dr with the
forces of Eqs. (1)-(6), total field smoothed (Sec. 2.1), pyramid by Gaussian
then even samples and fields upsampled as 2 * u(x / 2) (Sec. 2.3).
Arrays are (nz, ny, nx); fields (3, nz, ny, nx) with components (x, y, z).
`register(..., dtype=np.float32)` runs the same steps in single precision: an
independent FP32 implementation whose deviation from the oracle calibrates the
single-precision parity criterion.
"""
from __future__ import annotations

import math

import numpy as np

AXIS = {0: 2, 1: 1, 2: 0}  # field component / spatial axis -> numpy axis


def interp(I, px, py, pz):
    nz, ny, nx = I.shape
    idx, wts = [], []
    for p, n in ((px, nx), (py, ny), (pz, nz)):
        p = np.clip(p, 0.0, n - 1.0)
        lo = np.clip(np.floor(p), 0, max(n - 2, 0)).astype(np.int64)
        hi = np.minimum(lo + 1, n - 1)
        idx.append((lo, hi))
        wts.append(p - lo.astype(p.dtype))
    (x0, x1), (y0, y1), (z0, z1) = idx
    fx, fy, fz = wts
    out = 0.0
    for zi, wz in ((z0, 1 - fz), (z1, fz)):
        for yi, wy in ((y0, 1 - fy), (y1, fy)):
            for xi, wx in ((x0, 1 - fx), (x1, fx)):
                out = out + wz * wy * wx * I[zi, yi, xi]
    return out


def grad(I):
    g = np.empty((3,) + I.shape)
    for c in range(3):
        a = AXIS[c]
        P = np.pad(I, [(1, 1) if ax == a else (0, 0) for ax in range(3)], mode="edge")
        hi = np.take(P, np.arange(2, I.shape[a] + 2), axis=a)
        lo = np.take(P, np.arange(0, I.shape[a]), axis=a)
        g[c] = (hi - lo) / 2.0
    return g


def taps(sigma, dtype=np.float64):
    R = int(math.ceil(3.0 * sigma))
    t = np.arange(-R, R + 1, dtype=np.float64)
    w = np.exp(-t * t / (2.0 * sigma * sigma))
    return (w / w.sum()).astype(dtype), R


def gauss3(I, sigma):
    w, R = taps(sigma, I.dtype)
    out = I
    for c in range(3):  # x, then y, then z
        a = AXIS[c]
        P = np.pad(out, [(R, R) if ax == a else (0, 0) for ax in range(3)], mode="edge")
        n = out.shape[a]
        acc = np.zeros_like(out)
        for q in range(2 * R + 1):
            acc = acc + w[q] * np.take(P, np.arange(q, q + n), axis=a)
        out = acc
    return out


def downsample(I):
    return gauss3(I, 1.0)[::2, ::2, ::2].copy()


def grid(shape, dtype=np.float64):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.astype(dtype), j.astype(dtype), k.astype(dtype)


def upsample(uc, shape):
    i, j, k = grid(shape, uc.dtype)
    return np.stack([2.0 * interp(uc[c], i / 2.0, j / 2.0, k / 2.0) for c in range(3)])


def safe_div(num, den):
    return np.where(den == 0.0, 0.0, num / np.where(den == 0.0, 1.0, den))


def force(variant, d, gs, gm, b, alpha):
    gs2 = np.sum(gs * gs, axis=0)
    gm2 = np.sum(gm * gm, axis=0)
    d2 = d * d
    if variant == 0:
        return safe_div(d * gs, d2 + gs2)
    if variant == 1:
        a = np.sqrt(gs2)
        s = a * a + b * b
        return gs * safe_div(4.0 * d * a * b, (2.0 * d2 + s) * s)
    if variant == 2:
        return safe_div(d * gm, d2 + gm2)
    if variant == 3:
        return safe_div(d * gs, d2 + gs2) + safe_div(d * gm, d2 + gm2)
    if variant == 4:
        return (safe_div(d * gs, alpha * alpha * d2 + gs2) +
                safe_div(d * gm, alpha * alpha * d2 + gm2))
    if variant == 5:
        return safe_div(d * gm, d2 + gm2)
    raise ValueError(variant)


def iterate(variant, S, M, u, sigma, alpha, gs, bm):
    i, j, k = grid(S.shape, S.dtype)
    W = interp(M, i + u[0], j + u[1], k + u[2])
    if variant == 5:
        Ws = interp(S, i - u[0], j - u[1], k - u[2])
        d = W - Ws
        gm = grad(W + Ws)
    else:
        d = W - S
        gm = grad(W) if variant in (2, 3, 4) else np.zeros_like(u)
    du = -force(variant, d, gs, gm, bm, alpha)
    red = np.array([np.sum(d * d), np.sum(np.sqrt(np.sum(du * du, 0))),
                    np.sum(np.sqrt(np.sum(u * u, 0)))])
    v = u + du
    return np.stack([gauss3(v[c], sigma) for c in range(3)]), red


def register(S, M, variant, levels, iters, sigma=1.0, alpha=0.4, dtype=np.float64):
    pyr_s, pyr_m = [S.astype(dtype)], [M.astype(dtype)]
    for _ in range(1, levels):
        pyr_s.append(downsample(pyr_s[-1]))
        pyr_m.append(downsample(pyr_m[-1]))
    u = None
    stats = []
    for lc in range(levels):
        lv = levels - 1 - lc
        Sl, Ml = pyr_s[lv], pyr_m[lv]
        u = np.zeros((3,) + Sl.shape, dtype) if u is None else upsample(u, Sl.shape)
        gs = grad(Sl)
        bm = np.sqrt(np.sum(grad(Ml) ** 2, axis=0))
        for _ in range(iters[lc]):
            u, red = iterate(variant, Sl, Ml, u, sigma, alpha, gs, bm)
            stats.append([red[0] / Sl.size, red[1], red[2]])
    return u, np.array(stats)


def ic_field(h, steps=20):
    i, j, k = grid(h.shape[1:], h.dtype)
    px, py, pz = i.copy(), j.copy(), k.copy()
    for _ in range(steps):
        ax, ay, az = (interp(h[c], px, py, pz) for c in range(3))
        px, py, pz = i + ax, j + ay, k + az
    return np.stack([2.0 * interp(h[c], px, py, pz) for c in range(3)])
