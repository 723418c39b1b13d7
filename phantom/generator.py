"""Seeded synthetic inputs for demons registration: lung phantoms and blob pairs.

This module only *generates inputs*.  It holds none of the registration
arithmetic (no trilinear interpolation, no gradient, no demons force, no
Gaussian smoothing of volumes): every image value is an analytic function of a
continuous position, evaluated directly.  Both the FP64 oracle and the CUDA
library consume the arrays it returns, so they see identical bytes.

The phantom stands in for the paper's thoracic 4DCT cases (Sec. 3.1, Table 1:
256x256x94..112 voxels, 0.97-1.16 mm in-plane, 2.5 mm slices, landmark
displacements of 4-9 mm), which are not available here.

Randomness comes from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so that a
seed gives the same volumes on any machine and numpy version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class SplitMix64Stream:
    """Counter-based stream: draw i of stream (seed, sid) is mix(key + (i+1)*gamma).

    key = mix(seed * gamma + sid), so separate stream ids give unrelated draws.
    """

    def __init__(self, seed: int, sid: int = 0):
        with np.errstate(over="ignore"):
            s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
            self.key = _mix64(s * _GAMMA + np.uint64(sid & 0xFFFFFFFFFFFFFFFF))[0]
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.key + i * _GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """Uniform on [lo, hi) from the top 53 bits."""
        x = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * x

    def normal(self, n: int) -> np.ndarray:
        """Standard normal by the Box-Muller transform."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 lies in (0, 1]
        t = 2.0 * math.pi * u2
        return np.concatenate([r * np.cos(t), r * np.sin(t)])[:n]

    def unit_vectors(self, n: int) -> np.ndarray:
        v = self.normal(3 * n).reshape(n, 3)
        return v / np.linalg.norm(v, axis=1, keepdims=True)


# --------------------------------------------------------------------------
# Lung phantom
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class PhantomSpec:
    """Shape of one synthetic 4DCT-like pair (static = exhale, moving = inhale)."""

    dims: tuple[int, int, int]                 # (nx, ny, nz) voxels, x fastest
    spacing: tuple[float, float, float]        # mm per voxel
    seed: int
    a_max_mm: float                            # largest RBF displacement amplitude
    compression: float                         # superior-inferior compression fraction
    compression_region: str = "global"         # "global" (from the apex) or "lower" lung
    n_vessels: int = 40
    n_rbf: int = 8
    noise_hu: float = 20.0
    n_landmarks: int = 1100
    rbf_width_mm: tuple[float, float] = (15.0, 30.0)


# The two named workloads.  The small one is the oracle-sized case; the full one
# has the shape of the paper's clinical cases.
SMALL = PhantomSpec(dims=(64, 64, 32), spacing=(1.0, 1.0, 2.5), seed=1, a_max_mm=4.0,
                    compression=0.05, compression_region="global", n_landmarks=300)
FULL = PhantomSpec(dims=(256, 256, 100), spacing=(0.9, 0.9, 2.5), seed=2, a_max_mm=12.0,
                   compression=0.20, compression_region="lower", n_landmarks=1100)

HU_AIR, HU_BODY, HU_LUNG, HU_VESSEL = -1000.0, 0.0, -850.0, 40.0


@dataclass
class _Geometry:
    spec: PhantomSpec
    body_c: np.ndarray            # centres / semi-axes in voxel units
    body_a: np.ndarray
    lung_c: list
    lung_a: np.ndarray
    seg_a: np.ndarray             # (S, 3) segment start, mm
    seg_b: np.ndarray             # (S, 3) segment end, mm
    seg_r: np.ndarray             # (S,) radius, mm
    bifurcations: np.ndarray      # (B, 3) mm
    ends: np.ndarray              # (E, 3) mm
    rbf_c: np.ndarray             # (R, 3) mm
    rbf_w: np.ndarray             # (R,) mm
    rbf_v: np.ndarray             # (R, 3) mm amplitude vectors
    z_ref_mm: float = 0.0
    edge_mm: float = 0.5
    extra: dict = field(default_factory=dict)


def _ellipsoid_occupancy(p_vox: np.ndarray, c: np.ndarray, a: np.ndarray, sp: np.ndarray,
                         edge_mm: float) -> np.ndarray:
    """Soft inside-indicator of an ellipsoid (voxel-unit centre and semi-axes)."""
    q = (p_vox - c) / a
    r = np.sqrt(np.sum(q * q, axis=-1))
    dist_mm = np.sqrt(np.sum(((p_vox - c) * sp) ** 2, axis=-1))
    # signed distance along the ray from the centre: |p - c| (1 - 1/r)
    with np.errstate(divide="ignore", invalid="ignore"):
        sd = np.where(r > 0, dist_mm * (1.0 - 1.0 / np.maximum(r, 1e-12)), -1e9)
    return 1.0 / (1.0 + np.exp(np.clip(sd / edge_mm, -60, 60)))


def _inside_lung(p_vox: np.ndarray, g: _Geometry, shrink: float = 0.9) -> bool:
    for c in g.lung_c:
        q = (p_vox - c) / (g.lung_a * shrink)
        if float(np.sum(q * q)) <= 1.0:
            return True
    return False


def _build_geometry(spec: PhantomSpec) -> _Geometry:
    nx, ny, nz = spec.dims
    sp = np.asarray(spec.spacing, dtype=np.float64)
    n = np.array([nx, ny, nz], dtype=np.float64)
    centre = (n - 1.0) / 2.0
    body_a = np.array([0.46 * nx, 0.38 * ny, 0.49 * nz])
    lung_a = np.array([0.16 * nx, 0.26 * ny, 0.42 * nz])
    lung_c = [np.array([(0.5 - 0.2) * (nx - 1), centre[1], centre[2]]),
              np.array([(0.5 + 0.2) * (nx - 1), centre[1], centre[2]])]
    g = _Geometry(spec=spec, body_c=centre, body_a=body_a, lung_c=lung_c, lung_a=lung_a,
                  seg_a=np.zeros((0, 3)), seg_b=np.zeros((0, 3)), seg_r=np.zeros(0),
                  bifurcations=np.zeros((0, 3)), ends=np.zeros((0, 3)),
                  rbf_c=np.zeros((0, 3)), rbf_w=np.zeros(0), rbf_v=np.zeros((0, 3)),
                  edge_mm=0.5 * float(min(sp)))

    rng = SplitMix64Stream(spec.seed, sid=1)

    def sample_in_lung() -> np.ndarray:
        for _ in range(10000):
            li = int(rng.uniform(1)[0] * 2) % 2
            q = rng.uniform(3, -1.0, 1.0)
            if float(np.sum(q * q)) <= 1.0:
                return lung_c[li] + 0.85 * q * lung_a
        raise RuntimeError("could not sample a point in the lungs")

    seg_a, seg_b, seg_r, bif, ends = [], [], [], [], []
    step_mm = 4.0

    def walk(start_mm, direction, n_steps, radius_mm):
        pts = [start_mm]
        d = direction / np.linalg.norm(direction)
        for _ in range(n_steps):
            d = d + 0.45 * rng.normal(3)
            d = d / np.linalg.norm(d)
            nxt = pts[-1] + step_mm * d
            if not _inside_lung(nxt / sp, g):
                break
            pts.append(nxt)
        for a, b in zip(pts[:-1], pts[1:]):
            seg_a.append(a)
            seg_b.append(b)
            seg_r.append(radius_mm)
        return pts

    for _ in range(spec.n_vessels):
        start = sample_in_lung() * sp
        d0 = rng.unit_vectors(1)[0]
        n_steps = 8 + int(rng.uniform(1)[0] * 10)
        radius = float(rng.uniform(1, 1.0, 3.0)[0]) * float(sp[0])
        pts = walk(start, d0, n_steps, radius)
        if len(pts) >= 2:
            ends.append(pts[-1])
        # about half of the vessels branch once
        if rng.uniform(1)[0] < 0.5 and len(pts) >= 4:
            at = 1 + int(rng.uniform(1)[0] * (len(pts) - 2))
            base = pts[at]
            parent = pts[at + 1] - pts[at - 1]
            side = rng.unit_vectors(1)[0]
            side = side - np.dot(side, parent) * parent / max(np.dot(parent, parent), 1e-12)
            nd = parent / np.linalg.norm(parent) + side / max(np.linalg.norm(side), 1e-12)
            bpts = walk(base, nd, max(3, n_steps // 2), 0.7 * radius)
            if len(bpts) >= 2:
                bif.append(base)
                ends.append(bpts[-1])

    g.seg_a = np.array(seg_a, dtype=np.float64).reshape(-1, 3)
    g.seg_b = np.array(seg_b, dtype=np.float64).reshape(-1, 3)
    g.seg_r = np.array(seg_r, dtype=np.float64)
    g.bifurcations = np.array(bif, dtype=np.float64).reshape(-1, 3)
    g.ends = np.array(ends, dtype=np.float64).reshape(-1, 3)

    # deformation parameters: Gaussian RBFs centred in the lungs
    rbf = SplitMix64Stream(spec.seed, sid=2)
    g.rbf_c = np.array([sample_in_lung() * sp for _ in range(spec.n_rbf)]).reshape(-1, 3)
    lo, hi = spec.rbf_width_mm
    g.rbf_w = rbf.uniform(spec.n_rbf, lo, hi)
    amp = rbf.uniform(spec.n_rbf, 0.5, 1.0) * spec.a_max_mm
    g.rbf_v = rbf.unit_vectors(spec.n_rbf) * amp[:, None]
    # the RBFs overlap, so rescale their sum to peak at a_max_mm over the lungs
    probe = np.array([sample_in_lung() for _ in range(512)]) * sp
    rbf_only = np.zeros_like(probe)
    for c, w, a in zip(g.rbf_c, g.rbf_w, g.rbf_v):
        rbf_only += np.exp(-np.sum((probe - c) ** 2, axis=-1) / (2.0 * w * w))[:, None] * a
    peak = float(np.max(np.linalg.norm(rbf_only, axis=1)))
    if peak > 0:
        g.rbf_v = g.rbf_v * (spec.a_max_mm / peak)
    lung_top = (centre[2] + lung_a[2]) * sp[2]
    g.z_ref_mm = float(lung_top if spec.compression_region == "global" else centre[2] * sp[2])
    return g


def backward_map_mm(g: _Geometry, p_mm: np.ndarray) -> np.ndarray:
    """v*(y) in mm: the moving image is M(y) = S_clean(y + v*(y)).

    A sum of Gaussian RBFs plus a superior-inferior stretch of the lung below
    z_ref (inhale: the moving image's lower lung reaches further down).
    """
    v = np.zeros_like(p_mm)
    for c, w, a in zip(g.rbf_c, g.rbf_w, g.rbf_v):
        r2 = np.sum((p_mm - c) ** 2, axis=-1)
        v += np.exp(-r2 / (2.0 * w * w))[..., None] * a
    below = np.maximum(g.z_ref_mm - p_mm[..., 2], 0.0)
    v[..., 2] += g.spec.compression * below
    return v


def _clean_image(g: _Geometry, p_vox: np.ndarray) -> np.ndarray:
    """Noise-free phantom intensity (HU) at continuous voxel positions (..., 3)."""
    sp = np.asarray(g.spec.spacing)
    body = _ellipsoid_occupancy(p_vox, g.body_c, g.body_a, sp, g.edge_mm)
    lung = np.maximum(_ellipsoid_occupancy(p_vox, g.lung_c[0], g.lung_a, sp, g.edge_mm),
                      _ellipsoid_occupancy(p_vox, g.lung_c[1], g.lung_a, sp, g.edge_mm))
    img = HU_AIR * (1.0 - body) + HU_BODY * body
    img = img * (1.0 - lung) + HU_LUNG * lung
    ves = _vessel_occupancy(g, p_vox)
    ves = ves * lung
    return img * (1.0 - ves) + HU_VESSEL * ves


def _vessel_occupancy(g: _Geometry, p_vox: np.ndarray) -> np.ndarray:
    """Max over tube segments of a soft inside-indicator, evaluated per segment
    only where the points can be near it (bounding box in point-index space)."""
    sp = np.asarray(g.spec.spacing)
    shape = p_vox.shape[:-1]
    occ = np.zeros(shape, dtype=np.float64)
    if g.seg_a.shape[0] == 0:
        return occ
    p_mm = p_vox * sp
    flat = p_mm.reshape(-1, 3)
    occ_flat = occ.reshape(-1)
    pad = g.seg_r.max() + 8.0 * g.edge_mm
    if len(shape) == 3:
        # points form a (possibly deformed) grid: restrict each segment to the
        # index box whose points lie inside the segment's padded bounding box
        nzp = shape[0]
        zmin = p_mm[..., 2].reshape(nzp, -1)
        zlo, zhi = zmin.min(axis=1), zmin.max(axis=1)
        ylo = p_mm[..., 1].min(axis=(0, 2))
        yhi = p_mm[..., 1].max(axis=(0, 2))
        xlo = p_mm[..., 0].min(axis=(0, 1))
        xhi = p_mm[..., 0].max(axis=(0, 1))
        for a, b, r in zip(g.seg_a, g.seg_b, g.seg_r):
            bl = np.minimum(a, b) - pad
            bh = np.maximum(a, b) + pad
            ks = np.nonzero((zhi >= bl[2]) & (zlo <= bh[2]))[0]
            js = np.nonzero((yhi >= bl[1]) & (ylo <= bh[1]))[0]
            is_ = np.nonzero((xhi >= bl[0]) & (xlo <= bh[0]))[0]
            if ks.size == 0 or js.size == 0 or is_.size == 0:
                continue
            sl = (slice(ks[0], ks[-1] + 1), slice(js[0], js[-1] + 1), slice(is_[0], is_[-1] + 1))
            sub = p_mm[sl]
            o = _segment_occupancy(sub, a, b, r, g.edge_mm)
            occ[sl] = np.maximum(occ[sl], o)
        return occ
    for a, b, r in zip(g.seg_a, g.seg_b, g.seg_r):
        o = _segment_occupancy(flat, a, b, r, g.edge_mm)
        np.maximum(occ_flat, o, out=occ_flat)
    return occ


def _segment_occupancy(p_mm, a, b, r, edge_mm):
    ab = b - a
    t = np.clip(np.sum((p_mm - a) * ab, axis=-1) / max(float(np.dot(ab, ab)), 1e-12), 0.0, 1.0)
    closest = a + t[..., None] * ab
    dist = np.sqrt(np.sum((p_mm - closest) ** 2, axis=-1))
    return 1.0 / (1.0 + np.exp(np.clip((dist - r) / edge_mm, -60, 60)))


def _grid_points(dims) -> np.ndarray:
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return np.stack([i, j, k], axis=-1)  # (nz, ny, nx, 3), (x, y, z) order


def true_field_mm(g: _Geometry, p_vox: np.ndarray, tol_mm: float = 1e-10,
                  max_steps: int = 2000) -> np.ndarray:
    """Static-grid field u_true(p) in mm, solving u = -v*(p + u) (so that
    M(p + u) = S_clean(p)), by damped fixed-point steps to tol_mm."""
    sp = np.asarray(g.spec.spacing)
    p_mm = np.asarray(p_vox, dtype=np.float64) * sp
    u = np.zeros_like(p_mm)
    for _ in range(max_steps):
        nu = -backward_map_mm(g, p_mm + u)
        step = nu - u
        u = u + 0.5 * step
        if float(np.max(np.abs(step))) < tol_mm:
            break
    return u


def _landmarks(g: _Geometry, n: int) -> np.ndarray:
    """Bifurcations, vessel ends, then centreline samples; voxel coordinates."""
    sp = np.asarray(g.spec.spacing)
    pts = [p for p in g.bifurcations] + [p for p in g.ends]
    rng = SplitMix64Stream(g.spec.seed, sid=4)
    nseg = g.seg_a.shape[0]
    while len(pts) < n and nseg > 0:
        s = int(rng.uniform(1)[0] * nseg) % nseg
        t = float(rng.uniform(1)[0])
        pts.append(g.seg_a[s] + t * (g.seg_b[s] - g.seg_a[s]))
    pts = np.array(pts[:n], dtype=np.float64).reshape(-1, 3)
    return pts / sp


def make_lung_phantom(spec: PhantomSpec, with_true_field: bool = False) -> dict:
    """Static/moving pair, landmarks and their true displacements.

    Returns a dict with
      S, M          float32 volumes of shape (nz, ny, nx) (x fastest), HU
      landmarks     (L, 3) static-image points, voxel coordinates (x, y, z)
      u_true_mm     (L, 3) true displacement at the landmarks, mm: the moving
                    point is landmark + u_true / spacing
      u_true_field  (3, nz, ny, nx) float64 true field in voxels, if asked
    """
    g = _build_geometry(spec)
    pts = _grid_points(spec.dims)
    sp = np.asarray(spec.spacing)
    s_clean = _clean_image(g, pts)
    v = backward_map_mm(g, pts * sp)
    m_clean = _clean_image(g, pts + v / sp)
    nvox = int(np.prod(spec.dims))
    noise_s = SplitMix64Stream(spec.seed + 1, sid=3).normal(nvox).reshape(s_clean.shape)
    noise_m = SplitMix64Stream(spec.seed + 2, sid=3).normal(nvox).reshape(s_clean.shape)
    S = (s_clean + spec.noise_hu * noise_s).astype(np.float32)
    M = (m_clean + spec.noise_hu * noise_m).astype(np.float32)
    lm = _landmarks(g, spec.n_landmarks)
    out = {"S": S, "M": M, "landmarks": lm, "u_true_mm": true_field_mm(g, lm),
           "spacing": sp, "dims": spec.dims, "spec": spec}
    if with_true_field:
        u = true_field_mm(g, pts.reshape(-1, 3)).reshape(pts.shape) / sp
        out["u_true_field"] = np.ascontiguousarray(np.moveaxis(u, -1, 0))
    return out


# --------------------------------------------------------------------------
# Smooth blob pair with a known rigid shift
# --------------------------------------------------------------------------

def make_blob_pair(dims, shift_vox, seed: int = 7, n_blobs: int = 12,
                   sigma_vox: float = 6.0, amplitude: float = 100.0,
                   noise: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """S(x) = sum of Gaussian blobs; M(y) = S(y - T) (moving = static shifted by +T).

    With W(x) = M(x + u(x)), the field that registers them is u = T everywhere.
    Returns float32 (S, M) of shape (nz, ny, nx).
    """
    nx, ny, nz = dims
    rng = SplitMix64Stream(seed, sid=5)
    n = np.array([nx, ny, nz], dtype=np.float64)
    centres = 0.25 * n + 0.5 * n * rng.uniform(3 * n_blobs).reshape(n_blobs, 3)
    signs = np.where(rng.uniform(n_blobs) < 0.5, -1.0, 1.0)
    widths = sigma_vox * rng.uniform(n_blobs, 0.7, 1.3)
    pts = _grid_points(dims)
    t = np.asarray(shift_vox, dtype=np.float64)

    def blobs(p):
        acc = np.zeros(p.shape[:-1])
        for c, s, w in zip(centres, signs, widths):
            acc += s * amplitude * np.exp(-np.sum((p - c) ** 2, axis=-1) / (2.0 * w * w))
        return acc

    S = blobs(pts)
    M = blobs(pts - t)
    if noise > 0:
        S = S + noise * SplitMix64Stream(seed + 1, sid=6).normal(S.size).reshape(S.shape)
        M = M + noise * SplitMix64Stream(seed + 2, sid=6).normal(M.size).reshape(M.shape)
    return S.astype(np.float32), M.astype(np.float32)


def make_wave_pair(dims, shift_vox, seed: int = 9, n_terms: int = 3,
                   wavelength_vox: tuple = (20.0, 60.0),
                   amplitude: float = 100.0) -> tuple[np.ndarray, np.ndarray]:
    """S = sum of separable products of cosines; M(y) = S(y - T).

    Each term is a * cos(2 pi x / lx + px) cos(2 pi y / ly + py) cos(2 pi z / lz + pz)
    with seeded wavelengths in `wavelength_vox` and phases, so a volume of any
    size is built from 1-D factors (outer products) in a second or two.  As for
    make_blob_pair, the field that registers the pair is u = T.  Returns
    float32 (S, M) of shape (nz, ny, nx).
    """
    nx, ny, nz = dims
    rng = SplitMix64Stream(seed, sid=7)
    lam = rng.uniform(3 * n_terms, wavelength_vox[0], wavelength_vox[1]).reshape(n_terms, 3)
    phase = rng.uniform(3 * n_terms, 0.0, 2.0 * math.pi).reshape(n_terms, 3)
    amp = amplitude * rng.uniform(n_terms, 0.5, 1.0)
    axes = [np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64),
            np.arange(nz, dtype=np.float64)]
    t = np.asarray(shift_vox, dtype=np.float64)

    def volume(off):
        acc = np.zeros((nz, ny, nx))
        for k in range(n_terms):
            f = [np.cos(2.0 * math.pi * (axes[a] - off[a]) / lam[k, a] + phase[k, a])
                 for a in range(3)]
            acc += amp[k] * f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
        return acc

    S = volume(np.zeros(3))
    M = volume(t)
    return S.astype(np.float32), M.astype(np.float32)


def random_volume(dims, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform random float64 volume of shape (nz, ny, nx), for unit tests."""
    nx, ny, nz = dims
    return SplitMix64Stream(seed, sid=9).uniform(nx * ny * nz, lo, hi).reshape(nz, ny, nx)
