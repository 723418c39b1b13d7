"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
invariants, special cases that reduce to another equation of the paper,
brute force on tiny inputs, and recovery of known deformations.
"""
import math

import numpy as np
import pytest

import oracle
from phantom import make_blob_pair, random_volume

VARIANTS = range(6)


def _grid(dims):
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.astype(float), j.astype(float), k.astype(float)


# ----------------------------------------------------------------- trilinear

def test_interp_exact_at_grid_points():
    # Sec. 2.5 interpolation: at a grid point the weights are 0/1.
    vol = random_volume((7, 5, 4), seed=11)
    i, j, k = _grid((7, 5, 4))
    assert np.array_equal(oracle.interp(vol, i, j, k), vol)


def test_interp_reproduces_multilinear_functions():
    # Trilinear interpolation is exact on span{1, x, y, z, xy, xz, yz, xyz}.
    dims = (9, 8, 7)
    i, j, k = _grid(dims)
    f = lambda x, y, z: 3.0 - 2.0 * x + 0.5 * y - z + 0.25 * x * y - 0.125 * x * z + 0.3 * y * z + 0.05 * x * y * z
    vol = f(i, j, k)
    from phantom import SplitMix64Stream
    r = SplitMix64Stream(5, 1)
    px, py, pz = r.uniform(500, 0, 8), r.uniform(500, 0, 7), r.uniform(500, 0, 6)
    np.testing.assert_allclose(oracle.interp(vol, px, py, pz), f(px, py, pz), rtol=0, atol=1e-12)


def test_interp_clamps_outside_points():
    vol = random_volume((6, 6, 6), seed=3)
    pts = np.array([[-3.0, 2.5, 1.25], [7.5, -1.0, 9.0], [2.2, 8.0, -0.5]])
    clamped = np.clip(pts, 0.0, 5.0)
    a = oracle.interp(vol, pts[:, 0], pts[:, 1], pts[:, 2])
    b = oracle.interp(vol, clamped[:, 0], clamped[:, 1], clamped[:, 2])
    assert np.array_equal(a, b)


def test_interp_upper_edge_and_single_voxel_axis():
    # point exactly on the last grid plane, and an axis of length 1
    vol = random_volume((4, 3, 1), seed=4)
    assert oracle.interp(vol, 3.0, 2.0, 0.0)[()] == vol[0, 2, 3]
    assert oracle.interp(vol, 3.0, 2.0, 5.0)[()] == vol[0, 2, 3]
    mid = oracle.interp(vol, 1.5, 0.0, 0.0)[()]
    assert mid == pytest.approx(0.5 * (vol[0, 0, 1] + vol[0, 0, 2]), abs=1e-15)


# ------------------------------------------------------------------ gradient

def test_grad_exact_on_linear_ramp_interior():
    dims = (8, 7, 6)
    i, j, k = _grid(dims)
    vol = 2.0 * i - 3.0 * j + 0.5 * k + 7.0
    g = oracle.grad(vol)
    inner = (slice(1, -1),) * 3
    assert np.allclose(g[0][inner], 2.0, atol=1e-13)
    assert np.allclose(g[1][inner], -3.0, atol=1e-13)
    assert np.allclose(g[2][inner], 0.5, atol=1e-13)


def test_grad_exact_on_quadratic_interior():
    # the central difference is exact for quadratics: d/dx x^2 = 2x
    dims = (9, 3, 3)
    i, j, k = _grid(dims)
    g = oracle.grad(i * i)
    assert np.allclose(g[0][:, :, 1:-1], 2.0 * i[:, :, 1:-1], atol=1e-12)


def test_grad_boundary_by_hand():
    # 4-voxel line [1, 2, 4, 8], replicated ends:
    # i=0: (2-1)/2, i=1: (4-1)/2, i=2: (8-2)/2, i=3: (8-4)/2
    vol = np.array([1.0, 2.0, 4.0, 8.0]).reshape(1, 1, 4)
    g = oracle.grad(vol)
    assert np.array_equal(g[0].ravel(), [0.5, 1.5, 3.0, 2.0])
    assert np.array_equal(g[1].ravel(), [0, 0, 0, 0])
    assert np.array_equal(g[2].ravel(), [0, 0, 0, 0])


# ------------------------------------------------------------------ Gaussian

def test_gauss_taps_closed_form():
    w = oracle.gauss_taps(1.0)
    assert w.size == 7  # R = ceil(3 sigma) = 3
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.array_equal(w, w[::-1])
    for t in range(1, 4):
        assert w[3 + t] / w[3] == pytest.approx(math.exp(-t * t / 2.0), rel=1e-14)
    assert oracle.gauss_taps(0.5).size == 5 and oracle.gauss_taps(2.0).size == 13


def test_gauss_keeps_constant_and_interior_ramp():
    dims = (12, 11, 10)
    c = np.full((10, 11, 12), 3.25)
    assert np.allclose(oracle.gauss3(c, 1.0), 3.25, atol=1e-14)
    i, j, k = _grid(dims)
    ramp = 0.5 * i - 2.0 * j + 1.5 * k
    out = oracle.gauss3(ramp, 1.0)
    inner = (slice(3, -3),) * 3
    assert np.allclose(out[inner], ramp[inner], atol=1e-12)


def test_gauss_matches_brute_force_3d_convolution():
    # separable x, y, z passes == one non-separable 7^3 convolution with
    # replicated edges (the replicate boundary commutes with separability)
    vol = random_volume((9, 9, 9), seed=21)
    w = oracle.gauss_taps(1.0)
    P = np.pad(vol, 3, mode="edge")
    brute = np.zeros_like(vol)
    for a in range(7):
        for b in range(7):
            for c in range(7):
                brute += w[a] * w[b] * w[c] * P[a:a + 9, b:b + 9, c:c + 9]
    np.testing.assert_allclose(oracle.gauss3(vol, 1.0), brute, rtol=0, atol=1e-12)


# ------------------------------------------------------------------- pyramid

def test_downsample_sizes_and_constant():
    for dims in ((8, 8, 8), (9, 7, 5), (1, 3, 2)):
        nx, ny, nz = dims
        out = oracle.downsample(np.full((nz, ny, nx), -850.0))
        assert out.shape == ((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2)
        assert np.allclose(out, -850.0, atol=1e-12)


def test_downsample_takes_even_samples_of_smoothed_ramp():
    dims = (20, 18, 16)
    i, j, k = _grid(dims)
    ramp = i + 2.0 * j - k
    out = oracle.downsample(ramp)
    ci, cj, ck = _grid((10, 9, 8))
    inner = (slice(2, -2),) * 3
    assert np.allclose(out[inner], (2 * ci + 4 * cj - 2 * ck)[inner], atol=1e-12)


def test_upsample_constant_doubles():
    up = oracle.upsample(np.full((3, 4, 5, 6), 1.25), (12, 10, 8))
    assert up.shape == (3, 8, 10, 12)
    assert np.allclose(up, 2.5, atol=1e-15)


def test_upsample_preserves_uniform_scaling_field():
    # a coarse field u_c(i) = s * i (coarse voxels) describes the same scaling
    # as u_f(x) = s * x in fine voxels: coarse point x/2, displacement s x/2
    # coarse voxels = s x fine voxels.  Odd fine sizes (ceil(n/2) = coarse size)
    # keep every x/2 inside the coarse grid, so no clamping is involved.
    s = 0.3
    ci, cj, ck = _grid((6, 5, 4))
    coarse = np.stack([s * ci, -s * cj, 2 * s * ck])
    fi, fj, fk = _grid((11, 9, 7))
    up = oracle.upsample(coarse, (11, 9, 7))
    np.testing.assert_allclose(up, np.stack([s * fi, -s * fj, 2 * s * fk]), atol=1e-12)


# --------------------------------------------------------------- force laws

def _force_samples(seed, n=4000):
    from phantom import SplitMix64Stream
    r = SplitMix64Stream(seed, 2)
    d = r.normal(n) * 50.0
    gs = r.normal(3 * n).reshape(3, n) * 30.0
    gm = r.normal(3 * n).reshape(3, n) * 30.0
    b = np.abs(r.normal(n)) * 40.0
    return d, gs, gm, b


@pytest.mark.parametrize("variant,bound_fn", [
    (0, lambda a: 0.5), (2, lambda a: 0.5), (5, lambda a: 0.5), (3, lambda a: 1.0),
    (4, lambda a: 1.0 / a), (1, lambda a: 2.0 * math.sqrt(6.0) / 9.0)])
def test_force_magnitude_bounds(variant, bound_fn):
    # AM-GM: |d||g| / (d^2 + |g|^2) <= 1/2; with alpha^2 d^2: <= 1/(2 alpha);
    # Eq. (2): (2d^2+s) >= 2 sqrt(2) |d| sqrt(s), and max a^2 b / s^(3/2) = 2/(3 sqrt 3)
    d, gs, gm, b = _force_samples(7)
    for alpha in (0.4, 1.0, 2.0):
        dr = oracle.force(variant, d, gs, gm, b, alpha=alpha)
        mag = np.sqrt(np.sum(dr * dr, axis=0))
        assert mag.max() <= bound_fn(alpha) * (1 + 1e-12)


def test_force_bounds_are_attained():
    # passive: |d| = |g| gives exactly 1/2
    dr = oracle.force(0, np.array([3.0]), np.array([[3.0], [0.0], [0.0]]))
    assert dr[0, 0] == pytest.approx(0.5, abs=1e-15)
    # evolved: b = a / sqrt(2), 2 d^2 = a^2 + b^2 attains 2 sqrt(6) / 9
    a = 2.0
    bb = a / math.sqrt(2.0)
    d = math.sqrt((a * a + bb * bb) / 2.0)
    dr = oracle.force(1, np.array([d]), np.array([[a], [0.0], [0.0]]), b=np.array([bb]))
    assert dr[0, 0] == pytest.approx(2.0 * math.sqrt(6.0) / 9.0, rel=1e-14)


def test_force_zero_when_images_equal():
    d = np.zeros(100)
    _, gs, gm, b = _force_samples(3, 100)
    for v in VARIANTS:
        assert np.array_equal(oracle.force(v, d, gs, gm, b, alpha=0.4), np.zeros((3, 100)))


def test_force_zero_zero_is_zero():
    # 0/0 where both d and the gradient vanish: the force is defined as 0
    z = np.zeros(1)
    g0 = np.zeros((3, 1))
    for v in VARIANTS:
        assert np.array_equal(oracle.force(v, z, g0, g0, z, alpha=2.0), np.zeros((3, 1)))


def test_evolved_reduces_to_passive_when_gradient_norms_match():
    # Eq. (2) with |grad I_m(0)| = |grad I_s(0)| equals Eq. (1)
    d, gs, _, _ = _force_samples(5)
    b = np.sqrt(np.sum(gs * gs, axis=0))
    np.testing.assert_allclose(oracle.force(1, d, gs, b=b), oracle.force(0, d, gs),
                               rtol=1e-13, atol=1e-15)


def test_adjusted_with_unit_alpha_equals_double():
    # Eq. (5) with alpha = 1 equals Eq. (4)
    d, gs, gm, _ = _force_samples(9)
    assert np.array_equal(oracle.force(4, d, gs, gm, alpha=1.0), oracle.force(3, d, gs, gm))


def test_double_is_sum_of_passive_and_active():
    d, gs, gm, _ = _force_samples(13)
    np.testing.assert_allclose(oracle.force(3, d, gs, gm),
                               oracle.force(0, d, gs) + oracle.force(2, d, None, gm),
                               rtol=1e-15, atol=1e-15)


def test_force_direction_and_newton_limit():
    # dr is parallel to the driving gradient with the sign of d; for |d| << |g|
    # it tends to the Newton step d g / |g|^2, so that I(x - dr) ~ I(x) - d
    d, gs, _, _ = _force_samples(17)
    dr = oracle.force(0, d, gs)
    dots = np.sum(dr * gs, axis=0)
    assert np.all(np.sign(dots[d != 0]) == np.sign(d[d != 0]))
    g = np.array([[4.0], [-2.0], [1.0]])
    small = np.array([1e-6])
    np.testing.assert_allclose(oracle.force(0, small, g), small * g / 21.0, rtol=1e-11)


def test_active_step_shrinks_difference_on_a_ramp():
    # On a ramp M(x) = m0 + g.x the active step leaves d * d^2/(d^2+|g|^2),
    # the exact residual of the force law; it pins the subtraction du = -dr.
    g = np.array([[3.0], [-1.0], [2.0]])
    for dval in (-40.0, -1.0, 0.5, 12.0):
        d = np.array([dval])
        dr = oracle.force(2, d, None, g)
        d_new = dval + float(np.sum(g[:, 0] * -dr[:, 0]))
        assert d_new == pytest.approx(dval * dval * dval / (dval * dval + 14.0), rel=1e-12)


# --------------------------------------------------------- whole iteration

def test_equal_images_give_zero_update_all_variants():
    # S == M and u == 0: d == 0 everywhere, the field stays exactly zero
    vol = random_volume((10, 9, 8), seed=31) * 500
    for v in VARIANTS:
        u, red = oracle.iterate(v, vol, vol, np.zeros((3,) + vol.shape), alpha=0.4)
        assert np.array_equal(u, np.zeros_like(u)), v
        assert red[0] == 0.0 and red[1] == 0.0 and red[2] == 0.0


def _brute_gauss(vol, sigma):
    """Non-separable (2R+1)^3 convolution with replicated edges, taps written
    out from the closed form exp(-t^2 / 2 sigma^2) / sum."""
    R = math.ceil(3 * sigma)
    t = np.arange(-R, R + 1, dtype=float)
    w = np.exp(-t * t / (2 * sigma * sigma))
    w /= w.sum()
    nz, ny, nx = vol.shape
    P = np.pad(vol, R, mode="edge")
    out = np.zeros_like(vol)
    for a in range(2 * R + 1):
        for b in range(2 * R + 1):
            for c in range(2 * R + 1):
                out += w[a] * w[b] * w[c] * P[a:a + nz, b:b + ny, c:c + nx]
    return out


@pytest.mark.parametrize("variant", VARIANTS)
def test_iteration_smooths_the_total_field(variant):
    # Sec. 2.1 (Thirion's regularisation): the Gaussian acts on the whole
    # displacement field u + du, not on the update du alone.  With S = M
    # constant, W - S and every gradient vanish, so du = 0 (Q7) and one
    # iteration must give G_sigma * u for a rough, nonzero u; smoothing only
    # du would leave u unchanged.
    dims = (11, 9, 8)
    vol = np.full(dims[::-1], -850.0)
    u = np.stack([random_volume(dims, seed=41 + c) * 3.0 - 1.5 for c in range(3)])
    for sigma in (1.0, 0.6):
        un, red = oracle.iterate(variant, vol, vol.copy(), u, sigma=sigma, alpha=0.4)
        for c in range(3):
            np.testing.assert_allclose(un[c], _brute_gauss(u[c], sigma), rtol=0, atol=1e-12)
        assert red[0] == 0.0 and red[1] == 0.0
        assert red[2] == pytest.approx(np.sqrt((u ** 2).sum(axis=0)).sum(), rel=1e-13)
        assert np.abs(un - u).max() > 0.1


def test_inverse_consistent_is_antisymmetric():
    # Eq. (6) treats S and M symmetrically: registering (M, S) gives exactly -h
    S, M = make_blob_pair((16, 14, 12), (1.0, -0.5, 0.25), seed=3, n_blobs=20, sigma_vox=3.0)
    a = oracle.register(S, M, variant=5, levels=2, iters=[4, 6], return_raw=True)
    b = oracle.register(M, S, variant=5, levels=2, iters=[4, 6], return_raw=True)
    assert np.array_equal(a["raw"], -b["raw"])


def test_ic_field_inverts_translation_exactly():
    # for a constant mid-space field h the output is u = 2 h exactly
    h = np.zeros((3, 6, 7, 8))
    h[0], h[1], h[2] = 0.75, -0.25, 0.5
    np.testing.assert_allclose(oracle.ic_field(h), 2 * h, atol=1e-14)


def test_ic_field_composition():
    # u(y) = 2 h(x*) with x* - h(x*) = y: check the defining relation
    dims = (14, 12, 10)
    i, j, k = _grid(dims)
    h = np.stack([0.4 * np.sin(j / 3.0), 0.3 * np.cos(i / 4.0), 0.2 * np.sin(k / 2.0)])
    u = oracle.ic_field(h)
    # x* = y + u/2; check x* - h(x*) = y inside (x* stays inside the volume)
    xs = [i + u[0] / 2, j + u[1] / 2, k + u[2] / 2]
    hx = [oracle.interp(h[c], *xs) for c in range(3)]
    inner = (slice(2, -2),) * 3
    for c, y in enumerate((i, j, k)):
        assert np.allclose((xs[c] - hx[c])[inner], y[inner], atol=1e-6)


# -------------------------------------------------------- known deformation

T_SHIFT = np.array([1.5, -0.75, 0.5])


@pytest.mark.parametrize("variant", VARIANTS)
def test_rigid_shift_recovery(variant):
    # M(y) = S(y - T): the registering field is u = T (and h = T/2 for Eq. 6).
    S, M = make_blob_pair((48, 48, 48), T_SHIFT, seed=7, n_blobs=200, sigma_vox=6.0)
    r = oracle.register(S, M, variant=variant, levels=3, iters=[100, 100, 100],
                        alpha=2.0, return_raw=True)
    inner = (slice(None),) + (slice(12, -12),) * 3
    u = r["u"][inner]
    err = np.sqrt(np.sum((u - T_SHIFT[:, None, None, None]) ** 2, axis=0))
    assert np.all(np.abs(u.mean(axis=(1, 2, 3)) - T_SHIFT) < 0.05)
    assert np.median(err) < 0.08
    assert np.percentile(err, 95) < 0.25
    if variant == 5:
        h = r["raw"][inner].mean(axis=(1, 2, 3))
        assert np.all(np.abs(h - T_SHIFT / 2) < 0.03)


def test_rigid_shift_single_scale_passive():
    S, M = make_blob_pair((48, 48, 48), T_SHIFT, seed=7, n_blobs=200, sigma_vox=6.0)
    r = oracle.register(S, M, variant=0, levels=1, iters=[200])
    u = r["u"][(slice(None),) + (slice(12, -12),) * 3]
    assert np.all(np.abs(u.mean(axis=(1, 2, 3)) - T_SHIFT) < 0.06)
    # MSE falls monotonically in this well-posed case
    mse = r["stats"][:, 0]
    assert mse[-1] < 0.05 * mse[0]


@pytest.mark.parametrize("variant", VARIANTS)
def test_lung_phantom_landmark_error_drops(variant, small_phantom):
    # the seeded analytic RBF deformation: landmark error falls well below the
    # initial landmark displacement (Sec. 3.2 evaluation on synthetic data)
    p = small_phantom
    r = oracle.register(p["S"], p["M"], variant=variant, levels=1, iters=[50],
                        alpha=0.4 if variant == 4 else 1.0)
    lm, sp = p["landmarks"], p["spacing"]
    ue = np.stack([oracle.interp(r["u"][c], lm[:, 0], lm[:, 1], lm[:, 2]) for c in range(3)], 1)
    err = np.linalg.norm(ue * sp - p["u_true_mm"], axis=1)
    init = np.linalg.norm(p["u_true_mm"], axis=1)
    assert np.sqrt(np.mean(err ** 2)) < 0.25 * np.sqrt(np.mean(init ** 2))


def test_stop_test_property(small_phantom):
    # Sec. 2.4 stop test read as |l(n) - l(n-10)| <= eps within a level
    p = small_phantom
    eps, w = 2e-3, 10
    r = oracle.register(p["S"], p["M"], variant=0, levels=1, iters=[300], stop_mode=1,
                        eps=eps, stop_window=w)
    st = r["stats"]
    n = r["iters_run"][0]
    assert w < n < 300
    l = np.where(st[:, 2] > 0, st[:, 1] / np.where(st[:, 2] > 0, st[:, 2], 1), np.nan)
    for it in range(w, n - 1):
        if not (np.isnan(l[it]) or np.isnan(l[it - w])):
            assert abs(l[it] - l[it - w]) > eps
    assert abs(l[n - 1] - l[n - 1 - w]) <= eps
    full = oracle.register(p["S"], p["M"], variant=0, levels=1, iters=[n])
    assert np.array_equal(full["u"], r["u"])


def test_threaded_oracle_is_bit_identical(small_phantom):
    p = small_phantom
    a = oracle.register(p["S"], p["M"], variant=3, levels=2, iters=[5, 5], threaded=False)
    b = oracle.register(p["S"], p["M"], variant=3, levels=2, iters=[5, 5], threaded=True)
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["stats"], b["stats"])


def test_conditioning_of_the_iteration(small_phantom):
    # The iteration amplifies input rounding very differently per force law:
    # perturbing every input voxel by one FP32 ulp (relative 2^-23) moves the
    # FP64 passive result by far less than the 1e-3 voxel parity bar, but the
    # double force (steps up to 1 voxel, Eq. 4) by more than the bar, on the
    # clamped boundary planes.  FP32 parity is therefore assessed on conditioned
    # voxels only, and the FP64 build of the kernels is compared everywhere.
    from phantom import SplitMix64Stream
    p = small_phantom
    S, M = p["S"].astype(np.float64), p["M"].astype(np.float64)
    r = SplitMix64Stream(77, 7)
    xs = np.floor(r.uniform(2 * S.size) * 3.0).reshape((2,) + S.shape) - 1.0
    Sp, Mp = S * (1 + 2.0 ** -23 * xs[0]), M * (1 + 2.0 ** -23 * xs[1])
    sens = {}
    for v in (0, 3):
        a = oracle.register(S, M, variant=v, levels=1, iters=[50])["u"]
        b = oracle.register(Sp, Mp, variant=v, levels=1, iters=[50])["u"]
        sens[v] = np.abs(a - b).max(axis=0)
    assert sens[0].max() < 1e-4
    assert sens[3].max() > 1e-3
    worst = np.unravel_index(np.argmax(sens[3]), sens[3].shape)
    assert worst[0] in (0, 1, 2, 29, 30, 31)  # a boundary slab in z


def test_single_precision_state_probe(small_phantom):
    # The ROUND32 probe keeps the method's arithmetic in FP64 but stores its
    # state in single precision.  Zero stays exactly zero (equal images), a
    # zero probe size switches it off, and on the passive 50-iteration run it
    # moves the result by more than nothing but far less than the 1e-3 bar,
    # while the double force (Eq. 4) is sensitive to it beyond the bar.
    p = small_phantom
    S, M = p["S"].astype(np.float64), p["M"].astype(np.float64)
    z = oracle.register(S, S, variant=3, levels=2, iters=[5, 5], probe_rel=1.0,
                        probe_seed=oracle.ROUND32)
    assert np.all(z["u"] == 0.0)
    plain = oracle.register(S, M, variant=0, levels=1, iters=[50])["u"]
    off = oracle.register(S, M, variant=0, levels=1, iters=[50], probe_rel=0.0,
                          probe_seed=oracle.ROUND32)["u"]
    assert np.array_equal(plain, off)
    r = oracle.register(S, M, variant=0, levels=1, iters=[50], probe_rel=1.0,
                        probe_seed=oracle.ROUND32)["u"]
    d = np.abs(r - plain).max()
    assert 0.0 < d < 1e-5
    # the stored field is float-representable after every iteration
    assert np.array_equal(r, r.astype(np.float32).astype(np.float64))
    a = oracle.register(S, M, variant=3, levels=1, iters=[50])["u"]
    b = oracle.register(S, M, variant=3, levels=1, iters=[50], probe_rel=1.0,
                        probe_seed=oracle.ROUND32)["u"]
    assert np.abs(a - b).max() > 1e-3


@pytest.mark.parametrize("variant", [0, 2, 5])
def test_two_iterations_are_local(variant):
    # the largest-size GPU parity test relies on this: after one level of two
    # iterations each output voxel depends only on a neighbourhood of radius
    # below 12, so a crop of the inputs reproduces the whole-volume result on
    # the voxels at least 12 from every crop face inside the volume
    from phantom import make_wave_pair
    dims = (80, 72, 60)
    S, M = make_wave_pair(dims, (1.5, -0.75, 0.5), seed=21)
    full = oracle.register(S, M, variant=variant, levels=1, iters=(2,))["u"]
    C, m = 40, 12
    for x0, y0, z0 in [(0, 0, 0), (dims[0] - C, dims[1] - C, dims[2] - C), (20, 17, 11)]:
        sl = (slice(z0, z0 + C), slice(y0, y0 + C), slice(x0, x0 + C))
        crop = oracle.register(np.ascontiguousarray(S[sl]), np.ascontiguousarray(M[sl]),
                               variant=variant, levels=1, iters=(2,))["u"]
        core = tuple(slice(0 if o == 0 else m, C if o + C == n else C - m)
                     for o, n in ((z0, dims[2]), (y0, dims[1]), (x0, dims[0])))
        a = full[(slice(None),) + sl][(slice(None),) + core]
        b = crop[(slice(None),) + core]
        assert np.abs(a - b).max() <= 1e-12
        assert np.abs(a).max() > 0.1  # the field has moved
    # and the margin matters: two voxels from an inner face the crop differs
    near = (slice(None),) + (slice(2, C - 2),) * 3
    assert np.abs(full[(slice(None),) + sl][near] - crop[near]).max() > 1e-3


# ------------------------------------------------------ correlation coefficient

def test_correlation_against_its_definition():
    # Secs. 2.4 and 3.3: the Pearson correlation of two images, checked
    # against numpy's corrcoef (an independent implementation) and its
    # invariants
    a = random_volume((9, 8, 7), seed=61) * 300 - 700
    b = 0.4 * a + random_volume((9, 8, 7), seed=62) * 50
    assert oracle.correlation(a, b) == pytest.approx(np.corrcoef(a.ravel(), b.ravel())[0, 1],
                                                     abs=1e-13)
    assert oracle.correlation(a, a) == pytest.approx(1.0, abs=1e-15)
    assert oracle.correlation(a, -a) == pytest.approx(-1.0, abs=1e-15)
    assert oracle.correlation(a, 3.0 * b + 11.0) == pytest.approx(oracle.correlation(a, b),
                                                                   abs=1e-14)
    assert math.isnan(oracle.correlation(a, np.full_like(a, 5.0)))


@pytest.mark.parametrize("variant", VARIANTS)
def test_iteration_correlation_is_that_of_the_warped_images(variant):
    # the per-iteration correlation is taken on the pre-update warped image
    # and S (Eq. 6: the two warped images M(x + h) and S(x - h))
    S, M = make_blob_pair((14, 12, 10), (0.7, -0.4, 0.3), seed=9, n_blobs=12, sigma_vox=2.5)
    u = np.stack([np.full(S.shape, 0.3), np.full(S.shape, -0.2), np.full(S.shape, 0.1)])
    u[0] += random_volume(S.shape[::-1], seed=3) * 0.2
    _, _, rho = oracle.iterate(variant, S, M, u, alpha=0.4, corr=True)
    if variant == 5:
        a, b = oracle.warp(M, u), oracle.warp(S, u, sign=-1.0)
    else:
        a, b = oracle.warp(M, u), S
    assert rho == pytest.approx(np.corrcoef(a.ravel(), b.ravel())[0, 1], abs=1e-12)
    _, _, one = oracle.iterate(variant, S, S.copy(), np.zeros_like(u), alpha=0.4, corr=True)
    assert one == pytest.approx(1.0, abs=1e-14)


def test_correlation_stop_test_property(small_phantom):
    # stop_mode 2: a level stops at the first iteration n >= window with
    # |rho(n) - rho(n - window)| <= eps, and not before
    S, M = small_phantom["S"], small_phantom["M"]
    eps, w = 2e-4, 5
    r = oracle.register(S, M, variant=0, levels=1, iters=[200], stop_mode=2, eps=eps,
                        stop_window=w)
    rho = r["corr"]
    n = r["iters_run"][0]
    assert w < n < 200 and rho.shape[0] == n
    for it in range(w, n - 1):
        assert abs(rho[it] - rho[it - w]) > eps
    assert abs(rho[n - 1] - rho[n - 1 - w]) <= eps
    full = oracle.register(S, M, variant=0, levels=1, iters=[n], return_corr=True)
    np.testing.assert_array_equal(full["corr"], rho)
    np.testing.assert_array_equal(full["u"], r["u"])
