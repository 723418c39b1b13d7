"""The C oracle against the independent NumPy twin on tiny volumes (<= 16^3), and
the twin in float32 as a calibration of the single-precision parity criterion."""
import numpy as np
import pytest

import numpy_twin as twin
import oracle
from phantom import make_blob_pair, random_volume


@pytest.mark.parametrize("dims", [(5, 7, 3), (16, 16, 16), (9, 4, 11)])
def test_primitives_match_twin(dims):
    vol = random_volume(dims, seed=sum(dims)) * 100
    np.testing.assert_allclose(oracle.grad(vol), twin.grad(vol), atol=1e-12, rtol=0)
    for sigma in (0.6, 1.0, 1.7):
        np.testing.assert_allclose(oracle.gauss3(vol, sigma), twin.gauss3(vol, sigma),
                                   atol=1e-11, rtol=0)
    np.testing.assert_allclose(oracle.downsample(vol), twin.downsample(vol), atol=1e-11)
    u = np.stack([random_volume(dims, seed=s) * 3 for s in (1, 2, 3)])
    np.testing.assert_allclose(oracle.warp(vol, u), twin.interp(vol, *[
        g + u[c] for c, g in enumerate(twin.grid(vol.shape))]), atol=1e-11)
    nx, ny, nz = dims
    fine = (2 * nx - 1, 2 * ny, 2 * nz - 1)
    np.testing.assert_allclose(oracle.upsample(u, fine), twin.upsample(u, fine[::-1]),
                               atol=1e-12)
    np.testing.assert_allclose(oracle.ic_field(u * 0.2), twin.ic_field(u * 0.2), atol=1e-11)


@pytest.mark.parametrize("variant", range(6))
@pytest.mark.parametrize("levels", [1, 2])
def test_registration_matches_twin(variant, levels):
    S, M = make_blob_pair((16, 13, 11), (0.8, -0.6, 0.4), seed=variant + 1, n_blobs=10,
                          sigma_vox=2.5, noise=1.0)
    iters = [5] if levels == 1 else [3, 5]
    r = oracle.register(S, M, variant=variant, levels=levels, iters=iters, alpha=0.4,
                        threaded=False, return_raw=True)
    u, stats = twin.register(S, M, variant, levels, iters, alpha=0.4)
    np.testing.assert_allclose(r["raw"], u, atol=1e-12, rtol=0)
    np.testing.assert_allclose(r["stats"], stats, rtol=1e-12, atol=1e-12)
    if variant == 5:
        np.testing.assert_allclose(r["u"], twin.ic_field(u), atol=1e-11)


# --------------------------------------------------------------------------
# Calibration of the single-precision parity criterion (parity_criteria.py):
# an independent FP32 implementation of the same steps (this twin in
# float32, written without the GPU path's care for rounding) must pass it,
# and the same twin with a plausible slip must not.

def _ragged(dims, seed):
    from phantom import PhantomSpec, make_lung_phantom
    spec = PhantomSpec(dims=dims, spacing=(1.2, 1.2, 2.5), seed=seed, a_max_mm=5.0,
                       compression=0.1, n_vessels=12, n_landmarks=50)
    p = make_lung_phantom(spec)
    return p["S"], p["M"]


@pytest.mark.parametrize("variant,dims,seed", [(5, (70, 9, 33), 16), (0, (45, 37, 19), 11),
                                               (2, (45, 37, 19), 13)])
def test_fp32_twin_passes_the_single_precision_criterion(variant, dims, seed):
    from parity_criteria import fp32_spread, shadow_check
    S, M = _ragged(dims, seed)
    sched = dict(levels=3, iters=[12, 8, 6])
    ref = oracle.register(S, M, variant=variant, alpha=0.4, **sched)
    spread = fp32_spread(oracle, S, M, variant, ref_u=ref["u"], **sched)
    u32, _ = twin.register(S, M, variant, 3, [12, 8, 6], dtype=np.float32)
    if variant == 5:
        u32 = twin.ic_field(u32)
    err = np.abs(u32.astype(np.float64) - ref["u"]).max(axis=0)
    assert err.max() > 0.0
    shadow_check(err, spread, 1e-3, f"twin32 v{variant} {dims}")


def test_the_criterion_rejects_a_slip():
    # a smoothing width off by 2% (a plausible slip in the taps) fails it
    from parity_criteria import fp32_spread, shadow_check
    S, M = _ragged((45, 37, 19), 11)
    sched = dict(levels=3, iters=[12, 8, 6])
    ref = oracle.register(S, M, variant=0, alpha=0.4, **sched)
    spread = fp32_spread(oracle, S, M, 0, ref_u=ref["u"], **sched)
    u, _ = twin.register(S, M, 0, 3, [12, 8, 6], sigma=1.02)
    err = np.abs(u - ref["u"]).max(axis=0)
    with pytest.raises(AssertionError):
        shadow_check(err, spread, 1e-3, "slipped twin")


def test_the_criteria_reject_a_slip_at_full_size(full_phantom):
    # The same kind of slip, planted in the oracle (a smoothing width 2 % too
    # small: the same 7 taps, slightly different values), on the 256 x 256 x 100
    # phantom: the every-voxel check of the short full-size schedules and the
    # shadow check of the long 200/100/50 schedule must both reject it, although
    # at full size the latter's conditioned set is a small part of the volume.
    from parity_criteria import (COND_LONG, TOL_U, fp32_spread, rel_rms, shadow_check,
                                 strict_check)
    S, M = full_phantom["S"], full_phantom["M"]
    short = dict(variant=0, levels=1, iters=[10])
    ref = oracle.register(S, M, **short)["u"]
    slip = oracle.register(S, M, sigma=0.98, **short)["u"]
    err = np.abs(slip - ref).max(axis=0)
    with pytest.raises(AssertionError):
        strict_check(err, "slipped oracle, 1 level x 10")
    print(f"short schedule: slip max|du| {err.max():.2e}, "
          f"rel-RMS(W) {rel_rms(oracle.warp(M, slip), oracle.warp(M, ref)):.1e}")
    sched = dict(levels=3, iters=[200, 100, 50])
    ref = oracle.register(S, M, variant=0, **sched)["u"]
    spread = fp32_spread(oracle, S, M, 0, ref_u=ref, **sched)
    slip = oracle.register(S, M, variant=0, sigma=0.98, **sched)["u"]
    err = np.abs(slip - ref).max(axis=0)
    with pytest.raises(AssertionError) as e:
        shadow_check(err, spread, TOL_U, "slipped oracle, 200/100/50", cond_level=COND_LONG)
    print(f"long schedule: {e.value}")
