"""The single-precision parity criterion, shared by the GPU parity tests and
the CPU test that calibrates it (tests/test_oracle_twin.py).

The demons iteration amplifies rounding unevenly, so the FP32 GPU field is
compared with the FP64 oracle against the oracle's own sensitivity: the
per-voxel spread of oracle runs whose state is perturbed at rounding size
(`oracle.register(..., probe_rel, probe_seed)`).

(1) Voxels whose 7^3 neighbourhood (the footprint of the sigma = 1 Gaussian,
    through which rounding spreads between iterations) keeps the spread within
    bar * COND must meet the bar.
(2) Over the whole volume each quantile of the error (median up to the
    maximum) must stay within SHADOW times the same quantile of the spread,
    plus bar * COND: the spread of a few probes predicts the size of the
    deviation a single-precision run has, not its exact place.  SHADOW is
    calibrated by an independent single-precision implementation (the NumPy
    twin in float32), which deviates from the oracle by up to about five times
    the probes' spread at the 99th percentile on small ragged volumes.
"""
import numpy as np

COND = 0.01       # conditioned: the neighbourhood's spread within bar * COND
SHADOW = 10.0     # error quantiles within SHADOW x the spread quantiles
QUANTILES = (0.5, 0.9, 0.99, 0.999, 0.9999, 1.0)


def conditioned(spread, bar):
    from scipy.ndimage import maximum_filter
    return maximum_filter(spread, size=7, mode="nearest") <= bar * COND


def shadow_check(err, spread, bar, label, min_cond=0.0):
    """Asserts (1) and (2); returns the fraction of voxels outside the
    conditioned set (at most 1 - min_cond)."""
    cond = conditioned(spread, bar)
    ill = 1.0 - float(cond.mean())
    assert 1.0 - ill >= min_cond, f"{label}: only {1 - ill:.1%} of voxels conditioned"
    if cond.any():
        worst = float(err[cond].max())
        assert worst <= bar, f"{label}: max|du| {worst:.3e} on conditioned voxels (bar {bar:g})"
    for q in QUANTILES:
        qe, qs = float(np.quantile(err, q)), float(np.quantile(spread, q))
        assert qe <= SHADOW * qs + bar * COND, (
            f"{label}: q{q} error {qe:.3e} vs oracle spread {qs:.3e}")
    return ill


def fp32_spread(oracle, S, M, variant, levels, iters, ref_u, alpha=0.4, sigma=1.0):
    """Spread of the single-precision probes: the state stored in float
    (oracle.ROUND32) and the coherent +-2^-24 nudge."""
    spread = np.zeros(S.shape)
    for seed, rel in ((oracle.ROUND32, 1.0), (0, 2.0 ** -24), (0, -(2.0 ** -24))):
        up = oracle.register(S, M, variant=variant, levels=levels, iters=iters, alpha=alpha,
                             sigma=sigma, probe_rel=rel, probe_seed=seed)["u"]
        spread = np.maximum(spread, np.abs(up - ref_u).max(axis=0))
    return spread
