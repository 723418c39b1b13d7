"""Host-side logic of the serving loop (no GPU): footprints, request streams."""
import numpy as np


def test_footprint_grows_with_volume_and_levels():
    from paper_0909_0928_gb300.serve import footprint_bytes
    a = footprint_bytes((64, 64, 32), 3)
    b = footprint_bytes((128, 128, 64), 3)
    c = footprint_bytes((128, 128, 64), 1)
    assert 0 < a < b and c < b
    # two fields of the finest level alone: 6 x N x 4 bytes
    assert b > 6 * 128 * 128 * 64 * 4


def test_poisson_requests_are_seeded_and_ordered():
    from paper_0909_0928_gb300 import serve
    sizes = [(32, 32, 16), (48, 32, 16)]
    r1 = serve.make_requests(12, rate=5.0, seed=3, sizes=sizes, iters=(2, 2, 2))
    r2 = serve.make_requests(12, rate=5.0, seed=3, sizes=sizes, iters=(2, 2, 2))
    t = [r.arrival for r in r1]
    assert t == sorted(t) and t == [r.arrival for r in r2]
    assert all(0 <= r.variant < 6 for r in r1)
    gaps = np.diff([0.0] + t)
    assert 0.05 < gaps.mean() < 0.6  # mean inter-arrival 1/rate = 0.2 s
