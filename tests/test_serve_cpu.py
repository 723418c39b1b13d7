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


def test_footprint_counts_the_difference_image_scratch():
    # Eqs. 3-6 under the default schedule hold u and D = W - S of the finest
    # level (4 floats per voxel; Eq. 6: 5), Eqs. 1-2 and other schedules do not
    from paper_0909_0928_gb300 import serve, dir_params_default
    S = np.zeros((64, 96, 128), np.int16)
    n0 = 128 * 96 * 64

    def need(variant, **kw):
        p = dir_params_default(levels=3, **kw)
        return serve.request_footprint(serve.Request(rid=0, S=S, M=S, spacing=(1, 1, 1),
                                                     variant=variant, params=p))
    base = need(0)
    assert need(1) == base and need(2, fuse=0) == base and need(5, plain_kernels=1) == base
    assert need(2) >= base + 4 * n0 * 4 and need(3, fuse=4) == need(2)
    assert need(5) >= need(2) + n0 * 4
