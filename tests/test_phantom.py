"""The seeded input generator: determinism, shapes and the true deformation."""
import numpy as np

from phantom import SMALL, SplitMix64Stream, make_lung_phantom, make_wave_pair, true_field_mm
from phantom.generator import _build_geometry, backward_map_mm


def test_splitmix64_reference_values():
    # SplitMix64 with state 0 (published test vector of the algorithm):
    # first outputs for seed 0 are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4
    from phantom.generator import _GAMMA, _mix64
    s = np.array([1, 2], dtype=np.uint64) * _GAMMA
    out = _mix64(s)
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_streams_are_deterministic_and_distinct():
    a = SplitMix64Stream(5, 1).uniform(10)
    b = SplitMix64Stream(5, 1).uniform(10)
    c = SplitMix64Stream(5, 2).uniform(10)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    n = SplitMix64Stream(9, 3).normal(20000)
    assert abs(n.mean()) < 0.03 and abs(n.std() - 1.0) < 0.03


def test_small_phantom_shapes_and_values(small_phantom):
    p = small_phantom
    assert p["S"].shape == (32, 64, 64) and p["S"].dtype == np.float32
    assert p["M"].shape == p["S"].shape
    assert p["landmarks"].shape == (SMALL.n_landmarks, 3)
    # background air, lung parenchyma and vessels are all present
    S = p["S"]
    assert (S < -950).mean() > 0.05 and (np.abs(S + 850) < 60).mean() > 0.05
    assert (S > 0).mean() > 0.001
    q = make_lung_phantom(SMALL)
    assert np.array_equal(q["S"], p["S"]) and np.array_equal(q["M"], p["M"])


def test_true_field_solves_the_backward_map(small_phantom):
    # u = -v*(p + u)  <=>  M(p + u) = S_clean(p)
    g = _build_geometry(SMALL)
    lm = small_phantom["landmarks"]
    u = true_field_mm(g, lm)
    sp = np.asarray(SMALL.spacing)
    resid = u + backward_map_mm(g, lm * sp + u)
    assert np.abs(resid).max() < 1e-8
    mag = np.linalg.norm(u, axis=1)
    assert 1.0 < mag.mean() < SMALL.a_max_mm + 5.0


def test_wave_pair_is_a_pure_shift():
    # M(y) = S(y - T): for an integer T the moving volume is the static one
    # moved by T voxels, value for value
    S, M = make_wave_pair((40, 30, 20), (2, 3, 1), seed=4)
    assert S.shape == (20, 30, 40) and S.dtype == np.float32
    assert np.array_equal(M[1:, 3:, 2:], S[:-1, :-3, :-2])
    S2, M2 = make_wave_pair((40, 30, 20), (2, 3, 1), seed=4)
    assert np.array_equal(S, S2) and np.array_equal(M, M2)
    assert not np.array_equal(S, make_wave_pair((40, 30, 20), (2, 3, 1), seed=5)[0])
