"""Batched registrations (one captured graph over many contexts) and the
launch-shape autotuner.

A registration's field does not depend on how its kernels are grouped or
shaped: the batch runs the same per-voxel arithmetic as a plain dir_register,
either as grouped launches over all the pairs of a level (one launch per
iteration step for the whole batch) or as each registration on concurrent
graph branches, and the autotuner changes only how many voxels a thread or
block covers.  So fields are
compared exactly with plain single registrations, and batched fields are held
to the FP64 oracle on every voxel (the short schedule keeps the oracle's own
single-precision sensitivity far below the bar)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0909_0928_gb300 as dl
    return dl


# uneven pairs: (dims, variant, image dtype)
CASES = [((48, 40, 24), 0, "f32"), ((64, 48, 32), 5, "i16"), ((40, 40, 40), 5, "f32"),
         ((72, 56, 20), 0, "i16"), ((96, 80, 36), 0, "f32"), ((33, 45, 27), 5, "f32"),
         ((128, 96, 48), 5, "i16")]


def _pair(k, dims, dtype):
    from phantom import make_blob_pair
    S, M = make_blob_pair(dims, (1.0, -0.5, 0.5), seed=40 + k, n_blobs=20, sigma_vox=3.0,
                          noise=0.5)
    if dtype == "i16":  # integer intensities, stored as int16
        return (np.round(S * 100).astype(np.int16), np.round(M * 100).astype(np.int16))
    return S, M


def _ctx(dl, S, M, variant, iters=(20, 12, 8)):
    nz, ny, nx = S.shape
    params = dl.dir_params_default(levels=3, iters=list(iters))
    St, Mt = torch.from_numpy(S).cuda(), torch.from_numpy(M).cuda()
    dt = dl.DIR_I16 if S.dtype == np.int16 else dl.DIR_F32
    return dl.dir_create(St, Mt, (nx, ny, nz), (1.0, 1.0, 2.0), dt, True, variant, params,
                         torch.cuda.current_stream())


def _field(dl, ctx, shape):
    out = np.empty((3,) + shape, np.float32)
    dl.dir_get_field(ctx, out)
    return out


def test_batch_equals_plain_registrations(dl):
    pairs = [_pair(k, d, t) for k, (d, _, t) in enumerate(CASES)]
    plain = []
    for (S, M), (_, v, _) in zip(pairs, CASES):
        ctx = _ctx(dl, S, M, v)
        try:
            dl.dir_register(ctx)
            plain.append(_field(dl, ctx, S.shape))
        finally:
            dl.dir_destroy(ctx)
    ctxs = [_ctx(dl, S, M, v) for (S, M), (_, v, _) in zip(pairs, CASES)]
    batch = None
    try:
        for grouped, branches in ((True, 8), (False, 3), (False, 8)):
            batch = dl.dir_batch_create(ctxs, branches=branches,
                                        stream=torch.cuda.current_stream(), grouped=grouped)
            assert dl.dir_batch_grouped(batch) == grouped
            for rep in range(2):  # a replay gives the same fields again
                ms = dl.dir_batch_run(batch)
                assert ms > 0.0
                for k, ctx in enumerate(ctxs):
                    f = _field(dl, ctx, pairs[k][0].shape)
                    assert np.array_equal(f, plain[k]), (
                        f"pair {k} grouped {grouped} branches {branches} rep {rep}")
                    h = dl.dir_get_history(ctx, 40)
                    assert h.shape[0] == 40 and np.all(np.isfinite(h[:, 0]))
            dl.dir_batch_destroy(batch)
            batch = None
        # every batched field against the FP64 oracle, every voxel
        import oracle
        from parity_criteria import TOL_U, strict_check
        for k, ((S, M), (_, v, _)) in enumerate(zip(pairs, CASES)):
            ref = oracle.register(S.astype(np.float64), M.astype(np.float64), variant=v,
                                  levels=3, iters=[20, 12, 8])["u"]
            err = np.abs(_field(dl, ctxs[k], S.shape).astype(np.float64) - ref).max(axis=0)
            strict_check(err, f"batched pair {k} v{v}", TOL_U)
        # contexts stay usable on their own after the batch is gone
        dl.dir_register(ctxs[0])
        assert np.array_equal(_field(dl, ctxs[0], pairs[0][0].shape), plain[0])
    finally:
        dl.dir_batch_destroy(batch)
        for c in ctxs:
            dl.dir_destroy(c)


@pytest.mark.parametrize("variant", [0, 2])
def test_grouped_batch_over_many_pairs_and_its_fallback(dl, variant):
    # 18 pairs of one force law: two launches of at most 16 jobs per step
    # (Eq. 3: of the z + D and stencil force kernels, each job writing u and D
    # to its own context's scratch).
    # The fields agree with plain registrations bit for bit; the histories to
    # single-precision rounding, because a grouped launch picks one brick
    # depth for the whole group and so partitions the FP32 per-block partial
    # sums differently.  A context with a stop test makes the batch fall back
    # to branches.
    dims = [(24 + 4 * (k % 5), 20 + 4 * (k % 3), 12 + 2 * (k % 4)) for k in range(18)]
    pairs = [_pair(100 + k, d, "f32") for k, d in enumerate(dims)]
    plain, hist = [], []
    for S, M in pairs:
        ctx = _ctx(dl, S, M, variant, iters=(6, 4, 3))
        try:
            dl.dir_register(ctx)
            plain.append(_field(dl, ctx, S.shape))
            hist.append(dl.dir_get_history(ctx, 13))
        finally:
            dl.dir_destroy(ctx)
    ctxs = [_ctx(dl, S, M, variant, iters=(6, 4, 3)) for S, M in pairs]
    batch = None
    try:
        batch = dl.dir_batch_create(ctxs, stream=torch.cuda.current_stream())
        assert dl.dir_batch_grouped(batch)
        dl.dir_batch_run(batch)
        for k, ctx in enumerate(ctxs):
            assert np.array_equal(_field(dl, ctx, pairs[k][0].shape), plain[k]), f"pair {k}"
            np.testing.assert_allclose(dl.dir_get_history(ctx, 13), hist[k], rtol=1e-5,
                                       atol=1e-9)
        dl.dir_batch_destroy(batch)
        batch = None
        S, M = pairs[0]
        nz, ny, nx = S.shape
        p = dl.dir_params_default(levels=3, iters=[6, 4, 3], stop_mode=1)
        odd = dl.dir_create(torch.from_numpy(S).cuda(), torch.from_numpy(M).cuda(), (nx, ny, nz),
                            (1.0, 1.0, 2.0), dl.DIR_F32, True, variant, p,
                            torch.cuda.current_stream())
        try:
            batch = dl.dir_batch_create(ctxs[:3] + [odd], stream=torch.cuda.current_stream())
            assert not dl.dir_batch_grouped(batch)
            dl.dir_batch_run(batch)
            for k in range(3):
                assert np.array_equal(_field(dl, ctxs[k], pairs[k][0].shape), plain[k])
        finally:
            dl.dir_batch_destroy(batch)
            batch = None
            dl.dir_destroy(odd)
    finally:
        dl.dir_batch_destroy(batch)
        for c in ctxs:
            dl.dir_destroy(c)


def test_grouped_batch_correlation(dl):
    # the correlation sums of every iteration through the grouped launches:
    # the plain registration's values (the sums are partitioned differently,
    # so to single-precision rounding), the fields bit for bit
    pairs = [_pair(200 + k, (40 + 8 * k, 36, 24), "f32") for k in range(4)]
    ctxs, plain, rho0 = [], [], []
    for k, (S, M) in enumerate(pairs):
        nz, ny, nx = S.shape
        p = dl.dir_params_default(levels=3, iters=[8, 6, 4], correlation=1)
        c = dl.dir_create(torch.from_numpy(S).cuda(), torch.from_numpy(M).cuda(), (nx, ny, nz),
                          (1.0, 1.0, 2.0), dl.DIR_F32, True, 5 if k % 2 else 0, p,
                          torch.cuda.current_stream())
        ctxs.append(c)
        dl.dir_register(c)
        plain.append(_field(dl, c, S.shape))
        rho0.append(dl.dir_get_correlation(c, 18))
    batch = None
    try:
        batch = dl.dir_batch_create(ctxs, stream=torch.cuda.current_stream())
        assert dl.dir_batch_grouped(batch)
        dl.dir_batch_run(batch)
        for k, c in enumerate(ctxs):
            assert np.array_equal(_field(dl, c, pairs[k][0].shape), plain[k])
            rho = dl.dir_get_correlation(c, 18)
            assert rho.shape == rho0[k].shape == (18,)
            np.testing.assert_allclose(rho, rho0[k], rtol=0, atol=1e-6)
    finally:
        dl.dir_batch_destroy(batch)
        for c in ctxs:
            dl.dir_destroy(c)


def test_batch_argument_errors(dl):
    S, M = _pair(0, (32, 24, 16), "f32")
    c = _ctx(dl, S, M, 0, iters=(2, 2, 2))
    try:
        with pytest.raises(dl.DirError):
            dl.dir_batch_create([c, c])           # the same context twice
        with pytest.raises(dl.DirError):
            dl.dir_batch_create([c], branches=0)
        with pytest.raises(dl.DirError):
            dl.dir_autotune(c)                    # needs a finished registration first
    finally:
        dl.dir_destroy(c)


@pytest.mark.parametrize("variant", [0, 5])
def test_autotune_keeps_the_field(dl, variant):
    S, M = _pair(3, (120, 100, 40), "f32")
    ctx = _ctx(dl, S, M, variant, iters=(15, 10, 6))
    try:
        dl.dir_register(ctx)
        before = _field(dl, ctx, S.shape)
        shapes = dl.dir_autotune(ctx, reps=3, levels=3)
        for depth, zc in shapes:  # 6: the split schedule's z + force kernel
            assert depth in (1, 2, 4, 6, 8) and zc >= 0
        after_tune = _field(dl, ctx, S.shape)     # the registered field is kept
        assert np.array_equal(after_tune, before)
        dl.dir_register(ctx)                      # re-captured with the tuned shapes
        assert np.array_equal(_field(dl, ctx, S.shape), before)
    finally:
        dl.dir_destroy(ctx)
