"""Serving loop: continuous batching over several streams with resident contexts.

A job's result must not depend on what else is on the GPU or on which
resident context served it: every registration is computed alone (a fresh
server, one slot) and again in a mix of concurrent jobs admitted as slots and
memory free up, where contexts are reused between requests of the same shape;
the fields must agree bit for bit (the reductions use atomics, whose
summation order varies, but the field does not depend on them).  Served
fields are also held to the oracle on a short schedule."""
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


def _requests(dl, serve, repeat=1):
    from phantom import make_blob_pair
    reqs = []
    shapes = [(48, 40, 24), (64, 48, 32), (40, 40, 40), (72, 56, 20), (64, 64, 32), (33, 45, 27)]
    for rep in range(repeat):
        for k, dims in enumerate(shapes):
            S, M = make_blob_pair(dims, (1.0, -0.5, 0.5), seed=20 + k + 7 * rep, n_blobs=20,
                                  sigma_vox=3.0, noise=0.5)
            params = dl.dir_params_default(levels=2, iters=[15, 10])
            reqs.append(serve.Request(rid=len(reqs), S=S, M=M, spacing=(1.0, 1.0, 2.0),
                                      variant=k % 6, params=params,
                                      arrival=0.002 * len(reqs)))
    return reqs


def test_same_result_alone_and_in_the_mix(dl):
    from paper_0909_0928_gb300 import serve
    alone = {}
    for req in _requests(dl, serve, repeat=2):
        srv = serve.Server(slots=1, reuse=False)
        (done,) = srv.run([req], realtime=False)
        alone[done.rid] = done.field
    # the second round of six shapes runs in contexts the first round left
    srv = serve.Server(slots=4, reuse=True)
    mixed = srv.run(_requests(dl, serve, repeat=2), realtime=True)
    assert len(mixed) == len(alone)
    assert srv.reused >= 1 and srv.created + srv.reused == len(mixed)
    for r in mixed:
        assert r.field is not None
        diff = float(np.abs(r.field - alone[r.rid]).max())
        assert diff == 0.0, f"job {r.rid}: alone vs mix differ by {diff}"
        assert r.done >= r.admitted >= r.arrival
    srv.close()
    assert srv.in_use == 0


def test_resident_context_serves_a_new_pair_like_a_fresh_one(dl):
    # dir_load into a context that already registered another pair of the
    # same size gives the field a fresh context gives
    from paper_0909_0928_gb300 import serve
    from phantom import make_blob_pair
    dims = (56, 48, 30)
    pairs = [make_blob_pair(dims, (0.8, -0.6, 0.4), seed=s, n_blobs=25, sigma_vox=3.0, noise=0.5)
             for s in (3, 4, 5)]
    params = dl.dir_params_default(levels=2, iters=[12, 8])
    mk = lambda k, S, M: serve.Request(rid=k, S=S, M=M, spacing=(1, 1, 2), variant=5,
                                       params=params)
    srv = serve.Server(slots=1, reuse=True)
    served = [srv.run([mk(k, S, M)], realtime=False)[0].field for k, (S, M) in enumerate(pairs)]
    assert srv.created == 1 and srv.reused == 2
    srv.close()
    for k, (S, M) in enumerate(pairs):
        fresh = serve.Server(slots=1, reuse=False).run([mk(k, S, M)], realtime=False)[0].field
        assert np.array_equal(served[k], fresh), k


@pytest.mark.parametrize("variant", [0, 5])
def test_served_int16_jobs_match_the_oracle(dl, variant):
    # int16 HU lung phantoms, 3-level pyramid (the serving mix's form) on a
    # short schedule: every voxel within 1e-3 of the FP64 oracle
    import oracle
    from paper_0909_0928_gb300 import serve
    from parity_criteria import TOL_U, strict_check
    from phantom import PhantomSpec, make_lung_phantom
    spec = PhantomSpec(dims=(96, 80, 48), spacing=(0.9, 0.9, 2.5), seed=40 + variant,
                       a_max_mm=15.0, compression=0.15, compression_region="lower",
                       n_landmarks=10)
    ph = make_lung_phantom(spec)
    S16, M16 = np.round(ph["S"]).astype(np.int16), np.round(ph["M"]).astype(np.int16)
    params = dl.dir_params_default(levels=3, iters=[6, 4, 2])
    srv = serve.Server(slots=2, reuse=True)
    reqs = [serve.Request(rid=k, S=S16, M=M16, spacing=spec.spacing, variant=variant,
                          params=params) for k in range(2)]
    done = srv.run(reqs, realtime=False)
    srv.close()
    ref = oracle.register(S16.astype(np.float64), M16.astype(np.float64), variant=variant,
                          levels=3, iters=[6, 4, 2])["u"]
    for r in done:
        err = np.abs(r.field.astype(np.float64) - ref).max(axis=0)
        strict_check(err, f"served job {r.rid} v{variant}", TOL_U)
        print(f"served int16 v{variant} job {r.rid}: max|du| {err.max():.2e}")


def test_admission_respects_the_memory_budget(dl):
    from paper_0909_0928_gb300 import serve
    reqs = _requests(dl, serve)
    biggest = max(serve.request_footprint(r) for r in reqs)
    srv = serve.Server(slots=6, hbm_budget_bytes=2 * biggest + 1, reuse=True)
    peak = {"jobs": 0, "bytes": 0}
    orig = srv._admit

    def admit_and_watch():
        orig()
        peak["jobs"] = max(peak["jobs"], len(srv.running))
        peak["bytes"] = max(peak["bytes"], srv.in_use)

    srv._admit = admit_and_watch
    done = srv.run(reqs, realtime=False)
    assert len(done) == len(reqs)
    assert peak["bytes"] <= srv.budget
    assert 1 <= peak["jobs"] <= len(reqs)
    assert srv.evicted >= 1   # six shapes cannot all stay resident in this budget
    srv.close()
