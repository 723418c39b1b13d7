"""Serving loop: continuous batching over several streams.

A job's result must not depend on what else is on the GPU: every registration
is computed alone (one slot) and again in a mix of concurrent jobs admitted as
slots and memory free up; the fields must agree.  The reductions use atomics
(their summation order varies) but the field does not depend on them, so the
fields are compared exactly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _requests(dl, serve):
    from phantom import make_blob_pair
    reqs = []
    shapes = [(48, 40, 24), (64, 48, 32), (40, 40, 40), (72, 56, 20), (64, 64, 32), (33, 45, 27)]
    for k, dims in enumerate(shapes):
        S, M = make_blob_pair(dims, (1.0, -0.5, 0.5), seed=20 + k, n_blobs=20, sigma_vox=3.0,
                              noise=0.5)
        params = dl.dir_params_default(levels=2, iters=[15, 10])
        reqs.append(serve.Request(rid=k, S=S, M=M, spacing=(1.0, 1.0, 2.0), variant=k % 6,
                                  params=params, arrival=0.002 * k))
    return reqs


@pytest.mark.gpu
def test_same_result_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0909_0928_gb300 as dl
    from paper_0909_0928_gb300 import serve
    alone = {}
    for req in _requests(dl, serve):
        srv = serve.Server(slots=1)
        (done,) = srv.run([req], realtime=False)
        alone[done.rid] = done.field
    srv = serve.Server(slots=4)
    mixed = srv.run(_requests(dl, serve), realtime=True)
    assert len(mixed) == len(alone)
    for r in mixed:
        assert r.field is not None
        diff = float(np.abs(r.field - alone[r.rid]).max())
        assert diff == 0.0, f"job {r.rid}: alone vs mix differ by {diff}"
        assert r.done >= r.admitted >= r.arrival


@pytest.mark.gpu
def test_admission_respects_the_memory_budget():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0909_0928_gb300 as dl
    from paper_0909_0928_gb300 import serve
    reqs = _requests(dl, serve)
    biggest = max(serve.footprint_bytes(r.dims, r.params.levels) for r in reqs)
    srv = serve.Server(slots=6, hbm_budget_bytes=2 * biggest + 1)
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
