"""dir_register_noalloc: the registration for callers that cannot allocate
device memory (their pool owns the device, or allocation is forbidden where
they run).  It must give the same field as the allocating entry points
(dir_create + dir_register + dir_get_field) on consecutive calls that share its
static scratch, reserve no device memory per call, and refuse volumes that do
not fit the scratch.  Collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5  # voxel; same kernels and launch shapes, so the fields agree closely


@pytest.fixture(scope="module")
def dl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0909_0928_gb300 as dl
    return dl


def _with_context(dl, S, M, variant, params):
    with dl.Registration(torch.from_numpy(S).cuda(), torch.from_numpy(M).cuda(), (1, 1, 1),
                         variant, params, torch.cuda.current_stream()) as reg:
        reg.register()
        return reg.field()


# the scratch layout changes with the element size of the field (2 bytes for
# BF16, 8 for FP64, whose images are 8 bytes too), and the field export
# converts from each of them
FORMS = {"f32": {}, "bf16_field": {"field_dtype": 3}, "f64": {"precision": 4}}


@pytest.mark.parametrize("form", list(FORMS))
def test_noalloc_matches_allocating_path_on_consecutive_calls(dl, form):
    from phantom import SMALL, make_lung_phantom
    p = make_lung_phantom(SMALL)
    S, M = p["S"], p["M"]
    nz, ny, nx = S.shape
    params = dl.dir_params_default(levels=2, iters=[8, 6], **FORMS[form])
    St, Mt = torch.from_numpy(S).cuda(), torch.from_numpy(M).cuda()
    out = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # two calls in a row with different force laws: the second must not see
    # anything the first left in the shared scratch
    for variant in (dl.DIR_PASSIVE, dl.DIR_INVERSE_CONSISTENT):
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = dl.dir_register_noalloc(St, Mt, (nx, ny, nz), variant, params, out, stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert st.iters_run[0] == 8 and st.iters_run[1] == 6
        want = _with_context(dl, S, M, variant, params)
        got = out.cpu().numpy()
        err = float(np.abs(got - want).max())
        assert err <= TOL, f"{form} variant {variant}: max |du| {err:.3e}"
        if variant == dl.DIR_INVERSE_CONSISTENT:
            # the first call on this device already looked up the scratch; this
            # one must not take device memory
            assert abs(free_before - free_after) < (2 << 20)


def test_noalloc_rejects_volumes_beyond_the_scratch(dl):
    S = torch.zeros((160, 256, 256), dtype=torch.float32, device="cuda")
    out = torch.empty((3,) + tuple(S.shape), dtype=torch.float32, device="cuda")
    with pytest.raises(dl.DirError) as e:
        dl.dir_register_noalloc(S, S, (256, 256, 160), dl.DIR_PASSIVE, None, out,
                                torch.cuda.current_stream())
    assert e.value.code == dl.DIR_EINVAL
    assert "MiB" in str(e.value)
