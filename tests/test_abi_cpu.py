"""The C-ABI library loads and exports every symbol include/dir.h declares;
host-side argument checks run without a GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "dir.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dir_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def dl():
    import paper_0909_0928_gb300 as dl
    return dl


def test_library_exports_every_declared_symbol(dl):
    declared = _declared_symbols()
    assert len(declared) >= 13
    lib = C.CDLL(dl.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(dl.EXPORTS) == declared


def test_params_default_and_status_strings(dl):
    p = dl.dir_params_default()
    assert p.levels == 3 and list(p.iters[:3]) == [200, 100, 50]
    assert p.sigma == 1.0 and p.alpha == 0.4
    assert p.eps == 1e-4 and p.stop_window == 10 and p.use_graph == 1
    assert dl.dir_status_string(0) == "ok"
    assert dl.dir_status_string(dl.DIR_EINVAL) == "invalid argument"
    assert "sm_103a" in dl.dir_version()


def test_struct_layouts_match_header(dl, tmp_path):
    # compile a probe against include/dir.h and compare every field offset
    fields = {"dir_params": [f for f, _ in dl.DirParams._fields_],
              "dir_stats": [f for f, _ in dl.DirStats._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dir.h"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.split("\n") if line)
    for st, cls in (("dir_params", dl.DirParams), ("dir_stats", dl.DirStats)):
        assert int(out[st]) == C.sizeof(cls), st
        for f in fields[st]:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_argument_checks_precede_device_work(dl):
    S = np.zeros((4, 4, 4), np.float32)
    with pytest.raises(dl.DirError) as e:
        dl.dir_create(S, S, (4, 4, 0), (1, 1, 1))
    assert e.value.code == dl.DIR_EINVAL
    with pytest.raises(dl.DirError) as e:
        dl.dir_create(S, S, (4, 4, 4), (1, -1, 1))
    assert e.value.code == dl.DIR_EINVAL
    with pytest.raises(dl.DirError) as e:
        dl.dir_create(S, S, (4, 4, 4), (1, 1, 1), variant=6)
    assert e.value.code == dl.DIR_EINVAL
    with pytest.raises(dl.DirError) as e:
        dl.dir_create(S, S, (4, 4, 4), (1, 1, 1), image_dtype=dl.DIR_F16)
    assert e.value.code == dl.DIR_EUNSUPPORTED
    for bad in (dict(levels=0), dict(levels=9), dict(sigma=0.0), dict(sigma=3.0),
                dict(stop_mode=1, stop_window=0), dict(iters=[-1, 1, 1])):
        p = dl.dir_params_default(**bad)
        with pytest.raises(dl.DirError) as e:
            dl.dir_create(S, S, (4, 4, 4), (1, 1, 1), params=p)
        assert e.value.code == dl.DIR_EINVAL, bad


def test_null_safe_destroy(dl):
    dl._lib.dir_destroy(None)


def test_binding_refuses_buffers_of_the_wrong_size_or_width(dl):
    # the C calls take plain pointers; the binding checks what it can before
    # handing one over
    S = np.zeros((4, 4, 4), np.float32)
    with pytest.raises(ValueError):
        dl.dir_create(S, S[:3], (4, 4, 4), (1, 1, 1))
    with pytest.raises(ValueError):
        dl.dir_create(S.astype(np.float64), S.astype(np.float64), (4, 4, 4), (1, 1, 1))
    with pytest.raises(ValueError):
        dl.dir_create(S, S, (4, 4, 4), (1, 1, 1), image_dtype=dl.DIR_I16)
    with pytest.raises(ValueError):
        dl.dir_create(S, S, (4, 4, 5), (1, 1, 1))


def test_noalloc_binding_checks_buffers_before_the_call(dl):
    # the library reads N floats from each image and writes 3N to field_out:
    # wrong sizes, widths, host memory or a missing output never reach it
    torch = pytest.importorskip("torch")
    dims = (8, 6, 4)
    n = 8 * 6 * 4
    good = torch.zeros(n, dtype=torch.float32)
    with pytest.raises(ValueError):
        dl.dir_register_noalloc(good, good, dims, 0, None, None)
    with pytest.raises(ValueError):
        dl.dir_register_noalloc(torch.zeros(n - 1), good, dims, 0, None, torch.zeros(3 * n))
    with pytest.raises(ValueError):
        dl.dir_register_noalloc(good, torch.zeros(n, dtype=torch.int16), dims, 0, None,
                                torch.zeros(3 * n))
    with pytest.raises(ValueError):
        dl.dir_register_noalloc(good, good, dims, 0, None, torch.zeros(2 * n))
    with pytest.raises(ValueError):   # correct sizes, but host tensors
        dl.dir_register_noalloc(good, good, dims, 0, None, torch.zeros(3 * n))
    with pytest.raises(ValueError):   # numpy arrays are host memory
        dl.dir_register_noalloc(np.zeros(n, np.float32), np.zeros(n, np.float32), dims, 0,
                                None, np.zeros(3 * n, np.float32))
