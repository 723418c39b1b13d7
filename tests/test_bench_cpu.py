"""Host-side pieces of bench.py that need no GPU: the source hash that ties a
recorded ncu traffic figure to the kernel code it was taken on."""
import os

import bench


def test_code_hash_ignores_comments_and_blank_lines():
    a = "int f(int x) {\n    return x + 1;  // add one\n}\n"
    b = "/* doc\n   block */\nint f(int x) {\n\n    return x + 1;\n}   \n"
    c = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_traffic_records_name_existing_sources():
    # every committed traffic record names its kernel's source files, and
    # those files exist; the figure is used only while their code is unchanged
    prof = os.path.join(bench.ROOT, "profiles")
    for name in os.listdir(prof):
        if not name.endswith("_traffic.txt"):
            continue
        kernel = name[: -len("_traffic.txt")]
        assert kernel in bench.KERNEL_SOURCES, kernel
        for f in bench.KERNEL_SOURCES[kernel]:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_0909_0928_gb300", "csrc", f))
        rec = dict(line.split(":", 1) for line in open(os.path.join(prof, name)) if ":" in line)
        assert float(rec["dram_bytes_per_launch_full_size"]) > 0
        assert len(rec["source_sha256"].strip()) == 64
