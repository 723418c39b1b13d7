"""Builds the oracle's C library (single-threaded and OpenMP forms) in place.

Test infrastructure: compiling the checker is part of the build, using it is
reserved for the tests, the smoke check and the benchmark's CPU baseline.
Flags avoid anything machine-specific, and -ffp-contract=off keeps fused
multiply-adds out so x86_64 and aarch64 builds round identically.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "demons_oracle.c")
_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def library_path(threaded: bool = False) -> str:
    return os.path.join(_HERE, "liboracle_omp.so" if threaded else "liboracle.so")


def build_commands() -> list[list[str]]:
    cc = os.environ.get("CC", "gcc")
    return [
        [cc, *_FLAGS, _SRC, "-o", library_path(False), "-lm"],
        [cc, *_FLAGS, "-fopenmp", _SRC, "-o", library_path(True), "-lm"],
    ]


def build() -> None:
    procs = [subprocess.Popen(cmd) for cmd in build_commands()]
    for cmd, p in zip(build_commands(), procs):
        if p.wait() != 0:
            raise RuntimeError("oracle build failed: " + " ".join(cmd))


if __name__ == "__main__":
    build()
