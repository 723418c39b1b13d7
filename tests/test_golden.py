"""The FP64 oracle against values evaluated by hand (tests/golden/).

force_laws_by_hand.txt holds the demons force of Eqs. (1)-(6) at single
voxels as exact fractions, each line with its derivation; the oracle's force
must reproduce them to FP64 rounding.
"""
import os
from fractions import Fraction

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases(name):
    out = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            inputs, expected, source = (part.split() for part in line.split("|"))
            vals = [float(Fraction(t)) for t in inputs]
            out.append((int(vals[0]), vals[1:], [float(Fraction(t)) for t in expected],
                        " ".join(source)))
    return out


def test_force_laws_by_hand():
    cases = _cases("force_laws_by_hand.txt")
    assert len(cases) >= 18 and {c[0] for c in cases} == set(range(6))
    for variant, (alpha, d, gsx, gsy, gsz, gmx, gmy, gmz, b), want, source in cases:
        dr = oracle.force(variant, np.array([d]), np.array([[gsx], [gsy], [gsz]]),
                          np.array([[gmx], [gmy], [gmz]]), np.array([b]), alpha=alpha)
        got = dr[:, 0]
        assert np.allclose(got, want, rtol=4e-16, atol=1e-300), (source, got, want)
