"""The paper's printed 1D results (tests/golden/sec3_line_abs_errors.txt, Sec. 3):
with the readings of the unstated layout and normalisation, the FP64 oracle's
Eq. 7 (which Eq. 8 evaluates) against its Eq. 2 reproduces the order of
magnitude of the printed largest intensity differences.  CPU only."""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle import line as oline
from paper_1203_3583_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "sec3_line_abs_errors.txt")


def printed():
    vals = {}
    for ln in open(GOLDEN):
        ln = ln.split("#", 1)[0].split()
        if len(ln) == 2:
            vals[ln[0]] = float(ln[1])
    return vals


@pytest.mark.parametrize("shape", ["facets", "quadratic"])
def test_sec3_difference_order_of_magnitude(shape):
    x1, d1, w = W.line_facets() if shape == "facets" else W.line_quadratic()
    g = W.line_geometry()
    u1 = np.ones(x1.size, np.complex128)
    i7 = np.abs(oline.line(g, x1, d1, w, u1, 7)) ** 2
    i2 = np.abs(oline.line(g, x1, d1, w, u1, 2)) ** 2
    diff = float(np.max(np.abs(i7 - i2)) / np.max(i2))
    want = printed()[shape]
    assert want / 3 < diff < want * 3, (shape, diff, want)
