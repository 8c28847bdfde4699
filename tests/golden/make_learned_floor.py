"""Writes learned_floor_sigma2.txt: the smallest relative L2 error any
width-w gridding (any tap table, any per-mode correction) can reach in the
sigma = 2 NUFFT of Eq. 8 (Sec. 2, after Eq. 9) for independent random-phase
sample values, next to the ES kernel's error at beta = 2.30 w.  Calls only
oracle/ (oracle.learned_floor).  Run from the repository root:
    python tests/golden/make_learned_floor.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import learned_floor as F  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "learned_floor_sigma2.txt")


def main() -> None:
    lines = [
        "# Width floor of the gridding step of the NUFFT that evaluates Eq. 8 (Sec. 2, after",
        "# Eq. 9), sigma = 2, sample offsets uniform, sample values independent with zero mean.",
        "# Written by tests/golden/make_learned_floor.py from oracle/learned_floor.py",
        "# (variable projection, delta grid 128, omega grid 256).  Columns:",
        "# width  floor_rel_l2_1d  floor_rel_l2_2d  es_rel_l2_1d  es_rel_l2_2d  (ES beta = 2.30 w)",
    ]
    for w in (3, 4, 5, 6, 7):
        e1, *_ = F.floor_1d(w)
        es = F.es_error_1d(w, 2.30 * w)
        lines.append("%d %.4e %.4e %.4e %.4e" % (
            w, np.sqrt(e1), np.sqrt(F.floor_2d_from_1d(e1)), np.sqrt(es),
            np.sqrt(F.floor_2d_from_1d(es))))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
