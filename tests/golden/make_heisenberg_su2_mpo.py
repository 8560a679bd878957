"""Writes heisenberg_su2_mpo.txt: the reduced blocks of the SU(2) Heisenberg MPO (J = 1) in the
storage order of W : W (x) P <- P (x) W, W = 2 (0) (+) (1), P = (1/2), projected by the oracle.

Run from the repository root: python tests/golden/make_heisenberg_su2_mpo.py
"""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import SU2, GradedSpace, TensorStructure  # noqa: E402
from oracle.dense import project  # noqa: E402
from oracle.models import heisenberg_su2_mpo_dense  # noqa: E402


def main():
    w, p = {0: 2, 2: 1}, {1: 1}
    st = TensorStructure([GradedSpace(SU2, w), GradedSpace(SU2, p)], [GradedSpace(SU2, p), GradedSpace(SU2, w)])
    red = project(st, heisenberg_su2_mpo_dense(1.0))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "heisenberg_su2_mpo.txt")
    with open(out, "w") as fh:
        fh.write("# SU(2) Heisenberg MPO, J = 1: reduced entries of W : W (x) P <- P (x) W in storage order\n")
        fh.write("# (W = 2 (0) (+) (1), P = (1/2)); written by make_heisenberg_su2_mpo.py from the oracle\n")
        for v in red:
            fh.write(f"{float(v).hex()}  # {float(v)!r}\n")


if __name__ == "__main__":
    main()
