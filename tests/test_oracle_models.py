"""Pins of the oracle's SU(2) Heisenberg MPO (the benchmark model of Sec. 6.1) and of its stored
reduced entries."""

import os

import numpy as np

from conftest import ROOT
from harness import total_generators
from oracle import SU2, GradedSpace, TensorStructure
from oracle.dense import embed, project
from oracle.models import heisenberg_su2_mpo_dense, heisenberg_two_site
from paper_2508_10076_gb300 import workloads as wl


def _mpo_structure():
    w, p = GradedSpace(SU2, {0: 2, 2: 1}), GradedSpace(SU2, {1: 1})
    return TensorStructure([w, p], [p, w])  # W : W (x) P <- P (x) W


def test_heisenberg_mpo_is_su2_invariant():
    """The dense MPO is annihilated by the total spin generators of W (x) P <- P (x) W, so it
    lies in the span of the canonical tree pairs and projection loses nothing."""
    st = _mpo_structure()
    dense = heisenberg_su2_mpo_dense(1.0)
    for g in total_generators(st):
        assert np.abs(g @ dense.reshape(-1)).max() < 1e-14
    assert np.allclose(embed(st, project(st, dense)), dense, atol=1e-15)


def test_heisenberg_mpo_two_site_operator():
    """End row of the first MPO times start column of the second gives J S.S, built directly
    from S+, S-, Sz; the boundary channels carry the identity."""
    for J in (1.0, 0.7):
        W = heisenberg_su2_mpo_dense(J)
        start, end = 0, 1
        ref = heisenberg_two_site(J)  # [s1', s2', s1, s2]
        # W[end, s1', s1, b] W[b, s2', s2, start] summed over the shared bond b
        got = np.einsum("pib,bqj->pqij", W[end], W[:, :, :, start])
        assert np.allclose(got, ref, atol=1e-15)
        assert np.allclose(W[start, :, :, start], np.eye(2)) and np.allclose(W[end, :, :, end], np.eye(2))
    # S.S on two spins 1/2: singlet energy -3/4, triplet +1/4
    ev = np.linalg.eigvalsh(heisenberg_two_site(1.0).reshape(4, 4))
    assert np.allclose(sorted(ev), [-0.75, 0.25, 0.25, 0.25])


def test_heisenberg_mpo_stored_entries():
    """The golden file (written by tests/golden/make_heisenberg_su2_mpo.py) is the oracle's
    projection bit for bit, and the workload table holds the same values."""
    st = _mpo_structure()
    red = project(st, heisenberg_su2_mpo_dense(1.0))
    vals = []
    with open(os.path.join(ROOT, "tests", "golden", "heisenberg_su2_mpo.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                vals.append(float.fromhex(line))
    assert st.numel == len(vals) == len(wl.HEISENBERG_SU2_MPO)
    assert np.array_equal(np.array(vals), red)
    assert np.array_equal(np.array(wl.HEISENBERG_SU2_MPO), red)
