"""The seeded workload definitions and their oracle evaluation (CPU)."""

import numpy as np
import pytest

from harness import oracle_heff, oracle_heff_inputs, ostruct
from oracle.dense import embed
from paper_2508_10076_gb300 import workloads as wl


def test_multiplicity_laws():
    v = wl.u1_virtual(1024)
    assert sum(v.values()) == 1024 and min(v) == -16 and max(v) == 16 and v[0] == max(v.values())
    assert sum(wl.u1_virtual(4096).values()) == 4096
    s = wl.su2_virtual(256)
    assert [s[tj] for tj in range(9)] == [64, 60, 49, 36, 23, 13, 7, 3, 1]
    assert sum((tj + 1) * n for tj, n in s.items()) == 750
    assert sum(wl.su2_virtual(512).values()) == 512


def test_xxz_mpo_two_site_hamiltonian():
    """W W contracted with the boundary bond states (4 on the left, 0 on the right) is the
    two-site XXZ Hamiltonian Jz Sz Sz + Jxy/2 (S+ S- + S- S+) (reading of the XXZ workload)."""
    from harness import oracle_mpo
    st = ostruct("U1", wl.heff_legs(*wl.heff_spaces("U1", 8))["W"])
    jz, jxy = 0.7, 1.3
    w = embed(st, oracle_mpo(st, wl.xxz_mpo_entries(jz, jxy)))   # [w_l, s', s, w_r]
    # dense bond order of W = {-2:1, 0:3, 2:1}: bond states 1 | 0, 3, 4 | 2
    left, right = 3, 1          # bond state 4 and bond state 0
    two = np.einsum("psk,kqt->pqst", w[left], w[:, :, :, right])   # [s1', s2', s1, s2]
    sz = np.diag([-0.5, 0.5])   # physical dense order: charge -1, then +1
    sp = np.array([[0.0, 0.0], [1.0, 0.0]])
    H = jz * np.kron(sz, sz) + 0.5 * jxy * (np.kron(sp, sp.T) + np.kron(sp.T, sp))
    assert np.allclose(two, H.reshape(2, 2, 2, 2))


def test_oracle_heff_dense_equals_block_small():
    for sym, D in (("U1", 24), ("SU2", 12)):
        a = oracle_heff(sym, D, tier="dense")
        b = oracle_heff(sym, D, tier="block")
        for (sa, da), (sb, db) in zip(a, b):
            assert sa.blocks == sb.blocks
            assert np.allclose(da, db, atol=1e-10 * max(1.0, np.abs(da).max()))


def test_heff_output_has_structure_of_x():
    st, _ = oracle_heff_inputs("U1", 16)
    out = oracle_heff("U1", 16, steps=4)[-1][0]
    assert out.blocks == st["x"].blocks


def test_serving_request_stream_is_seeded_and_mixed():
    from paper_2508_10076_gb300.serve import dimension_grid, request_stream
    grid = dimension_grid()
    assert grid[0] == 64 and grid[-1] == 4096 and len(grid) == 25
    a, b = request_stream(4000, seed=3), request_stream(4000, seed=3)
    assert a == b
    syms = {r["sym"] for r in a}
    dts = {r["dtype"] for r in a}
    assert syms == {"U1", "SU2"} and dts == {"f64", "c128"}
    frac_u1 = sum(r["sym"] == "U1" for r in a) / len(a)
    frac_c = sum(r["dtype"] == "c128" for r in a) / len(a)
    assert abs(frac_u1 - 0.5) < 0.05 and abs(frac_c - 0.5) < 0.05
    assert all(r["D"] in grid for r in a)
    # log-uniform: about as many draws below sqrt(64 * 4096) = 512 as above
    below = sum(r["D"] < 512 for r in a) / len(a)
    assert 0.4 < below < 0.6


def test_single_site_heff_dense_equals_block_and_keeps_structure():
    """Algorithm 11 chain on small spaces: the oracle's dense tier (explicit CG embedding) and
    block tier agree, and x' has the block structure of x, for U(1) and SU(2)."""
    from harness import oracle_heff, oracle_heff_inputs
    for sym, D in (("U1", 24), ("SU2", 10)):
        st, _ = oracle_heff_inputs(sym, D, sites=1)
        blk = oracle_heff(sym, D, sites=1, tier="block")
        den = oracle_heff(sym, D, sites=1, tier="dense")
        assert len(blk) == 3
        for (sb, db), (sd, dd) in zip(blk, den):
            assert sb.blocks == sd.blocks
            assert np.allclose(db, dd, rtol=1e-12, atol=1e-12 * max(1.0, float(np.abs(dd).max())))
        assert blk[-1][0].blocks == st["x"].blocks
