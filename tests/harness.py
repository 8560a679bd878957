"""Oracle-side construction of the seeded workloads (tests only)."""

import numpy as np

from oracle import GradedSpace, TensorStructure, sym_from_name
from oracle import ops
from paper_2508_10076_gb300 import workloads as wl


def ostruct(sym, legs):
    s = sym_from_name(sym)
    cod, dom = legs
    return TensorStructure([GradedSpace(s, x, d) for x, d in cod], [GradedSpace(s, x, d) for x, d in dom])


def oracle_mpo(struct, entries):
    data = np.zeros(struct.numel)
    lookup = {}
    for (wl_q, wl_k), sp, s, (wr_q, wr_k), v in entries:
        lookup[(wl_q, sp, s, wr_q, wl_k, wr_k)] = v
    for p in struct.pairs:
        wl_q, sp = p.split_unc
        s, wr_q = p.fuse_unc
        for kl in range(p.dims[0]):
            for kr in range(p.dims[3]):
                v = lookup.get((wl_q, sp, s, wr_q, kl, kr))
                if v is not None:
                    data[p.offset + kl + kr * p.ld] = v
    return data


def oracle_heff_inputs(sym, D, seed=0, dtype="f64", sites=2):
    V, P, W = wl.heff_spaces(sym, D)
    legs = wl.heff_legs(V, P, W) if sites == 2 else wl.heff1_legs(V, P, W)
    st = {k: ostruct(sym, legs[k]) for k in ("x", "L", "W", "R")}
    rnd = wl.normal_complex if dtype == "c128" else wl.normal
    data = {k: rnd(seed * 16 + i, st[k].numel) for i, k in enumerate(("x", "L", "R"))}
    if sym == "U1":
        data["W"] = oracle_mpo(st["W"], wl.xxz_mpo_entries())
        if dtype == "c128":
            data["W"] = data["W"].astype(np.complex128)
    else:
        data["W"] = rnd(seed * 16 + 3, st["W"].numel)
    return st, data


def oracle_heff(sym, D, seed=0, tier="block", dtype="f64", steps=None, sites=2):
    """[(structure, data)] of every intermediate and x' computed by the oracle: the two-site chain
    (T1, T2, T3, x'; Algorithm 12) or with sites=1 the single-site chain (T1, T2, x'; Algorithm 11)."""
    st, data = oracle_heff_inputs(sym, D, seed, dtype, sites)
    specs = wl.HEFF_SPECS if sites == 2 else wl.HEFF1_SPECS
    others = ("L", "W", "W", "R") if sites == 2 else ("L", "W", "R")
    out = []
    cur_s, cur_d = st["x"], data["x"]
    for i in range(len(specs) if steps is None else steps):
        spec = specs[i]
        if i == 0:
            a, ad, b, bd = st["L"], data["L"], cur_s, cur_d
        else:
            other = others[i]
            a, ad, b, bd = cur_s, cur_d, st[other], data[other]
        cur_s, cur_d = ops.contract(a, ad, spec[0], spec[1], b, bd, spec[2], spec[3], spec[4], spec[5], tier=tier)
        out.append((cur_s, cur_d))
    return out


def rel_frobenius_per_block(struct, got, ref):
    """max over blocks of ||got - ref||_F / ||ref||_F.

    A block whose exact value is zero (an empty inner dimension, or a reference norm at the
    rounding level of the whole tensor) is measured against the norm of the whole tensor.
    """
    got, ref = np.asarray(got), np.asarray(ref)
    total = max(float(np.linalg.norm(ref)), 1e-300)
    worst = 0.0
    for c, r, k, off in struct.blocks:
        g, f = got[off:off + r * k], ref[off:off + r * k]
        nf = float(np.linalg.norm(f))
        den = nf if nf > 1e-13 * total else total
        worst = max(worst, float(np.linalg.norm(g - f) / den))
    return worst
