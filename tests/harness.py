"""Oracle-side construction of the seeded workloads and symmetry generators (tests only)."""

import math

import numpy as np

from oracle import SU2, U1, GradedSpace, TensorStructure, sym_from_name
from oracle.symmetry import ProductSymmetry
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


def oracle_heff_inputs(sym, D, seed=0, dtype="f64", sites=2, mpo=None):
    V, P, W = wl.heff_spaces(sym, D)
    legs = wl.heff_legs(V, P, W) if sites == 2 else wl.heff1_legs(V, P, W)
    st = {k: ostruct(sym, legs[k]) for k in ("x", "L", "W", "R")}
    rnd = wl.normal_complex if dtype == "c128" else wl.normal
    data = {k: rnd(seed * 16 + i, st[k].numel) for i, k in enumerate(("x", "L", "R"))}
    if sym == "U1":
        data["W"] = oracle_mpo(st["W"], wl.xxz_mpo_entries())
        if dtype == "c128":
            data["W"] = data["W"].astype(np.complex128)
    elif mpo == "heisenberg":
        data["W"] = np.array(wl.HEISENBERG_SU2_MPO, dtype=np.complex128 if dtype == "c128" else np.float64)
    else:
        data["W"] = rnd(seed * 16 + 3, st["W"].numel)
    return st, data


def oracle_heff(sym, D, seed=0, tier="block", dtype="f64", steps=None, sites=2, mpo=None):
    """[(structure, data)] of every intermediate and x' computed by the oracle: the two-site chain
    (T1, T2, T3, x'; Algorithm 12) or with sites=1 the single-site chain (T1, T2, x'; Algorithm 11)."""
    st, data = oracle_heff_inputs(sym, D, seed, dtype, sites, mpo)
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

    A block that the reference holds at exactly zero (every entry 0: a coupled sector with an
    empty inner dimension, Algorithm 8, carried through the output permute) must be exactly zero
    in `got` too; any other value there makes the result infinite.  A reference block that is not
    exactly zero but sits at the rounding level of the whole tensor (the dense tier's projection
    of such a block) is measured against the norm of the whole tensor.
    """
    got, ref = np.asarray(got), np.asarray(ref)
    total = max(float(np.linalg.norm(ref)), 1e-300)
    worst = 0.0
    for c, r, k, off in struct.blocks:
        g, f = got[off:off + r * k], ref[off:off + r * k]
        if f.size and not np.any(f):
            if np.any(g != 0):
                return float("inf")
            continue
        nf = float(np.linalg.norm(f))
        den = nf if nf > 1e-13 * total else total
        worst = max(worst, float(np.linalg.norm(g - f) / den))
    return worst


# ---------------------------------------------------------------- symmetry generators (pins)
def _multiplet_generators(sym, a):
    """[(matrix on the d_a-dim multiplet of sector a, kind)]: Lie generators ('lie') or group
    elements ('group').  SU(2): J_z, J_+, J_- in the |j, m> basis (m ascending); U(1): the charge;
    Z2: the parity; a Deligne product: each factor's generators on its tensor factor."""
    if isinstance(sym, ProductSymmetry):
        a1, a2 = sym.split(a)
        d1, d2 = sym.s1.dim(a1), sym.s2.dim(a2)
        return ([(np.kron(g, np.eye(d2)), k) for g, k in _multiplet_generators(sym.s1, a1)] +
                [(np.kron(np.eye(d1), g), k) for g, k in _multiplet_generators(sym.s2, a2)])
    if sym is SU2:
        d = a + 1
        j = a / 2
        ms = [(2 * i - a) / 2 for i in range(d)]
        jp = np.zeros((d, d))
        for i in range(d - 1):
            jp[i + 1, i] = math.sqrt(j * (j + 1) - ms[i] * (ms[i] + 1))
        return [(np.diag(ms), "lie"), (jp, "lie"), (jp.T, "lie")]
    if sym is U1:
        return [(np.array([[float(a)]]), "lie")]
    return [(np.array([[(-1.0) ** a]]), "group")]


def _leg_generators(sym, sp):
    """[(generator on the dense basis of one leg, kind)], block diagonal over its sectors."""
    per = {a: _multiplet_generators(sym, a) for a in sp.sectors}
    ngen = len(next(iter(per.values())))
    out = []
    for g in range(ngen):
        blocks = [np.kron(np.eye(n), per[a][g][0]) for a, n in sp.sectors.items()]
        out.append((_blockdiag(blocks), per[next(iter(per))][g][1]))
    return out


def _blockdiag(ms):
    n = sum(m.shape[0] for m in ms)
    out = np.zeros((n, n))
    o = 0
    for m in ms:
        k = m.shape[0]
        out[o:o + k, o:o + k] = m
        o += k
    return out


def total_generators(struct):
    """Generators of the symmetry on the tensor space V_1 (x) .. (x) W_1* (x) .. ."""
    legs = []
    for i, sp in enumerate(struct.spaces()):
        gens = _leg_generators(struct.sym, sp)
        in_domain = i >= len(struct.cod)
        dualized = sp.dual != in_domain          # acts through the contragredient
        if dualized:
            gens = [((-m.T if kind == "lie" else np.linalg.inv(m).T), kind) for m, kind in gens]
        legs.append(gens)
    dims = [sp.dim for sp in struct.spaces()]
    total = []
    for g in range(len(legs[0])):
        if legs[0][g][1] == "lie":
            acc = np.zeros((math.prod(dims),) * 2)
            for i in range(len(dims)):
                op = np.array([[1.0]])
                for k in range(len(dims)):
                    op = np.kron(op, legs[k][g][0] if k == i else np.eye(dims[k]))
                acc += op
            total.append(acc)
        else:
            op = np.array([[1.0]])
            for k in range(len(dims)):
                op = np.kron(op, legs[k][g][0])
            total.append(op - np.eye(op.shape[0]))
    return total
