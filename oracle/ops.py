"""Permute, compose and contract in the oracle (test infrastructure).

Two tiers, both in float64 (complex128 for complex data):

Dense tier ("O-dense"):
  * permute(t, (p, q)): output codomain V'_i = p_i-th space of (V_1.., W_1*..), domain
    W'_j = q_j-th space of (V_1*.., W_1..) (Algorithm 2).  For group representations tau is the
    plain swap and ev the canonical pairing, so the dense array is permuted (Sec. 2.2, the
    reduction of eq. permute_coeffs to an array permutation; Sec. 5.4, Rep G).
  * compose: C = A o B is a matrix product over the grouped domain of A (eq. tm_composition);
    domain(A) must equal codomain(B) including duality.
  * contract: Algorithm 4 (the second permute takes (p^B, q^B); the printed q^A is read as a typo).

Block tier ("O-block"), used where a dense array does not fit:
  * permute: Algorithm 10 with ``transform`` computed by the overlap route of Sec. 4.2 --
    permute the explicit tree-pair tensor E_{s,f} and project it on every canonical output tree
    pair with the same uncoupled sectors, coef = <E_{s',f'}, perm(E_{s,f})> / d_{c'}.  For abelian
    symmetries this is coefficient 1 onto exactly one output pair (Algorithm 6).
  * compose: per coupled sector c, C^c = A^c B^c, zero block when the inner dimension is empty
    (eq. abelian_compostion and the remark that follows it; Sec. 4.4 for the non-abelian case).
"""

from functools import lru_cache

import numpy as np

from .dense import _tree_cached, embed, project, reduced_array
from .structure import TensorStructure

__all__ = [
    "permute_spaces", "permute_dense", "compose_dense", "contract_dense",
    "permute_block", "compose_block", "contract_block", "contract", "permute", "check_perm",
]


def check_perm(nleg, p, q):
    p, q = tuple(int(x) for x in p), tuple(int(x) for x in q)
    if sorted(p + q) != list(range(nleg)):
        raise ValueError(f"(p, q) = ({p}, {q}) is not a permutation of {nleg} legs")
    return p, q


def permute_spaces(struct: TensorStructure, p, q):
    p, q = check_perm(struct.nleg, p, q)
    as_cod = list(struct.cod) + [w.flip() for w in struct.dom]
    as_dom = [v.flip() for v in struct.cod] + list(struct.dom)
    return [as_cod[i] for i in p], [as_dom[j] for j in q]


# --------------------------------------------------------------------------- dense tier
def permute_dense(dense, p, q):
    return np.transpose(dense, tuple(p) + tuple(q))


def compose_dense(a_dense, a_struct, b_dense, b_struct):
    if [s.key() for s in a_struct.dom] != [s.key() for s in b_struct.cod]:
        raise ValueError("domain(A) != codomain(B)")
    k = len(a_struct.dom)
    return np.tensordot(a_dense, b_dense, axes=(list(range(len(a_struct.cod), a_struct.nleg)),
                                                list(range(k))))


def contract_dense(a_struct, a_data, pa, qa, b_struct, b_data, pb, qb, pab, qab):
    """Algorithm 4 on dense embeddings; returns (C structure, C flat reduced data)."""
    at_cod, at_dom = permute_spaces(a_struct, pa, qa)
    bt_cod, bt_dom = permute_spaces(b_struct, pb, qb)
    at = TensorStructure(at_cod, at_dom)
    bt = TensorStructure(bt_cod, bt_dom)
    ad = permute_dense(embed(a_struct, a_data), pa, qa)
    bd = permute_dense(embed(b_struct, b_data), pb, qb)
    cd = compose_dense(ad, at, bd, bt)
    ct = TensorStructure(at_cod, bt_dom)
    c_cod, c_dom = permute_spaces(ct, pab, qab)
    cs = TensorStructure(c_cod, c_dom)
    return cs, project(cs, permute_dense(cd, pab, qab))


# --------------------------------------------------------------------------- block tier
# Magnitude below which an overlap is rounding residue of an exact zero.  Genuine recoupling
# coefficients of the labels used here (j <= 10) are many orders of magnitude larger.
OVERLAP_ZERO = 1e-12


@lru_cache(maxsize=None)
def _e_tensor(sym, su, si, c, fu, fi, cod_duals, dom_duals):
    ys = _tree_cached(sym.name, sym, su, si, c, cod_duals)
    yf = _tree_cached(sym.name, sym, fu, fi, c, dom_duals)
    e = np.tensordot(ys, yf, axes=([ys.ndim - 1], [yf.ndim - 1]))
    e.setflags(write=False)
    return e


@lru_cache(maxsize=None)
def _overlap_coeffs(sym, in_labels, in_duals, out_cands, out_duals, perm):
    """coef(out) = <E_out, perm(E_in)> / d_{c_out} for every candidate output pair."""
    e_in = np.transpose(_e_tensor(sym, *in_labels, *in_duals), perm)
    res = []
    for lab in out_cands:
        e_out = _e_tensor(sym, *lab, *out_duals)
        coef = float(np.sum(e_out * e_in)) / sym.dim(lab[2])
        # Canonical tree pairs are orthonormal (eq. fusiontreeorthogonality): an overlap that is
        # zero in exact arithmetic shows up only as rounding residue of the CG sums.
        if abs(coef) > OVERLAP_ZERO:
            res.append((lab, coef))
    return tuple(res)


def _pair_labels(pr):
    return (pr.split_unc, pr.split_inner, pr.coupled, pr.fuse_unc, pr.fuse_inner)


def permute_transform(struct: TensorStructure, p, q, out_struct=None):
    """Sparse transform {input pair labels: [(output pair labels, coef), ...]} (overlap route)."""
    p, q = check_perm(struct.nleg, p, q)
    if out_struct is None:
        out_struct = TensorStructure(*permute_spaces(struct, p, q))
    perm = p + q
    out_spaces = out_struct.spaces()
    groups = {}
    for pr in out_struct.pairs:
        und = tuple(sp.underlying(l) for sp, l in zip(out_spaces, pr.split_unc + pr.fuse_unc))
        groups.setdefault(und, []).append(_pair_labels(pr))
    in_spaces = struct.spaces()
    in_duals = (tuple(s.dual for s in struct.cod), tuple(s.dual for s in struct.dom))
    out_duals = (tuple(s.dual for s in out_struct.cod), tuple(s.dual for s in out_struct.dom))
    result = {}
    for pr in struct.pairs:
        und_in = tuple(sp.underlying(l) for sp, l in zip(in_spaces, pr.split_unc + pr.fuse_unc))
        und_out = tuple(und_in[i] for i in perm)
        cands = tuple(groups.get(und_out, ()))
        if struct.sym.abelian:
            # Algorithm 6: the unique output channel with these sectors, coefficient 1
            if len(cands) != 1:
                raise AssertionError("abelian permute must map a channel onto exactly one channel")
            result[pr.labels] = [(cands[0], 1.0)]
            continue
        result[pr.labels] = list(_overlap_coeffs(struct.sym, _pair_labels(pr), in_duals, cands,
                                                 out_duals, perm))
    return out_struct, result


def permute_block(struct: TensorStructure, data, p, q):
    p, q = check_perm(struct.nleg, p, q)
    if p + q == tuple(range(struct.nleg)) and len(p) == len(struct.cod):
        return struct, np.array(data, copy=True)  # permute with the identity (p, q) is the identity
    out_struct, tr = permute_transform(struct, p, q)
    data = np.asarray(data)
    out = np.zeros(out_struct.numel, dtype=data.dtype)
    idx = out_struct.pair_index()
    perm = p + q
    for pr in struct.pairs:
        x = np.transpose(reduced_array(struct, data, pr), perm)
        for lab, coef in tr[pr.labels]:
            y = idx[lab]
            r = int(np.prod(y.dims[:len(out_struct.cod)], dtype=np.int64))
            c = int(np.prod(y.dims[len(out_struct.cod):], dtype=np.int64))
            sub = (coef * x).reshape((r, c), order="F")
            it = out.itemsize
            view = np.lib.stride_tricks.as_strided(out[y.offset:], shape=(r, c),
                                                   strides=(it, y.ld * it))
            view += sub
    return out_struct, out


def compose_block(a_struct, a_data, b_struct, b_data):
    """C~ = A~ o B~ block by block; blocks with an empty inner dimension are zero."""
    if [s.key() for s in a_struct.dom] != [s.key() for s in b_struct.cod]:
        raise ValueError("domain(A) != codomain(B)")
    cs = TensorStructure(a_struct.cod, b_struct.dom)
    a_data, b_data = np.asarray(a_data), np.asarray(b_data)
    out = np.zeros(cs.numel, dtype=np.result_type(a_data, b_data))
    ab, bb = a_struct.block_dict(), b_struct.block_dict()
    for c, rows, cols, off in cs.blocks:
        if c in ab and c in bb:
            ar, ak, aoff = ab[c]
            bk, bc, boff = bb[c]
            assert ar == rows and bc == cols and ak == bk
            am = a_data[aoff:aoff + ar * ak].reshape(ak, ar).T
            bm = b_data[boff:boff + bk * bc].reshape(bc, bk).T
            out[off:off + rows * cols] = (am @ bm).T.reshape(-1)
        # else: K_c = 0 -> zero block (already zero)
    return cs, out


def permute(struct, data, p, q, tier="block"):
    if tier == "dense":
        cod, dom = permute_spaces(struct, p, q)
        cs = TensorStructure(cod, dom)
        return cs, project(cs, permute_dense(embed(struct, data), p, q))
    return permute_block(struct, data, p, q)


def contract_block(a_struct, a_data, pa, qa, b_struct, b_data, pb, qb, pab, qab):
    at, ad = permute_block(a_struct, a_data, pa, qa)
    bt, bd = permute_block(b_struct, b_data, pb, qb)
    ct, cd = compose_block(at, ad, bt, bd)
    return permute_block(ct, cd, pab, qab)


def contract(a_struct, a_data, pa, qa, b_struct, b_data, pb, qb, pab, qab, tier="dense"):
    f = contract_dense if tier == "dense" else contract_block
    return f(a_struct, a_data, pa, qa, b_struct, b_data, pb, qb, pab, qab)


def adjoint_dense(struct: TensorStructure, data):
    """t^dagger : dom <- cod of t : cod <- dom (the adjoint of the paper's Sec. 2): the dense array
    conjugated with codomain and domain axes exchanged, projected onto the canonical trees of the
    exchanged spaces."""
    dense = embed(struct, data)
    n1 = len(struct.cod)
    perm = list(range(n1, struct.nleg)) + list(range(n1))
    adj = TensorStructure(struct.dom, struct.cod)
    return adj, project(adj, np.conj(dense).transpose(perm))


def adjoint_block(struct: TensorStructure, data):
    """Block tier of the adjoint: with orthonormal canonical trees the splitting and fusion trees
    exchange roles, so block c of t^dagger is the conjugate transpose of block c of t."""
    adj = TensorStructure(struct.dom, struct.cod)
    data = np.asarray(data)
    out = np.zeros(adj.numel, dtype=data.dtype)
    src = struct.block_dict()
    for c, rows, cols, off in adj.blocks:
        r0, c0, o0 = src[c]
        assert r0 == cols and c0 == rows
        blk = data[o0:o0 + r0 * c0].reshape(c0, r0).T          # rows x cols of t, column-major storage
        out[off:off + rows * cols] = np.conj(blk).reshape(-1)   # its transpose, column-major
    return adj, out


def adjoint(struct, data, tier="block"):
    return adjoint_dense(struct, data) if tier == "dense" else adjoint_block(struct, data)


def svd_block(struct: TensorStructure, data):
    """Block SVD (Algorithm 9): per coupled sector c, t_c = U_c diag(s_c) V_c^dagger with
    r_c = min(rows_c, cols_c) values, descending.  Returns [(c, U_c, s_c, Vh_c)] in sector order
    (dense numpy matrices; sectors with an empty block are skipped)."""
    data = np.asarray(data)
    out = []
    for c, rows, cols, off in struct.blocks:
        if min(rows, cols) == 0:
            continue
        blk = data[off:off + rows * cols].reshape(cols, rows).T
        u, s, vh = np.linalg.svd(blk, full_matrices=False)
        out.append((c, u, s, vh))
    return out


def truncation_keep(struct: TensorStructure, svals, dmax):
    """Keep counts per block for a truncation to at most dmax states (the truncated SVD after the
    two-site step of Algorithm 12; the paper fixes no rule, this is the reading used here).  Every
    value of sector c stands for d_c states (an SU(2) multiplet), so the dense spectrum of t is
    the block values each repeated d_c times.  Values are taken in descending order over all
    sectors (ties: ascending sector), whole multiplets only, and the walk stops at the first
    multiplet that no longer fits: the kept states are a prefix of the dense spectrum cut at a
    multiplet boundary.  Returns (keep per block, relative discarded weight
    sqrt(sum_discarded d_c s^2 / sum_all d_c s^2))."""
    entries = []
    for b, (c, s) in enumerate(svals):
        for v in s:
            entries.append((-float(v), c, b))
    entries.sort()
    keep = [0] * len(svals)
    used, kept_w, total_w = 0, 0.0, 0.0
    full = False
    for negv, c, b in entries:
        d = struct.sym.dim(c)
        total_w += d * negv * negv
        if not full and used + d <= dmax:
            keep[b] += 1
            used += d
            kept_w += d * negv * negv
        else:
            full = True
    err = np.sqrt(max(total_w - kept_w, 0.0) / total_w) if total_w > 0 else 0.0
    return keep, err
