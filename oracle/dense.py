"""Dense embedding and projection of symmetric tensor maps (oracle; test infrastructure).

A tensor map is stored as reduced arrays t^{s,f} per fusion-tree pair.  Its dense form over the
full basis |a, k, m> of every leg is (Wigner-Eckart theorem and canonical expansion, Sec. 4.1)

    T = sum_{(s,f)} sum_mu  Y_s[m_1..; mu] t^{s,f}[k_1..; l_1..] Y_f[n_1..; mu]

where Y_s is the canonical splitting tree built from explicit splitting tensors (CG
coefficients for SU(2)) left to right (eq. canonicalsplitting) and, on every leg that is a
dual space, contracted with Z_a (Sec. 4.2: Z on the uncoupled legs of dual spaces).  All
representation data is real, so the fusion tree is the transpose of the splitting tree.

Projection back uses orthonormality of canonical trees (eq. fusiontreeorthogonality):
t^{s,f} = <E_{s,f}, T> / d_c with E_{s,f} = sum_mu Y_s Y_f.
"""

from functools import lru_cache

import numpy as np

from .structure import TensorStructure

__all__ = ["tree_tensor", "pair_tensor", "embed", "project", "reduced_array", "set_reduced_array"]


def _tree_core(sym, unc, inner, c):
    """Canonical splitting tree as array [m_1, ..., m_N, M] (no Z)."""
    n = len(unc)
    if n == 0:
        return np.ones((1,))
    x = np.eye(sym.dim(unc[0]))  # [m_1, u]
    u = unc[0]
    for k in range(1, n):
        v = inner[k - 1] if k < n - 1 else c
        x = np.tensordot(x, sym.cg_tensor(u, unc[k], v), axes=([x.ndim - 1], [0]))
        u = v
    return x


def tree_tensor(sym, unc, inner, c, spaces):
    """Y_s: canonical tree with Z_a applied on the legs whose space is dual.

    Axis i of the result indexes the dense inner basis m of leg i (for a dual leg: the dual
    basis <a m| of the underlying sector a), the last axis the coupled sector.
    """
    return _tree_cached(sym.name, sym, tuple(unc), tuple(inner), c,
                        tuple(sp.dual for sp in spaces))


@lru_cache(maxsize=None)
def _tree_cached(_name, sym, unc, inner, c, duals):
    x = _tree_core(sym, unc, inner, c)
    for i, d in enumerate(duals):
        if d:
            z = sym.zmat(sym.dual(unc[i]))  # Z_a : (V^a)* -> V^abar, a = underlying sector
            x = np.moveaxis(np.tensordot(x, z, axes=([i], [0])), -1, i)
    x.setflags(write=False)
    return x


def pair_tensor(struct: TensorStructure, p):
    """E_{s,f}[m..; n..] = sum_mu Y_s[m..; mu] Y_f[n..; mu]."""
    ys = tree_tensor(struct.sym, p.split_unc, p.split_inner, p.coupled, struct.cod)
    yf = tree_tensor(struct.sym, p.fuse_unc, p.fuse_inner, p.coupled, struct.dom)
    return np.tensordot(ys, yf, axes=([ys.ndim - 1], [yf.ndim - 1]))


def reduced_array(struct: TensorStructure, data, p):
    """t^{s,f} as an N-d array (codomain legs then domain legs), copied out of flat storage."""
    n1 = len(struct.cod)
    rdims, cdims = p.dims[:n1], p.dims[n1:]
    r, c = int(np.prod(rdims, dtype=np.int64)), int(np.prod(cdims, dtype=np.int64))
    data = np.asarray(data)
    it = data.itemsize
    sub = np.lib.stride_tricks.as_strided(data[p.offset:], shape=(r, c), strides=(it, p.ld * it),
                                          writeable=False)
    return np.array(sub).reshape(tuple(rdims) + tuple(cdims), order="F")


def set_reduced_array(struct: TensorStructure, data, p, arr):
    rows = p.ld
    n1 = len(struct.cod)
    rdims, cdims = p.dims[:n1], p.dims[n1:]
    r, c = int(np.prod(rdims, dtype=np.int64)), int(np.prod(cdims, dtype=np.int64))
    sub = np.asarray(arr).reshape((r, c), order="F")
    for j in range(c):
        start = p.offset + j * rows
        data[start:start + r] = sub[:, j]


def _leg_slices(struct, p):
    sls, nd = [], []
    for sp, lab, n in zip(struct.spaces(), p.split_unc + p.fuse_unc, p.dims):
        a = sp.underlying(lab)
        d = struct.sym.dim(a)
        off = sp.dense_offsets[a]
        sls.append(slice(off, off + n * d))
        nd.append((n, d))
    return sls, nd


def embed(struct: TensorStructure, data):
    """Dense array of shape (dim(V_1), ..., dim(W_1), ...) from flat reduced data."""
    data = np.asarray(data)
    dense = np.zeros([sp.dim for sp in struct.spaces()], dtype=data.dtype)
    nleg = struct.nleg
    for p in struct.pairs:
        t = reduced_array(struct, data, p)              # [k_1 .. k_N]
        e = pair_tensor(struct, p)                       # [m_1 .. m_N]
        sls, nd = _leg_slices(struct, p)
        # outer product arranged as (k_1, m_1, k_2, m_2, ...)
        contrib = np.multiply.outer(t, e)                # [k.., m..]
        order = [x for i in range(nleg) for x in (i, nleg + i)]
        contrib = contrib.transpose(order).reshape([n * d for n, d in nd])
        dense[tuple(sls)] += contrib
    return dense


def project(struct: TensorStructure, dense):
    """Flat reduced data from a dense array (orthogonal projection onto the canonical basis)."""
    dense = np.asarray(dense)
    out = np.zeros(struct.numel, dtype=dense.dtype)
    nleg = struct.nleg
    for p in struct.pairs:
        e = pair_tensor(struct, p)
        sls, nd = _leg_slices(struct, p)
        view = dense[tuple(sls)].reshape([x for n, d in nd for x in (n, d)])
        # contract the m axes (odd positions) with e
        t = np.tensordot(view, e, axes=(list(range(1, 2 * nleg, 2)), list(range(nleg))))
        t = t / struct.sym.dim(p.coupled)
        set_reduced_array(struct, out, p, t)
    return out
