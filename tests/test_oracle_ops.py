"""Pins of the oracle's permute / compose / contract (dense and block tiers)."""

import itertools

import numpy as np
import pytest

from golden_io import matrix
from oracle.symmetry import U1xSU2, Z2xU1
from oracle import SU2, U1, Z2, GradedSpace, TensorStructure
from oracle import ops
from oracle.dense import embed, project

# trees of the SU(2) worked example in 2j notation: (uncoupled labels, coupled sector)
_FIG_TREES = {1: ((0, 0), 0), 2: ((1, 1), 0), 3: ((0, 1), 1), 4: ((1, 0), 1), 5: ((1, 1), 2)}
_CHANNELS = [(1, 1), (2, 1), (1, 2), (2, 2), (3, 3), (4, 3), (3, 4), (4, 4), (5, 5)]


def _channel_labels(i, j):
    (su, c), (fu, c2) = _FIG_TREES[i], _FIG_TREES[j]
    assert c == c2
    return (su, (), c, fu, ())


@pytest.mark.parametrize("fixture,p,q", [
    ("su2_transpose_matrix.txt", (1, 3), (0, 2)),   # clockwise cycle: s : V* (x) V -> V (x) V*
    ("su2_permute_matrix.txt", (1, 0), (3, 2)),     # swap both codomain and domain indices
])
def test_su2_worked_example_matrices(fixture, p, q):
    """The printed transition matrices M (rows: transformed trees, columns: canonical trees)
    satisfy s = M^T t on the nine channels, with the figure's trees (3) = (0, 1/2) and
    (4) = (1/2, 0) (the numbering exists only in the figure; Sec. 4.3)."""
    v = GradedSpace(SU2, {0: 1, 1: 1})
    t = TensorStructure([v, v], [v, v])
    out, tr = ops.permute_transform(t, p, q)
    m = np.array(matrix(fixture))
    got = np.zeros((9, 9))
    idx = {_channel_labels(*ch): k for k, ch in enumerate(_CHANNELS)}
    for src, lst in tr.items():
        for dst, coef in lst:
            got[idx[dst], idx[src]] += coef
    assert np.allclose(got, m.T, atol=1e-14)
    if p == (1, 3):
        assert [s.dual for s in out.cod] == [False, True] and [s.dual for s in out.dom] == [True, False]


def _rand_struct(sym, cod, dom):
    return TensorStructure([GradedSpace(sym, s, d) for s, d in cod], [GradedSpace(sym, s, d) for s, d in dom])


SMALL = [
    (SU2, [({0: 1, 1: 2, 2: 1}, False), ({1: 1}, False)], [({0: 1, 1: 1, 2: 2}, True), ({1: 1}, True)]),
    (SU2, [({1: 2, 3: 1}, True), ({0: 1, 2: 1}, False)], [({1: 1, 3: 2}, False)]),
    (U1, [({-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}, False), ({-1: 1, 1: 1}, False)],
     [({-2: 1, -1: 2, 0: 3, 1: 2, 2: 1}, True), ({-1: 1, 1: 1}, True)]),
    (Z2, [({0: 2, 1: 3}, False), ({0: 1, 1: 2}, True)], [({0: 2, 1: 1}, False)]),
    (U1xSU2, [({U1xSU2.pair(0, 0): 1, U1xSU2.pair(1, 1): 2}, False), ({U1xSU2.pair(-1, 1): 1}, True)],
     [({U1xSU2.pair(0, 0): 1, U1xSU2.pair(0, 2): 1, U1xSU2.pair(2, 0): 1, U1xSU2.pair(1, 1): 1}, True),
      ({U1xSU2.pair(0, 1): 1}, False)]),
    (Z2xU1, [({Z2xU1.pair(0, 0): 2, Z2xU1.pair(1, 1): 1}, False), ({Z2xU1.pair(1, -1): 1}, True)],
     [({Z2xU1.pair(0, 0): 1, Z2xU1.pair(1, 0): 2, Z2xU1.pair(0, 2): 1}, False)]),
]


@pytest.mark.parametrize("case", range(len(SMALL)))
def test_block_permute_equals_dense_permute(case):
    st = _rand_struct(*SMALL[case])
    x = np.random.default_rng(case).standard_normal(st.numel)
    n = st.nleg
    rng = np.random.default_rng(100 + case)
    for _ in range(6):
        perm = list(rng.permutation(n))
        k = int(rng.integers(0, n + 1))
        p, q = tuple(perm[:k]), tuple(perm[k:])
        s1, y1 = ops.permute(st, x, p, q, tier="dense")
        s2, y2 = ops.permute(st, x, p, q, tier="block")
        assert s1.blocks == s2.blocks
        assert np.allclose(y1, y2, atol=1e-13)


@pytest.mark.parametrize("case", range(len(SMALL)))
def test_permute_coherence_and_inverse(case):
    """permute(permute(t, s1), s2) = permute(t, s2 o s1); the inverse restores t (Sec. 2.2
    coherence; Sec. 5.2, MacLane)."""
    st = _rand_struct(*SMALL[case])
    x = np.random.default_rng(7 + case).standard_normal(st.numel)
    n = st.nleg
    rng = np.random.default_rng(200 + case)
    for _ in range(4):
        s1, s2 = list(rng.permutation(n)), list(rng.permutation(n))
        k1, k2 = int(rng.integers(0, n + 1)), int(rng.integers(0, n + 1))
        a, ya = ops.permute_block(st, x, tuple(s1[:k1]), tuple(s1[k1:]))
        b, yb = ops.permute_block(a, ya, tuple(s2[:k2]), tuple(s2[k2:]))
        comp = [s1[i] for i in s2]
        c, yc = ops.permute_block(st, x, tuple(comp[:k2]), tuple(comp[k2:]))
        assert b.blocks == c.blocks and np.allclose(yb, yc, atol=1e-13)
        inv = list(np.argsort(s1))
        r, yr = ops.permute_block(a, ya, tuple(inv[:len(st.cod)]), tuple(inv[len(st.cod):]))
        assert r.blocks == st.blocks and np.allclose(yr, x, atol=1e-13)


def _spec_c0():
    v = GradedSpace(U1, {-2: 1, -1: 2, 0: 3, 1: 2, 2: 1})
    a = TensorStructure([v, v], [v, v])
    b = TensorStructure([v, v.flip()], [v, v])
    return a, b


def test_c0_contraction_dense_block_and_bruteforce():
    """C[a,b,e,f] = sum_{c,d} A[a,c,b,d] B[d,c,e,f]: dense tier, block tier and explicit loops."""
    a, b = _spec_c0()
    rng = np.random.default_rng(0)
    xa, xb = rng.standard_normal(a.numel), rng.standard_normal(b.numel)
    args = (a, xa, (0, 2), (3, 1), b, xb, (0, 1), (2, 3), (0, 1), (2, 3))
    cs1, y1 = ops.contract(*args, tier="dense")
    cs2, y2 = ops.contract(*args, tier="block")
    assert cs1.blocks == cs2.blocks
    assert np.allclose(y1, y2, atol=1e-12)
    # explicit loops on the dense arrays
    da, db = embed(a, xa), embed(b, xb)
    n = da.shape[0]
    dc = np.zeros((n, n, n, n))
    for i, j, k, l in itertools.product(range(n), repeat=4):
        s = 0.0
        for c, d in itertools.product(range(n), repeat=2):
            s += da[i, c, j, d] * db[d, c, k, l]
        dc[i, j, k, l] = s
    assert np.allclose(embed(cs1, y1), dc, atol=1e-12)
    # square per-charge GEMMs of the permuted A (block work 34,362 flops)
    at = TensorStructure(*ops.permute_spaces(a, (0, 2), (3, 1)))
    assert [(c, r, k) for c, r, k, _ in at.blocks] == [
        (-4, 1, 1), (-3, 4, 4), (-2, 10, 10), (-1, 16, 16), (0, 19, 19), (1, 16, 16), (2, 10, 10),
        (3, 4, 4), (4, 1, 1)]
    assert sum(2 * r * k * k for _, r, k, _ in at.blocks) == 34362


def test_su2_contraction_dense_vs_block():
    v = GradedSpace(SU2, {0: 2, 1: 2, 2: 1})
    w = GradedSpace(SU2, {0: 2, 2: 1})
    p = GradedSpace(SU2, {1: 1})
    # L : V <- V (x) W ; x : V (x) P <- V (x) P*
    L = TensorStructure([v], [v, w])
    X = TensorStructure([v, p], [v, p.flip()])
    rng = np.random.default_rng(3)
    xl, xx = rng.standard_normal(L.numel), rng.standard_normal(X.numel)
    # contract L's domain V (leg 1) with x's codomain V (leg 0)
    args = (L, xl, (0, 2), (1,), X, xx, (0,), (1, 2, 3), (0, 1, 2, 3, 4), ())
    cs1, y1 = ops.contract(*args, tier="dense")
    cs2, y2 = ops.contract(*args, tier="block")
    assert cs1.blocks == cs2.blocks
    assert np.allclose(y1, y2, atol=1e-12)


def test_empty_inner_dimension_gives_zero_block():
    """A coupled sector present in codomain(A) and domain(B) but not in the contracted space
    gives a zero block (remark after eq. abelian_compostion)."""
    va = GradedSpace(U1, {0: 2, 1: 1})
    k = GradedSpace(U1, {0: 3})
    a = TensorStructure([va], [k])          # only c = 0 survives ...
    b = TensorStructure([k], [va])
    # ... so build C~ : va <- va directly from compose
    xa = np.ones(a.numel)
    xb = np.ones(b.numel)
    cs, y = ops.compose_block(a, xa, b, xb)
    bd = cs.block_dict()
    assert 1 in bd
    r, c, off = bd[1]
    assert np.all(y[off:off + r * c] == 0.0)
    assert np.all(y[bd[0][2]: bd[0][2] + 4] == 3.0)


def test_embed_project_roundtrip_complex():
    st = _rand_struct(*SMALL[0])
    rng = np.random.default_rng(11)
    x = rng.standard_normal(st.numel) + 1j * rng.standard_normal(st.numel)
    assert np.allclose(project(st, embed(st, x)), x, atol=1e-14)


def _su2_tensor(seed, cod, dom, cplx=False):
    st = TensorStructure([GradedSpace(SU2, *x) for x in cod], [GradedSpace(SU2, *x) for x in dom])
    rng = np.random.default_rng(seed)
    d = rng.normal(size=st.numel)
    if cplx:
        d = d + 1j * rng.normal(size=st.numel)
    return st, d


def test_adjoint_dense_equals_block_and_is_an_involution():
    """The dense definition (conjugate, exchange codomain and domain, project) and the block
    form agree; applying the adjoint twice gives back t; the Frobenius norm is kept."""
    st, d = _su2_tensor(3, [({0: 2, 1: 1}, False), ({1: 2}, True)], [({0: 1, 1: 2, 2: 1}, False)], cplx=True)
    s1, a1 = ops.adjoint(st, d, tier="dense")
    s2, a2 = ops.adjoint(st, d, tier="block")
    assert s1.blocks == s2.blocks
    assert np.allclose(a1, a2, atol=1e-13)
    s3, a3 = ops.adjoint(s2, a2, tier="dense")
    assert s3.blocks == st.blocks and np.allclose(a3, d, atol=1e-13)
    assert np.isclose(np.linalg.norm(a2), np.linalg.norm(d))


def test_adjoint_reverses_composition():
    """(A o B)^dagger = B^dagger o A^dagger, on SU(2) maps with dual legs (dense tier throughout)."""
    V = ({0: 1, 1: 2}, False)
    W = ({1: 1, 2: 1}, True)
    U = ({0: 2, 2: 1}, False)
    sa, da = _su2_tensor(4, [V, W], [U, V], cplx=True)       # A : V W <- U V
    sb, db = _su2_tensor(5, [U, V], [W], cplx=True)          # B : U V <- W
    sab, dab = ops.contract(sa, da, (0, 1), (2, 3), sb, db, (0, 1), (2,), (0, 1), (2,), tier="dense")
    s_l, d_l = ops.adjoint(sab, dab, tier="dense")           # (A o B)^dagger : W <- V W
    sbd, dbd = ops.adjoint(sb, db, tier="dense")             # B^dagger : W <- U V
    sad, dad = ops.adjoint(sa, da, tier="dense")             # A^dagger : U V <- V W
    s_r, d_r = ops.contract(sbd, dbd, (0,), (1, 2), sad, dad, (0, 1), (2, 3), (0,), (1, 2), tier="dense")
    assert s_l.blocks == s_r.blocks
    assert np.allclose(d_l, d_r, atol=1e-12)


def test_block_svd_matches_dense_spectrum_and_reconstructs():
    """The block SVD of an SU(2) tensor map: every block singular value appears d_c times among
    the singular values of the dense embedded matrix (codomain x domain), the blocks reconstruct
    t, and the truncation rule keeps whole multiplets."""
    st, d = _su2_tensor(9, [({0: 2, 1: 2}, False), ({1: 1}, False)], [({0: 1, 1: 2, 2: 1}, False), ({1: 1}, True)])
    blocks = ops.svd_block(st, d)
    n1 = len(st.cod)
    dense = embed(st, d)
    rows = int(np.prod(dense.shape[:n1]))
    sv_dense = np.sort(np.linalg.svd(dense.reshape(rows, -1), compute_uv=False))[::-1]
    sv_blocks = np.sort(np.concatenate([np.repeat(s, st.sym.dim(c)) for c, _, s, _ in blocks]))[::-1]
    nz = sv_dense[sv_dense > 1e-10]
    assert np.allclose(nz, sv_blocks[:len(nz)], rtol=1e-12)
    assert np.all(sv_blocks[len(nz):] < 1e-10)
    bd = st.block_dict()
    for c, u, s, vh in blocks:
        r, k, off = bd[c]
        assert np.allclose((u * s) @ vh, d[off:off + r * k].reshape(k, r).T, atol=1e-12)
    keep, err = ops.truncation_keep(st, [(c, s) for c, _, s, _ in blocks], dmax=7)
    assert sum(st.sym.dim(c) * k for (c, _, _, _), k in zip(blocks, keep)) <= 7
    assert 0 < err < 1
    # the kept values are the largest: any discarded value of a sector is below every kept one of it
    for (c, _, s, _), k in zip(blocks, keep):
        assert np.all(s[:k][:, None] >= s[k:][None, :])


def _dense_spectrum(st, d):
    """Singular values of the dense embedded matrix (codomain x domain), descending."""
    dense = embed(st, d)
    rows = int(np.prod(dense.shape[:len(st.cod)]))
    return np.sort(np.linalg.svd(dense.reshape(rows, -1), compute_uv=False))[::-1]


def _check_truncation_against_dense(st, d, dmax, keep_fn=None):
    """The truncation rule checked against the dense SVD of t, which knows nothing of sectors:
    the kept states are the largest dense singular values (a prefix of the dense spectrum), the
    cut falls on a multiplet boundary (the next dense value's multiplet would not fit), and the
    error is the discarded share of the dense spectrum's weight."""
    keep_fn = keep_fn or ops.truncation_keep
    blocks = ops.svd_block(st, d)
    keep, err = keep_fn(st, [(c, s) for c, _, s, _ in blocks], dmax)
    dense = _dense_spectrum(st, d)
    kept = np.sort(np.concatenate([np.repeat(s[:k], st.sym.dim(c)) for (c, _, s, _), k in zip(blocks, keep)]))[::-1]
    n = len(kept)
    assert n <= dmax
    assert np.allclose(kept, dense[:n], rtol=1e-12, atol=1e-13 * dense[0])
    if n < len(dense):
        nxt = dense[n]
        mult = int(np.sum(np.abs(dense - nxt) <= 1e-9 * dense[0]))
        assert n + mult > dmax, "a whole multiplet below the cut would still have fitted"
    want = np.sqrt(np.sum(dense[n:] ** 2) / np.sum(dense ** 2))
    assert abs(err - want) <= 1e-12
    return keep, err


@pytest.mark.parametrize("dmax", list(range(1, 26)))
def test_truncation_keep_is_a_prefix_of_the_dense_spectrum(dmax):
    """SU(2): multiplets of dimension 1, 2 and 3 compete across sectors; every bond dimension from
    1 to beyond the full rank is checked against the dense SVD."""
    st, d = _su2_tensor(11, [({0: 2, 1: 2, 2: 1}, False), ({1: 1}, False)],
                        [({0: 1, 1: 2, 2: 1}, False), ({1: 1}, True)])
    _check_truncation_against_dense(st, d, dmax)


def test_truncation_keep_u1_takes_the_top_values():
    """U(1): every multiplet has one state, so keeping dmax states is the top dmax dense values."""
    v = GradedSpace(U1, {-1: 2, 0: 3, 1: 2})
    st = TensorStructure([v, v], [v])
    d = np.random.default_rng(3).standard_normal(st.numel)
    for dmax in (1, 3, 5, 8, 13):
        keep, _ = _check_truncation_against_dense(st, d, dmax)
        assert sum(keep) == min(dmax, len(_dense_spectrum(st, d)))


def test_truncation_pin_rejects_planted_mistakes():
    """The dense check fails a rule that picks per sector without comparing across sectors, and a
    rule whose error leaves out the d_c weight."""
    st, d = _su2_tensor(11, [({0: 2, 1: 2, 2: 1}, False), ({1: 1}, False)],
                        [({0: 1, 1: 2, 2: 1}, False), ({1: 1}, True)])

    def per_sector(struct, svals, dmax):  # the same share of each sector, no comparison across them
        total = sum(len(s) * struct.sym.dim(c) for c, s in svals)
        keep = [int(len(s) * min(1.0, dmax / total)) for c, s in svals]
        _, err = ops.truncation_keep(struct, svals, dmax)
        return keep, err

    def unweighted(struct, svals, dmax):  # the right keep counts, error without d_c
        keep, _ = ops.truncation_keep(struct, svals, dmax)
        tot = sum(float(np.sum(s ** 2)) for _, s in svals)
        kept = sum(float(np.sum(s[:k] ** 2)) for (_, s), k in zip(svals, keep))
        return keep, np.sqrt(max(tot - kept, 0.0) / tot)

    for bad in (per_sector, unweighted):
        failed = 0
        for dmax in range(2, 20):
            try:
                _check_truncation_against_dense(st, d, dmax, keep_fn=bad)
            except AssertionError:
                failed += 1
        assert failed > 0, bad.__name__


def test_product_symmetry_contraction_dense_vs_block_and_bruteforce():
    """U(1) x SU(2) (charge x spin, Sec. 5.2 product sectors): the block contraction (overlap-route
    recoupling of Kronecker-product splitting tensors) equals the dense contraction, and the dense
    result is a plain einsum of the dense operands."""
    P = U1xSU2.pair
    v = GradedSpace(U1xSU2, {P(-1, 1): 1, P(0, 0): 2, P(0, 2): 1, P(1, 1): 1})
    p = GradedSpace(U1xSU2, {P(1, 1): 1})
    w = GradedSpace(U1xSU2, {P(0, 0): 1, P(0, 2): 1})
    L = TensorStructure([v], [v, w])
    X = TensorStructure([v, p], [v, p.flip()])
    rng = np.random.default_rng(5)
    xl, xx = rng.standard_normal(L.numel), rng.standard_normal(X.numel)
    args = (L, xl, (0, 2), (1,), X, xx, (0,), (1, 2, 3), (0, 1, 2, 3, 4), ())
    cs1, y1 = ops.contract(*args, tier="dense")
    cs2, y2 = ops.contract(*args, tier="block")
    assert cs1.blocks == cs2.blocks
    assert np.allclose(y1, y2, atol=1e-12)
    dl, dx = embed(L, xl), embed(X, xx)
    ref = np.einsum("abw,bpcq->awpcq", dl, dx)  # contract L's domain V with x's codomain V
    assert np.allclose(embed(cs1, y1), ref, atol=1e-12)


def test_product_splitting_tensors_orthonormal_complete():
    """Kronecker-product splitting tensors of U(1) x SU(2) and Z2 x U(1) form an orthonormal basis
    of a (x) b (d_a d_b = sum_c N_ab^c d_c), channel by channel."""
    for sym, labels in ((U1xSU2, [U1xSU2.pair(q, t) for q in (-1, 0, 2) for t in (0, 1, 2, 3)]),
                        (Z2xU1, [Z2xU1.pair(z, q) for z in (0, 1) for q in (-2, 0, 1)])):
        for a, b in itertools.product(labels, labels):
            cs = sym.fuse(a, b)
            assert sym.dim(a) * sym.dim(b) == sum(sym.dim(c) for c in cs)
            u = np.concatenate([sym.cg_tensor(a, b, c).reshape(sym.dim(a) * sym.dim(b), sym.dim(c)) for c in cs],
                               axis=1)
            assert np.allclose(u.T @ u, np.eye(u.shape[0]), atol=1e-14)
