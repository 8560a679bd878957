"""Graded spaces and the canonical fusion-tree block layout of a TensorMap (oracle).

Test infrastructure (see the package header).  The layout written out here is the fixed
storage order that the paper leaves "arbitrary but fixed" (Sec. 3.2, eq. abeliangrouping and
the remark after it; Sec. 4.1, canonical left-to-right trees and the block embedding):

* a graded space is a list of (sector, multiplicity) pairs plus a dual flag (Sec. 5.2); a leg
  of a dual space carries, in every tree, the dual sector "as if it were a normal space"
  (Sec. 3.2, transpositions);
* sectors are ordered by value: U(1) ascending integer, Z2 0 < 1, SU(2) ascending 2j;
* a canonical splitting tree on legs (a_1..a_N) is ((a_1 a_2)_{u_2} a_3)_{u_3} ... a_N)_c
  (eq. canonicalsplitting); trees are ordered colexicographically (first leg fastest, like
  eq. linearindex) by the uncoupled labels (a_1, ..., a_N) and then colexicographically by the
  inner labels (u_2, ..., u_{N-1}) -- the order in which the Z2 worked example lists its
  fusion channels (Sec. 3.2, eq. abeliangroupexample and the right-bend example after it);
  the fusion trees of the domain use the same rule;
* blocks are keyed by the coupled sector c, ascending; inside block c the splitting trees with
  coupled sector c occupy consecutive row ranges in tree order, each of height prod_i n_{a_i},
  and the fusion trees consecutive column ranges;
* the reduced array of a tree pair is stored column-major with the first leg fastest
  (eq. linearindex), rows = codomain legs, columns = domain legs;
* each block is a column-major rows_c x cols_c matrix; blocks are concatenated in c order and
  only blocks with rows_c > 0 and cols_c > 0 are stored.

Pinned by the Z2 and SU(2) worked examples of the paper (block shapes and tree counts) and by
brute-force counting of invariant-subspace dimensions (tests/test_oracle_structure.py).
"""

from dataclasses import dataclass, field
from functools import cached_property
from itertools import product
from math import prod

from .symmetry import Symmetry

__all__ = ["GradedSpace", "TreePair", "TensorStructure", "enumerate_trees"]


class GradedSpace:
    """V = (+)_a C^{n_a} (x) V^(a), stored as sorted (sector, n_a) pairs plus a dual flag."""

    def __init__(self, sym: Symmetry, sectors, dual: bool = False):
        if isinstance(sectors, dict):
            items = list(sectors.items())
        else:
            items = list(sectors)
        clean = {}
        for a, n in items:
            a = int(a)
            n = int(n)
            if not sym.valid(a):
                raise ValueError(f"invalid {sym.name} sector {a}")
            if n <= 0:
                raise ValueError("multiplicities must be positive")
            if a in clean:
                raise ValueError("duplicate sector")
            clean[a] = n
        self.sym = sym
        self.sectors = dict(sorted(clean.items()))
        self.dual = bool(dual)

    # -- identity -------------------------------------------------------------
    def key(self):
        return (self.sym.name, tuple(self.sectors.items()), self.dual)

    def __eq__(self, other):
        return isinstance(other, GradedSpace) and self.key() == other.key()

    def __hash__(self):
        return hash(self.key())

    def __repr__(self):
        s = ", ".join(f"{a}:{n}" for a, n in self.sectors.items())
        return f"{self.sym.name}[{s}]" + ("*" if self.dual else "")

    def flip(self) -> "GradedSpace":
        """The dual space V* (same underlying sectors, dual flag toggled)."""
        return GradedSpace(self.sym, self.sectors, not self.dual)

    # -- tree labels ----------------------------------------------------------
    def tree_label(self, a):
        """Label carried in fusion trees by underlying sector a of this leg."""
        return self.sym.dual(a) if self.dual else a

    def underlying(self, label):
        return self.sym.dual(label) if self.dual else label

    @cached_property
    def labels(self):
        """Sorted tree labels of this leg."""
        return sorted(self.tree_label(a) for a in self.sectors)

    def mult_of_label(self, label):
        return self.sectors[self.underlying(label)]

    # -- dense basis |a, k, m> (oracle-internal order: a ascending, then k, then m) ---------
    @cached_property
    def dense_offsets(self):
        off, out = 0, {}
        for a, n in self.sectors.items():
            out[a] = off
            off += n * self.sym.dim(a)
        return out

    @cached_property
    def dim(self):
        return sum(n * self.sym.dim(a) for a, n in self.sectors.items())

    @cached_property
    def reduced_dim(self):
        return sum(self.sectors.values())


def enumerate_trees(sym: Symmetry, legs):
    """All canonical trees on ``legs`` (a list of GradedSpace), in the canonical order.

    Returns a list of (uncoupled labels tuple, inner labels tuple, coupled).
    """
    n = len(legs)
    if n == 0:
        return [((), (), sym.unit())]
    out = []
    for unc in product(*[leg.labels for leg in legs]):
        if n == 1:
            out.append((unc, (), unc[0]))
            continue
        # running couplings u_2 .. u_N ; inner = (u_2..u_{N-1}), coupled = u_N
        partial = [((), unc[0])]
        for k in range(1, n):
            nxt = []
            for inner, u in partial:
                for v in sorted(sym.fuse(u, unc[k])):
                    nxt.append((inner + (v,), v))
            partial = nxt
        for chain, c in partial:
            out.append((unc, chain[:-1], c))
    # canonical order: colexicographic (first leg fastest) in the uncoupled labels, then
    # colexicographic in the inner labels -- the channel order of the Z2 worked examples
    out.sort(key=lambda t: (tuple(reversed(t[0])), tuple(reversed(t[1]))))
    return out


@dataclass(frozen=True)
class TreePair:
    coupled: int
    split_unc: tuple
    split_inner: tuple
    fuse_unc: tuple
    fuse_inner: tuple
    offset: int          # element offset of the (0,..,0) entry in the flat storage
    ld: int              # leading dimension (= rows of the block)
    row_off: int
    col_off: int
    dims: tuple = field(default=())   # extents: codomain legs then domain legs

    @property
    def labels(self):
        return (self.split_unc, self.split_inner, self.coupled, self.fuse_unc, self.fuse_inner)


class TensorStructure:
    """Block layout of a TensorMap  dom[0] (x) ... -> cod[0] (x) ...  (codomain <- domain)."""

    def __init__(self, cod, dom):
        cod, dom = list(cod), list(dom)
        legs = cod + dom
        if not legs:
            raise ValueError("a tensor map needs at least one leg")
        sym = legs[0].sym
        if any(l.sym is not sym for l in legs):
            raise ValueError("mixed symmetries")
        self.sym, self.cod, self.dom = sym, cod, dom

        def group(trees, spaces):
            by_c = {}
            for unc, inner, c in trees:
                size = prod(sp.mult_of_label(a) for sp, a in zip(spaces, unc))
                by_c.setdefault(c, []).append((unc, inner, size))
            return by_c

        split = group(enumerate_trees(sym, cod), cod)
        fuse = group(enumerate_trees(sym, dom), dom)
        blocks, pairs, off = [], [], 0
        for c in sorted(set(split) & set(fuse)):
            rows = sum(t[2] for t in split[c])
            cols = sum(t[2] for t in fuse[c])
            if rows == 0 or cols == 0:
                continue
            blocks.append((c, rows, cols, off))
            roff = 0
            for su, si, rs in split[c]:
                coff = 0
                for fu, fi, cs in fuse[c]:
                    dims = tuple(sp.mult_of_label(a) for sp, a in zip(cod, su)) + \
                        tuple(sp.mult_of_label(a) for sp, a in zip(dom, fu))
                    pairs.append(TreePair(c, su, si, fu, fi, off + roff + coff * rows, rows,
                                          roff, coff, dims))
                    coff += cs
                roff += rs
            off += rows * cols
        self.blocks = blocks
        self.pairs = pairs
        self.numel = off

    @property
    def nleg(self):
        return len(self.cod) + len(self.dom)

    def spaces(self):
        return self.cod + self.dom

    def block_dict(self):
        return {c: (rows, cols, off) for c, rows, cols, off in self.blocks}

    def pair_index(self):
        return {p.labels: p for p in self.pairs}

    def __repr__(self):
        return f"TensorStructure({self.cod} <- {self.dom}, blocks={len(self.blocks)}, numel={self.numel})"
