"""Sector algebra of the three symmetries on the path (oracle; test infrastructure).

* Z2: sectors {0, 1}, a (x) b = a xor b, self-dual (fusion table of Sec. 3.2).
* U(1): integer charges, a (x) b = a + b, dual(a) = -a (abelian, N_ab^c = delta_{c,ab}).
* SU(2): sectors 2j, triangle rule, self-dual, d_j = 2j+1 (eq. SU2NSymbol).
* Deligne products S1 x S2 (Sec. 5.2): sectors are pairs (a1, a2); fusion, duals and dimensions
  act factor by factor and the splitting tensor of a pair is the Kronecker product of the
  factors' splitting tensors (the product basis |m1> (x) |m2> in row-major order).  A pair is
  held as the integer a1 * 4096 + f(a2), f(a2) = a2 + 2048 for a U(1) second factor and a2
  otherwise, so that integer order is lexicographic pair order (the layout's sector order).

Abelian sectors are one-dimensional: the splitting tensor is the number 1 and Z = 1.  SU(2)
splitting tensors are explicit CG arrays from :mod:`oracle.su2`.
"""

import numpy as np

from . import su2

__all__ = ["Symmetry", "U1", "Z2", "SU2", "U1xSU2", "Z2xU1", "ProductSymmetry", "sym_from_name"]


class Symmetry:
    name = "?"
    abelian = True

    def fuse(self, a, b):
        raise NotImplementedError

    def dual(self, a):
        raise NotImplementedError

    def dim(self, a):
        return 1

    def unit(self):
        return 0

    def valid(self, a):
        raise NotImplementedError

    def nsym(self, a, b, c):
        return 1 if c in self.fuse(a, b) else 0

    # explicit representation data used by the dense embedding
    def cg_tensor(self, a, b, c):
        return np.ones((1, 1, 1)) if self.nsym(a, b, c) else np.zeros((1, 1, 1))

    def zmat(self, a):
        return np.ones((1, 1))

    def __repr__(self):
        return self.name


class _U1(Symmetry):
    name = "U1"

    def fuse(self, a, b):
        return [a + b]

    def dual(self, a):
        return -a

    def valid(self, a):
        return isinstance(a, (int, np.integer))


class _Z2(Symmetry):
    name = "Z2"

    def fuse(self, a, b):
        return [a ^ b]

    def dual(self, a):
        return a

    def valid(self, a):
        return a in (0, 1)


class _SU2(Symmetry):
    name = "SU2"
    abelian = False

    def fuse(self, a, b):
        return list(range(abs(a - b), a + b + 1, 2))

    def dual(self, a):
        return a

    def dim(self, a):
        return a + 1

    def valid(self, a):
        return isinstance(a, (int, np.integer)) and a >= 0

    def cg_tensor(self, a, b, c):
        return su2.cg_tensor(a, b, c)

    def zmat(self, a):
        return su2.zmat(a)


class ProductSymmetry(Symmetry):
    """Deligne product of two symmetries with integer-encoded pair sectors (module header)."""

    SHIFT = 4096

    def __init__(self, s1: Symmetry, s2: Symmetry):
        self.s1, self.s2 = s1, s2
        self.name = f"{s1.name}x{s2.name}"
        self.abelian = s1.abelian and s2.abelian
        self.off = 2048 if s2 is U1 else 0

    def pair(self, a1, a2):
        return int(a1) * self.SHIFT + int(a2) + self.off

    def split(self, a):
        a1, f = divmod(int(a), self.SHIFT)
        return a1, f - self.off

    def fuse(self, a, b):
        (a1, a2), (b1, b2) = self.split(a), self.split(b)
        return sorted(self.pair(c1, c2) for c1 in self.s1.fuse(a1, b1) for c2 in self.s2.fuse(a2, b2))

    def dual(self, a):
        a1, a2 = self.split(a)
        return self.pair(self.s1.dual(a1), self.s2.dual(a2))

    def dim(self, a):
        a1, a2 = self.split(a)
        return self.s1.dim(a1) * self.s2.dim(a2)

    def unit(self):
        return self.pair(self.s1.unit(), self.s2.unit())

    def valid(self, a):
        if not isinstance(a, (int, np.integer)):
            return False
        a1, a2 = self.split(a)
        return self.s1.valid(a1) and self.s2.valid(a2) and 0 <= a2 + self.off < self.SHIFT

    def cg_tensor(self, a, b, c):
        (a1, a2), (b1, b2), (c1, c2) = self.split(a), self.split(b), self.split(c)
        t1, t2 = self.s1.cg_tensor(a1, b1, c1), self.s2.cg_tensor(a2, b2, c2)
        t = np.einsum("ijk,lmn->iljmkn", t1, t2)
        return t.reshape(t1.shape[0] * t2.shape[0], t1.shape[1] * t2.shape[1], t1.shape[2] * t2.shape[2])

    def zmat(self, a):
        a1, a2 = self.split(a)
        return np.kron(self.s1.zmat(a1), self.s2.zmat(a2))


U1 = _U1()
Z2 = _Z2()
SU2 = _SU2()
U1xSU2 = ProductSymmetry(U1, SU2)
Z2xU1 = ProductSymmetry(Z2, U1)


def sym_from_name(name: str) -> Symmetry:
    return {"U1": U1, "Z2": Z2, "SU2": SU2, "U1xSU2": U1xSU2, "Z2xU1": Z2xU1}[name]
