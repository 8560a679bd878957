"""Sector algebra of the three symmetries on the path (oracle; test infrastructure).

* Z2: sectors {0, 1}, a (x) b = a xor b, self-dual (fusion table of Sec. 3.2).
* U(1): integer charges, a (x) b = a + b, dual(a) = -a (abelian, N_ab^c = delta_{c,ab}).
* SU(2): sectors 2j, triangle rule, self-dual, d_j = 2j+1 (eq. SU2NSymbol).

Abelian sectors are one-dimensional: the splitting tensor is the number 1 and Z = 1.  SU(2)
splitting tensors are explicit CG arrays from :mod:`oracle.su2`.
"""

import numpy as np

from . import su2

__all__ = ["Symmetry", "U1", "Z2", "SU2", "sym_from_name"]


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


U1 = _U1()
Z2 = _Z2()
SU2 = _SU2()


def sym_from_name(name: str) -> Symmetry:
    return {"U1": U1, "Z2": Z2, "SU2": SU2}[name]
