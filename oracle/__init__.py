"""CPU oracle for the symmetric TensorMap contraction path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct restatement of what the paper defines:

* graded spaces of Z2, U(1) and SU(2) sectors with multiplicities (Sec. 5.2, objects;
  Sec. 3, eq. gradedbasis);
* the canonical fusion-tree block layout of a TensorMap (Sec. 4.1, eq. canonicalsplitting and
  the block-diagonal form; Sec. 3.2, eq. abeliangrouping);
* the dense embedding t = sum_(s,f) X_s (t^(s,f) (x) 1_c) X_f^dagger built from explicit
  Clebsch-Gordan coefficients (Wigner-Eckart theorem, Sec. 4.1) with Z on dual legs (Sec. 4.2);
* permute as an array permutation and composition as a matrix product in the dense picture
  (Sec. 2.2 eq. permute_coeffs and the unstructured reduction; eq. tm_composition), and the
  pairwise contraction of Algorithm 4;
* a block-sparse second tier whose recoupling coefficients come from projecting permuted
  explicit fusion trees onto the canonical basis (the overlap route of Sec. 4.2).

It shares no code with the CUDA path (``paper_2508_10076_gb300``) and never imports it; the
product never imports this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or execute
anything here.

Sector encoding (shared *interface* convention, not shared code): U(1) integer charge, Z2 in
{0,1}, SU(2) twice the spin (2j).

Parity status: every function here is pinned by tests under ``tests/test_oracle_*.py``; see the
header of each module.  The only items pinned up to figure-only labelling are the two SU(2)
worked examples (transposition and permutation matrices), whose tree numbering exists only in
the paper's figures.
"""

from .symmetry import Symmetry, U1, Z2, SU2, sym_from_name  # noqa: F401
from .structure import GradedSpace, TensorStructure  # noqa: F401
