"""Dense matrix-product operators of the benchmark models (oracle; test infrastructure).

Only tests/, the smoke check and the benchmark's CPU baseline use this package.

SU(2) Heisenberg chain H = J sum_i S_i . S_{i+1} (the paper's SU(2) benchmark model, Sec. 6.1)
as the lower-triangular MPO with bond space 2 (0) (+) (1) (the two identity channels and the
spin vector), on the legs W : W (x) P <- P (x) W of the heff workload, P = (1/2).

Dense layout W[w_l, s', s, w_r] = <w_l, s'| W |s, w_r>: bond basis (j = 0, copy 0) = "start",
(j = 0, copy 1) = "end", then (j = 1, m = -1, 0, 1); physical basis m_s = -1/2, +1/2.  With the
spherical components T_{+1} = -S^+ / sqrt 2, T_0 = S^z, T_{-1} = S^- / sqrt 2 of the spin vector:

    W[start][start] = W[end][end] = 1,
    W[(1, m)][start] = (-1)^m T_{-m},      W[end][(1, m)] = J T_m,

so that the two-site operator sum_m W[end][(1, m)] (x) W[(1, m)][start] is
J sum_m (-1)^m T_m (x) T_{-m} = J S . S.  The first column transforms contragrediently and the
last row covariantly under rotations, which makes the whole array invariant (the pins in
tests/test_oracle_models.py check invariance and the two-site operator directly).
"""

import math

import numpy as np

__all__ = ["spin_half_ops", "heisenberg_su2_mpo_dense", "heisenberg_two_site"]


def spin_half_ops():
    """(S^+, S^-, S^z) on the basis (m_s = -1/2, +1/2); matrices act as [out, in]."""
    sp = np.zeros((2, 2))
    sp[1, 0] = 1.0
    return sp, sp.T.copy(), np.diag([-0.5, 0.5])


def heisenberg_su2_mpo_dense(J: float = 1.0) -> np.ndarray:
    sp, sm, sz = spin_half_ops()
    r2 = math.sqrt(2.0)
    T = {1: -sp / r2, 0: sz, -1: sm / r2}
    W = np.zeros((5, 2, 2, 5))
    start, end = 0, 1
    W[start, :, :, start] = np.eye(2)
    W[end, :, :, end] = np.eye(2)
    for i, m in enumerate((-1, 0, 1)):
        W[2 + i, :, :, start] = (-1) ** m * T[-m]
        W[end, :, :, 2 + i] = J * T[m]
    return W


def heisenberg_two_site(J: float = 1.0) -> np.ndarray:
    """J S . S on two spins-1/2 as a [s1', s2', s1, s2] array, from S^+, S^-, S^z directly."""
    sp, sm, sz = spin_half_ops()
    h = J * (np.kron(sz, sz) + 0.5 * (np.kron(sp, sm) + np.kron(sm, sp)))
    return h.reshape(2, 2, 2, 2)
