"""Low multilinear rank (Tucker) compression of the Toeplitz defining tensors (oracle; test
infrastructure only).

Section III-C notes that the Toeplitz defining tensors of the N (and K) operator can be
compressed further by low multilinear rank decompositions.  The oracle takes the textbook
truncated higher-order SVD (De Lathauwer, De Moor & Vandewalle, SIAM J. Matrix Anal. Appl. 21,
2000): for each mode k of a tensor T (axes z, y, x) the left singular vectors U_k of the mode-k
unfolding T_(k), truncated to the smallest rank r_k whose discarded singular values satisfy

    sum_{i > r_k} sigma_i(T_(k))^2 <= tol^2 ||T||_F^2 / 3,

and the core S = T x_1 U_1^H x_2 U_2^H x_3 U_3^H.  Because the three projections are orthogonal,
||T - S x_1 U_1 x_2 U_2 x_3 U_3||_F^2 <= sum over modes of the discarded energy <= tol^2 ||T||_F^2.
"""

from __future__ import annotations

import numpy as np


def unfold(T, k):
    """Mode-k unfolding: the axis k first, the other two flattened in order."""
    return np.moveaxis(T, k, 0).reshape(T.shape[k], -1)


def mode_product(T, U, k):
    """T x_k U: contracts axis k of T with the columns of U (U has T.shape[k] columns)."""
    return np.moveaxis(np.tensordot(U, T, axes=(1, k)), 0, k)


def truncation_rank(sigma, threshold):
    """Smallest r with sum_{i >= r} sigma_i^2 <= threshold (sigma in decreasing order)."""
    tail = np.concatenate([np.cumsum((sigma ** 2)[::-1])[::-1], [0.0]])
    return int(np.argmax(tail <= threshold))


def hosvd(T, tol):
    """Truncated HOSVD of a 3-way array T at relative tolerance tol: (core, [U_z, U_y, U_x])."""
    T = np.asarray(T, dtype=complex)
    thr = tol * tol * np.vdot(T, T).real / 3.0
    Us = []
    for k in range(3):
        U, s, _ = np.linalg.svd(unfold(T, k), full_matrices=False)
        r = max(truncation_rank(s, thr), 1)
        Us.append(U[:, :r])
    S = T
    for k, U in enumerate(Us):
        S = mode_product(S, U.conj().T, k)
    return S, Us


def reconstruct(S, Us):
    T = S
    for k, U in enumerate(Us):
        T = mode_product(T, U, k)
    return T


def compressed_values(S, Us):
    """Complex values stored by the Tucker form: the core plus the three factors."""
    return S.size + sum(U.size for U in Us)
