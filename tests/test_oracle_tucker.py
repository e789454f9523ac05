"""Pins of the oracle's truncated HOSVD (oracle/tucker.py): exact recovery of a known multilinear
rank, the closed-form ranks and error of a superdiagonal tensor and their invariance under unitary
changes of basis in each mode, the error bound, and the compression of the Green tensors with the
matvec they give."""

import numpy as np
import pytest

from oracle import green as OG
from oracle import operator as O
from oracle import tucker as T
from synth import Grid, random_coefficients


def _unitary(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    q, r = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_known_multilinear_rank_is_recovered():
    rng = np.random.Generator(np.random.PCG64(1))
    S = rng.standard_normal((3, 4, 5)) + 1j * rng.standard_normal((3, 4, 5))
    Us = [_unitary(n, 10 + n)[:, :r] for n, r in ((9, 3), (8, 4), (11, 5))]
    A = T.reconstruct(S, Us)
    S2, U2 = T.hosvd(A, 1e-12)
    assert [U.shape[1] for U in U2] == [3, 4, 5]
    assert np.linalg.norm(T.reconstruct(S2, U2) - A) <= 1e-13 * np.linalg.norm(A)


@pytest.mark.parametrize("tol", [3e-1, 1e-2, 1e-4])
def test_superdiagonal_ranks_and_error_in_closed_form(tol):
    """T[i, i, i] = 2^-i: every unfolding has singular values 2^-i, so the rank is the smallest r
    with sum_{i >= r} 4^-i <= tol^2 sum 4^-i / 3 and the error is sqrt(sum_{i >= r} 4^-i) exactly;
    unitary changes of basis in the three modes change neither."""
    n = 10
    d = 2.0 ** -np.arange(n)
    D = np.zeros((n, n, n), dtype=complex)
    D[np.arange(n), np.arange(n), np.arange(n)] = d
    total = np.sum(d ** 2)
    r = next(r for r in range(n + 1) if np.sum(d[r:] ** 2) <= tol * tol * total / 3)
    err = np.sqrt(np.sum(d[r:] ** 2))
    for A in (D, T.reconstruct(D, [_unitary(n, 3), _unitary(n, 4), _unitary(n, 5)])):
        S, Us = T.hosvd(A, tol)
        assert [U.shape[1] for U in Us] == [r, r, r]
        assert abs(np.linalg.norm(T.reconstruct(S, Us) - A) - err) <= 1e-12 * np.sqrt(total)
        assert err <= tol * np.sqrt(total)


def test_rank_one_and_error_bound():
    rng = np.random.Generator(np.random.PCG64(7))
    a, b, c = (rng.standard_normal(n) + 1j * rng.standard_normal(n) for n in (6, 7, 8))
    A = np.einsum("i,j,k->ijk", a, b, c)
    S, Us = T.hosvd(A, 1e-10)
    assert [U.shape[1] for U in Us] == [1, 1, 1]
    assert np.linalg.norm(T.reconstruct(S, Us) - A) <= 1e-13 * np.linalg.norm(A)
    # a full-rank tensor with decaying multilinear spectrum: the bound holds at every tolerance
    core = np.einsum("i,j,k->ijk", *(0.5 ** np.arange(n) for n in (9, 8, 11))) * (
        1 + 0.1 * (rng.standard_normal((9, 8, 11)) + 1j * rng.standard_normal((9, 8, 11))))
    B = T.reconstruct(core, [_unitary(9, 1), _unitary(8, 2), _unitary(11, 3)])
    for tol in (1e-1, 1e-3, 1e-6):
        S, Us = T.hosvd(B, tol)
        assert np.linalg.norm(T.reconstruct(S, Us) - B) <= tol * np.linalg.norm(B)


@pytest.mark.slow
def test_green_tensors_compress_and_keep_the_matvec():
    """The 60 unique Toeplitz tensors of a 12^3 grid at 298 MHz compress below their full size at
    tol 1e-6, and the N matvec from the reconstructed tensors stays within a few tol of the exact one."""
    g = Grid(12, 12, 12, 0.005, 0.005, 0.005)
    k0 = O.k0_of(298e6)
    TT = OG.toeplitz_tensors(g, k0)  # (12, 12, 2Nz-1, 2Ny-1, 2Nx-1)
    tol = 1e-6
    full = comp = 0
    TR = np.empty_like(TT)
    for a in range(12):
        for b in range(12):
            S, Us = T.hosvd(TT[a, b], tol)
            TR[a, b] = T.reconstruct(S, Us)
            full += TT[a, b].size
            comp += T.compressed_values(S, Us)
            assert np.linalg.norm(TR[a, b] - TT[a, b]) <= tol * np.linalg.norm(TT[a, b])
    assert comp < 0.5 * full
    x = random_coefficients(g, 1, seed=5)
    y = O.NOperator(g, k0, TT).apply(x)
    yr = O.NOperator(g, k0, TR).apply(x)
    assert np.linalg.norm(yr - y) <= 10 * tol * np.linalg.norm(y)
