"""MoM system of the dielectric current-based VIE (oracle; test infrastructure only).

  A = M_eps G - M_chi N,   b = c_e M_chi e_inc          (Section III-B, Eq. 24)
  P = M_eps G,  P^-1 A = I - M_tau G^-1 N,  tau = chi/eps   (Section IV-B, Eq. 17)

with eps = eps' - i sigma/(omega eps0) per voxel (Eq. 2, 23; time factor
exp(i omega t)), chi = eps - 1 (Eq. 7), c_e = i omega eps0 (Eq. 6), G the
diagonal Gram matrix (Eq. 33) and N the Galerkin matrix of the N operator
(green.py).  N x is evaluated either densely (tiny grids) or by embedding the
Toeplitz defining tensors (Eq. 43) into 2N circulant tensors and using the FFT
(Section IV-A).  Unknowns are ordered x[alpha][z][y][x], alpha = 4 p + l - 1.
"""

from __future__ import annotations

import dataclasses
import os

import numpy as np
import scipy.fft


from . import C0, EPS0
from .green import NCOMP, gram, k_toeplitz_tensors, toeplitz_tensors


# The FFT steps go through scipy.fft with one worker thread per core this process may run
# on; the transform is the plain DFT of Section IV-A either way.
FFT_WORKERS = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _fftn(a):
    return scipy.fft.fftn(a, axes=(-3, -2, -1), workers=FFT_WORKERS)


def _ifftn(a):
    return scipy.fft.ifftn(a, axes=(-3, -2, -1), workers=FFT_WORKERS)


def k0_of(freq):
    """Free-space wavenumber k0 = omega sqrt(mu0 eps0) = 2 pi f / c0 (Section II)."""
    return 2.0 * np.pi * freq / C0


@dataclasses.dataclass
class Problem:
    grid: object
    freq: float
    eps_real: np.ndarray
    sigma: np.ndarray

    @property
    def omega(self):
        return 2.0 * np.pi * self.freq

    @property
    def k0(self):
        return k0_of(self.freq)

    @property
    def ce(self):
        return 1j * self.omega * EPS0

    @property
    def eps(self):
        return self.eps_real - 1j * self.sigma / (self.omega * EPS0)

    @property
    def chi(self):
        return self.eps - 1.0

    @property
    def tau(self):
        return self.chi / self.eps

    @property
    def dV(self):
        g = self.grid
        return g.dx * g.dy * g.dz

    def gram_vector(self):
        """G^l per component alpha (12,), Eq. 33."""
        return np.array([gram(a % 4 + 1, self.dV) for a in range(NCOMP)])


def circulant(T, shape):
    """Embed Toeplitz tensors T[..., 2Nz-1, 2Ny-1, 2Nx-1] into 2N circulants.

    C(j) = T(j) for 0 <= j < N, C(N) = 0, C(j) = T(j - 2N) for N < j < 2N, per axis
    (offset d stored at index d + N - 1 of T)."""
    nz, ny, nx = shape

    def idx(n):
        # circulant positions j != N and the Toeplitz array index (d + n - 1) they take
        j = np.array([i for i in range(2 * n) if i != n])
        d = np.where(j < n, j, j - 2 * n)
        return j, d + n - 1

    out = np.zeros(T.shape[:-3] + (2 * nz, 2 * ny, 2 * nx), dtype=complex)
    (jz, tz), (jy, ty), (jx, tx) = idx(nz), idx(ny), idx(nx)
    out[..., jz[:, None, None], jy[None, :, None], jx[None, None, :]] = T[
        ..., tz[:, None, None], ty[None, :, None], tx[None, None, :]
    ]
    return out


class NOperator:
    """N x by circulant embedding + FFT (Section IV-A), from the oracle's own Toeplitz tensors."""

    def __init__(self, grid, k0, T=None):
        self.grid = grid
        self.shape = grid.shape
        if T is None:
            T = toeplitz_tensors(grid, k0)
        self.T = T
        self.Chat = _fftn(circulant(T, self.shape))

    def apply(self, x):
        """x: (..., 12, Nz, Ny, Nx) complex -> N x of the same shape."""
        nz, ny, nx = self.shape
        pad = np.zeros(x.shape[:-3] + (2 * nz, 2 * ny, 2 * nx), dtype=complex)
        pad[..., :nz, :ny, :nx] = x
        X = _fftn(pad)
        Y = _block_apply(self.Chat, X)
        y = _ifftn(Y)
        return y[..., :nz, :ny, :nx]


class KOperator(NOperator):
    """K x (K u = curl S u, Eq. 8) by the same circulant embedding + FFT, from the K tensors."""

    def __init__(self, grid, k0, T=None):
        super().__init__(grid, k0, k_toeplitz_tensors(grid, k0) if T is None else T)


def _block_apply(Chat, X):
    """Y_alpha(k) = sum_beta Chat_{alpha beta}(k) X_beta(k) at every frequency point k."""
    Y = np.zeros_like(X)
    for a in range(NCOMP):
        acc = np.zeros(X.shape[:-4] + X.shape[-3:], dtype=complex)
        for b in range(NCOMP):
            acc += Chat[a, b] * X[..., b, :, :, :]
        Y[..., a, :, :, :] = acc
    return Y


def apply_A(prob: Problem, Nop: NOperator, x):
    """A x = M_eps G x - M_chi N x (Eq. 24)."""
    G = prob.gram_vector()[:, None, None, None]
    return prob.eps * G * x - prob.chi * Nop.apply(x)


def apply_PA(prob: Problem, Nop: NOperator, x):
    """P^-1 A x with P = M_eps G (Section IV-B)."""
    G = prob.gram_vector()[:, None, None, None]
    return (prob.eps * G * x - prob.chi * Nop.apply(x)) / (prob.eps * G)


def apply_Pinv(prob: Problem, v):
    G = prob.gram_vector()[:, None, None, None]
    return v / (prob.eps * G)


# PWC variant (the paper's comparison solver, Section V-A): one constant function per
# component and voxel, f = N^1 p-hat, so its Galerkin system is exactly the l = 1 sub-block
# of the PWL system (Eq. 19-22 with l = l' = 1: N entries, Gram G^1 = DV, P = M_eps G, b).
PWC_COMPONENTS = (0, 4, 8)


def pwc_mask():
    """(12, 1, 1, 1) mask keeping the l = 1 components: the PWC unknowns inside the PWL layout."""
    m = np.zeros((NCOMP, 1, 1, 1))
    m[list(PWC_COMPONENTS)] = 1.0
    return m


def apply_PA_pwc(prob: Problem, Nop: NOperator, x):
    """P^-1 A of the PWC system on vectors in the PWL layout: the l = 1 sub-block, zero elsewhere."""
    m = pwc_mask()
    return m * apply_PA(prob, Nop, m * x)


def dense_N(grid, T):
    """Dense Galerkin matrix N (12 N_V x 12 N_V) from the Toeplitz values, entry (m alpha, n beta) = T^{alpha beta}(m - n)."""
    nz, ny, nx = grid.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    zz, yy, xx = zz.ravel(), yy.ravel(), xx.ravel()
    nv = zz.size
    dz = zz[:, None] - zz[None, :] + nz - 1
    dy = yy[:, None] - yy[None, :] + ny - 1
    dx = xx[:, None] - xx[None, :] + nx - 1
    M = np.zeros((NCOMP, nv, NCOMP, nv), dtype=complex)
    for a in range(NCOMP):
        for b in range(NCOMP):
            M[a, :, b, :] = T[a, b][dz, dy, dx]
    return M.reshape(NCOMP * nv, NCOMP * nv)


def dense_A(prob: Problem, T):
    """Dense MoM matrix A = M_eps G - M_chi N (Eq. 24) for tiny grids."""
    nv = prob.grid.nv
    N = dense_N(prob.grid, T)
    G = np.repeat(prob.gram_vector(), nv)
    eps = np.tile(prob.eps.ravel(), NCOMP)
    chi = np.tile(prob.chi.ravel(), NCOMP)
    return np.diag(eps * G) - chi[:, None] * N
