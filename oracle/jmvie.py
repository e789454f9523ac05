"""Full JM-VIE: polarization and magnetization currents together (oracle; test infrastructure only).

With j = c_e chi_e e and m = c_m chi_m h (Eq. 6), chi_e = eps_r - 1 and chi_m = mu_r - 1
(Eq. 7), and the scattered fields of Eq. 13, the total fields e = e_inc + e_sca,
h = h_inc + h_sca give the system of Eq. 14-15:

    [ M_eps - M_chie N        c_e M_chie K     ] [j]   [ c_e M_chie e_inc ]
    [ -c_m M_chim K           M_mu - M_chim N  ] [m] = [ c_m M_chim h_inc ]

Both currents are expanded in the same PWL functions (Section III-A notes that the
magnetization current takes the basis of the polarization current), and Galerkin testing
turns M_eps into M_eps G (G the Gram matrix, Eq. 33) and N, K into their Galerkin matrices
(green.py, Eq. 25).

Scaled magnetization unknown.  The two currents differ in size by about eta0 = sqrt(mu0/eps0)
(j ~ c_e e, m ~ c_m h, |e| ~ eta0 |h|).  Here the unknown is m' = m / eta0, and the second row
is divided by eta0.  Since c_e eta0 = c_m / eta0 = i k0, the system reads

    [ M_eps G - M_chie N      i k0 M_chie K      ] [j ]   [ c_e M_chie e_inc  ]
    [ -i k0 M_chim K          M_mu G - M_chim N  ] [m'] = [ i k0 M_chim h_inc ]

It has the same solution as Eq. 15 with m = eta0 m'.  With D = diag(1/chi_e, -1/chi_m) the
product D A is complex symmetric (N and K are), which is the discrete form of reciprocity.
The preconditioner is P = diag(M_eps G, M_mu G), the material terms of both rows (Section
IV-B does the same for Eq. 16).

Fields (Eq. 13, tested, then divided by the Gram matrix as in post.py):
    e~ = e_inc + (1/c_e)(N - G) j - eta0 K m'
    h~ = h_inc + K j + (1/(i k0))(N - G) m'
Absorbed power: the electric part of Eq. 44 plus its magnetic analogue
    1/2 Re{ m^* (c_m M_chim)^-1 G m } = 1/2 Re{ eta0 |m'|^2 G / (i k0 chi_m) },
which equals 1/2 int omega mu0 mu'' |h|^2 (the magnetic loss).

Vectors are (..., 2, 12, Nz, Ny, Nx): index 0 of the axis before the components holds j,
index 1 holds m'.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import EPS0, MU0
from .operator import Problem, dense_N

ETA0 = float(np.sqrt(MU0 / EPS0))


@dataclasses.dataclass
class MagProblem(Problem):
    """A Problem with a relative permeability mu_r = mu_real - i mu_imag per voxel (Eq. 1-2)."""

    mu_real: np.ndarray = None
    mu_imag: np.ndarray = None

    @property
    def mu(self):
        mr = np.ones(self.grid.shape) if self.mu_real is None else self.mu_real
        mi = np.zeros(self.grid.shape) if self.mu_imag is None else self.mu_imag
        return mr - 1j * mi

    @property
    def chim(self):
        return self.mu - 1.0


def _split(x):
    return x[..., 0, :, :, :, :], x[..., 1, :, :, :, :]


def apply_A(prob: MagProblem, Nop, Kop, x):
    """A x of the scaled system above (Eq. 14-15 with m = eta0 m')."""
    G = prob.gram_vector()[:, None, None, None]
    j, mp = _split(x)
    ik0 = 1j * prob.k0
    y1 = prob.eps * G * j - prob.chi * Nop.apply(j) + ik0 * prob.chi * Kop.apply(mp)
    y2 = prob.mu * G * mp - prob.chim * Nop.apply(mp) - ik0 * prob.chim * Kop.apply(j)
    return np.stack([y1, y2], axis=-5)


def apply_Pinv(prob: MagProblem, v):
    """P^-1 v with P = diag(M_eps G, M_mu G)."""
    G = prob.gram_vector()[:, None, None, None]
    v1, v2 = _split(v)
    return np.stack([v1 / (prob.eps * G), v2 / (prob.mu * G)], axis=-5)


def apply_PA(prob: MagProblem, Nop, Kop, x):
    """P^-1 A x."""
    return apply_Pinv(prob, apply_A(prob, Nop, Kop, x))


def rhs(prob: MagProblem, e_tested, h_tested):
    """b = (c_e M_chie e_inc, i k0 M_chim h_inc): the right side of Eq. 14 with its second row / eta0."""
    return np.stack([prob.ce * prob.chi * e_tested, 1j * prob.k0 * prob.chim * h_tested], axis=-5)


def dense_A(prob: MagProblem, TN, TK):
    """Dense matrix of the scaled system for tiny grids, from the Toeplitz tensors of N and K;
    unknown order (half, alpha, z, y, x)."""
    G = np.repeat(prob.gram_vector(), prob.grid.nv)
    eps = np.tile(prob.eps.ravel(), 12)
    mu = np.tile(prob.mu.ravel(), 12)
    ce = np.tile(prob.chi.ravel(), 12)
    cm = np.tile(prob.chim.ravel(), 12)
    N = dense_N(prob.grid, TN)
    K = dense_N(prob.grid, TK)
    ik0 = 1j * prob.k0
    top = np.hstack([np.diag(eps * G) - ce[:, None] * N, ik0 * ce[:, None] * K])
    bot = np.hstack([-ik0 * cm[:, None] * K, np.diag(mu * G) - cm[:, None] * N])
    return np.vstack([top, bot])


def fields(prob: MagProblem, Nop, Kop, x, e_tested, h_tested):
    """PWL coefficients (e, h), each (..., 12, Nz, Ny, Nx), of the total fields (Eq. 13)."""
    G = prob.gram_vector()[:, None, None, None]
    j, mp = _split(x)
    et = e_tested + (Nop.apply(j) - G * j) / prob.ce - ETA0 * Kop.apply(mp)
    ht = h_tested + Kop.apply(j) + (Nop.apply(mp) - G * mp) / (1j * prob.k0)
    return et / G, ht / G


def absorbed_power(prob: MagProblem, x):
    """(p (..., Nz, Ny, Nx) in W/m^3, P (...) in W): electric plus magnetic loss."""
    G = prob.gram_vector()[:, None, None, None]
    j, mp = _split(x)
    te, tm = prob.chi != 0, prob.chim != 0
    de = np.where(te, prob.ce * prob.chi, 1.0)
    dm = np.where(tm, 1j * prob.k0 * prob.chim, 1.0)
    pe = np.where(te, 0.5 * np.real((np.abs(j) ** 2 * G).sum(-4) / de), 0.0)
    pm = np.where(tm, 0.5 * np.real(ETA0 * (np.abs(mp) ** 2 * G).sum(-4) / dm), 0.0)
    p = (pe + pm) / prob.dV
    return p, p.sum(axis=(-3, -2, -1)) * prob.dV
