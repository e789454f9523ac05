"""Fields, absorbed power and magnetic quantities from the solution (oracle; test infrastructure only).

Section IV-C: the tested total field follows from the discrete analogue of
e_tot = e_inc + (1/c_e)(N - I) j (Section II, total fields),

    e~ = e_inc_tested + (1/c_e) (N x - G x),

and the PWL field coefficients are e~ divided by the (diagonal) Gram matrix.
Absorbed power (Eq. 44):  P_abs = 1/2 Re{ x^* (c_e M_chi)^-1 G x },  split per
voxel into the absorbed-power density p_abs(m) = (1/2 Re{...}_m) / DV (W/m^3),
zero in air (chi = 0).

Magnetic field (Section II total fields, h_tot = h_inc + K j): the tested field is
h~ = h_inc_tested + K x and its PWL coefficients h~ / G.  The transmit field
b1+ = mu0 (h_x + i h_y) (Section V-D) is taken from the voxel-average (l = 1)
coefficients, and the magnetic energy W_m = 1/4 int mu |h|^2 dV (Section V-D,
mu = mu0 in tissue) over the scatterer (chi != 0) is exact for the PWL field
because the four scalar functions of a voxel are orthogonal:
int |sum_l h_l N^l|^2 = sum_l G^l |h_l|^2.
"""

from __future__ import annotations

import numpy as np

from . import MU0


def fields(prob, Nop, x, e_tested):
    """PWL field coefficients e (..., 12, Nz, Ny, Nx)."""
    G = prob.gram_vector()[:, None, None, None]
    et = e_tested + (Nop.apply(x) - G * x) / prob.ce
    return et / G


def absorbed_power(prob, x):
    """(p_abs (..., Nz, Ny, Nx) in W/m^3, P_abs (...) in W) from the current coefficients x."""
    G = prob.gram_vector()[:, None, None, None]
    chi = prob.chi
    tissue = chi != 0
    denom = np.where(tissue, prob.ce * chi, 1.0)
    q = (np.abs(x) ** 2 * G).sum(-4)
    p = np.where(tissue, 0.5 * np.real(q / denom), 0.0) / prob.dV
    return p, p.sum(axis=(-3, -2, -1)) * prob.dV


def magnetic_fields(prob, Kop, x, h_tested):
    """PWL magnetic-field coefficients h (..., 12, Nz, Ny, Nx) from the current coefficients x."""
    G = prob.gram_vector()[:, None, None, None]
    return (h_tested + Kop.apply(x)) / G


def b1_plus(h):
    """b1+ = mu0 (h_x + i h_y) per voxel from the l = 1 coefficients (components 0 and 4)."""
    return MU0 * (h[..., 0, :, :, :] + 1j * h[..., 4, :, :, :])


def magnetic_energy(prob, h):
    """(w_m (..., Nz, Ny, Nx) voxel-average density in J/m^3, W_m (...) in J) over the scatterer."""
    G = prob.gram_vector()[:, None, None, None]
    tissue = prob.chi != 0
    e = 0.25 * MU0 * (np.abs(h) ** 2 * G).sum(-4)  # J per voxel
    w = np.where(tissue, e / prob.dV, 0.0)
    return w, w.sum(axis=(-3, -2, -1)) * prob.dV
