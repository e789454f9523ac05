"""Fields and absorbed power from the solution (oracle; test infrastructure only).

Section IV-C: the tested total field follows from the discrete analogue of
e_tot = e_inc + (1/c_e)(N - I) j (Eq. tot_fields),

    e~ = e_inc_tested + (1/c_e) (N x - G x),

and the PWL field coefficients are e~ divided by the (diagonal) Gram matrix.
Absorbed power (Eq. 44):  P_abs = 1/2 Re{ x^* (c_e M_chi)^-1 G x },  split per
voxel into the absorbed-power density p_abs(m) = (1/2 Re{...}_m) / DV (W/m^3),
zero in air (chi = 0).
"""

from __future__ import annotations

import numpy as np


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
