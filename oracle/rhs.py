"""Tested incident fields and right-hand side (oracle; test infrastructure only).

  e_inc^{pl}(m) = int_{V_m} N^l_m(r) e_inc^p(r) dV                     (Eq. 27, Eq. 30)
  b^{pl}(m)     = c_e chi(m) e_inc^{pl}(m)                            (Eq. 31)

Sources:
  * plane wave e_inc = pol exp(-i k0 dir . r) (Section V-A uses x-pol along z);
    the voxel integrals are separable and done in closed form;
  * Hertzian dipole with current moment p = I l (A m) at r0: the field of the
    point current j = p delta(r - r0) through Eq. 13 with N - I = grad div S + k0^2 S,
    e_inc(r) = (1/c_e) (k0^2 g(R) p + grad (p . grad g)(R)),  R = r - r0,
    tested with an n^3 Gauss-Legendre rule per voxel (n = 6).
"""

from __future__ import annotations

import math

import numpy as np

from .green import NCOMP, lin_axis
from .quadrature import gauss01


def _f0(k):
    """int_{-1/2}^{1/2} exp(-i k s) ds."""
    k = np.asarray(k, dtype=float)
    small = np.abs(k) < 1e-4
    ks = np.where(small, 1.0, k)
    exact = 2.0 * np.sin(ks / 2.0) / ks
    series = 1.0 - k * k / 24.0 + k**4 / 1920.0
    return np.where(small, series, exact).astype(complex)


def _f1(k):
    """int_{-1/2}^{1/2} s exp(-i k s) ds = i d/dk _f0(k).

    The closed form i (cos(k/2)/k - 2 sin(k/2)/k^2) cancels for small k; below
    |k| = 1/4 the Taylor series sum_{n odd} (-i k)^n 2^-(n+1) / (n! (n+2)) is used
    (terms to k^9; the first omitted term is below 1e-17 relative there)."""
    k = np.asarray(k, dtype=float)
    small = np.abs(k) < 0.25
    ks = np.where(small, 1.0, k)
    exact = 1j * (np.cos(ks / 2.0) / ks - 2.0 * np.sin(ks / 2.0) / ks**2)
    series = np.zeros_like(k, dtype=complex)
    for n in (1, 3, 5, 7, 9):
        series = series + (-1j * k) ** n * 0.5 ** (n + 1) / (math.factorial(n) * (n + 2))
    return np.where(small, series, exact)


def planewave_tested(grid, k0, pol=(1.0, 0.0, 0.0), direction=(0.0, 0.0, 1.0)):
    """Tested plane-wave field (12, Nz, Ny, Nx) in closed form."""
    pol = np.asarray(pol, dtype=float)
    kv = k0 * np.asarray(direction, dtype=float)
    xx, yy, zz = grid.centres()
    delta = np.array([grid.dx, grid.dy, grid.dz])
    phase = np.exp(-1j * (kv[0] * xx + kv[1] * yy + kv[2] * zz))
    dV = float(np.prod(delta))
    kappa = kv * delta
    out = np.zeros((NCOMP,) + grid.shape, dtype=complex)
    for p in range(3):
        for l in range(1, 5):
            fac = 1.0 + 0j
            for i in range(3):
                fac *= _f1(kappa[i]) if lin_axis(l) == i else _f0(kappa[i])
            out[4 * p + l - 1] = pol[p] * dV * fac * phase
    return out


def dipole_field(r, r0, moment, k0, ce):
    """Incident E field (..., 3) at points r (..., 3) of a Hertzian dipole p = moment (A m) at r0."""
    R = r - np.asarray(r0, dtype=float)
    Rn = np.sqrt((R**2).sum(-1))
    Rh = R / Rn[..., None]
    g = np.exp(-1j * k0 * Rn) / (4.0 * np.pi * Rn)
    p = np.asarray(moment, dtype=float)
    pr = (Rh * p).sum(-1)
    # grad grad g = g [ (-1/R^2 - i k/R) I + (3/R^2 + 3 i k/R - k^2) R^ R^ ]
    a = g * (-1.0 / Rn**2 - 1j * k0 / Rn)
    c = g * (3.0 / Rn**2 + 3j * k0 / Rn - k0 * k0)
    E = (k0 * k0 * g)[..., None] * p + a[..., None] * p + (c * pr)[..., None] * Rh
    return E / ce


def dipole_hfield(r, r0, moment, k0):
    """Incident H field (..., 3) at points r of a Hertzian dipole p = moment (A m) at r0:
    h = K (p delta_r0) = curl (g p) = grad g x p (Eq. 8), grad g = g (-1/R - i k0) R^."""
    R = r - np.asarray(r0, dtype=float)
    Rn = np.sqrt((R**2).sum(-1))
    Rh = R / Rn[..., None]
    g = np.exp(-1j * k0 * Rn) / (4.0 * np.pi * Rn)
    grad = (g * (-1.0 / Rn - 1j * k0))[..., None] * Rh
    return np.cross(grad, np.broadcast_to(np.asarray(moment, dtype=float), grad.shape))


def tested_field_quadrature(grid, field, n=6):
    """Tested field of an arbitrary callable field(r (..., 3)) -> (..., 3) with n^3 Gauss points per voxel."""
    x, w = gauss01(n)
    s = x - 0.5
    xx, yy, zz = grid.centres()
    delta = np.array([grid.dx, grid.dy, grid.dz])
    dV = float(np.prod(delta))
    out = np.zeros((NCOMP,) + grid.shape, dtype=complex)
    for i in range(n):
        for j in range(n):
            for k in range(n):
                sv = np.array([s[i], s[j], s[k]])
                r = np.stack([xx + delta[0] * sv[0], yy + delta[1] * sv[1], zz + delta[2] * sv[2]], axis=-1)
                E = field(r)
                wt = w[i] * w[j] * w[k] * dV
                for p in range(3):
                    for l in range(1, 5):
                        la = lin_axis(l)
                        phi = 1.0 if la is None else sv[la]
                        out[4 * p + l - 1] += wt * phi * E[..., p]
    return out


def dipoles_tested(grid, k0, ce, positions, moments, n=6):
    """Tested fields of R dipoles: (R, 12, Nz, Ny, Nx)."""
    out = []
    for r0, mom in zip(positions, moments):
        out.append(tested_field_quadrature(grid, lambda r: dipole_field(r, r0, mom, k0, ce), n))
    return np.array(out)


def dipoles_tested_h(grid, k0, positions, moments, n=6):
    """Tested incident magnetic fields of R dipoles: (R, 12, Nz, Ny, Nx)."""
    out = []
    for r0, mom in zip(positions, moments):
        out.append(tested_field_quadrature(grid, lambda r: dipole_hfield(r, r0, mom, k0), n))
    return np.array(out)


def rhs(prob, e_tested):
    """b = c_e M_chi e_inc (Eq. 31); e_tested (..., 12, Nz, Ny, Nx)."""
    return prob.ce * prob.chi * e_tested
