"""Mie series: power absorbed by a homogeneous lossy sphere in a plane wave (oracle; test infrastructure only).

Section V-A compares the absorbed power of the PWL solver with the Mie series.
This module computes it from the published method of Bohren & Huffman,
"Absorption and Scattering of Light by Small Particles" (1983), Section 4.4
and Appendix A: Riccati-Bessel functions psi_n, xi_n of the size parameter
x = k0 a by upward recurrence, the logarithmic derivative D_n(m x) by downward
recurrence, the coefficients a_n, b_n, and

    C_ext = (2 pi / k0^2) sum (2n+1) Re(a_n + b_n),
    C_sca = (2 pi / k0^2) sum (2n+1) (|a_n|^2 + |b_n|^2),
    P_abs = (C_ext - C_sca) |E0|^2 / (2 eta0).

Bohren & Huffman use the time factor exp(-i omega t); the paper uses
exp(+i omega t) with eps = eps' - i eps''.  The refractive index is therefore
m = sqrt(conj(eps)) (positive imaginary part for a lossy sphere).

A magnetic sphere (relative permeability mu = mu' - i mu'', for the JM-VIE of Eq. 14-15)
takes Bohren & Huffman's coefficients for a sphere whose permeability differs from the
medium's (their Eq. 4.53, medium mu = 1): m = sqrt(conj(eps) conj(mu)), and the logarithmic
derivative enters a_n as mu D_n / m and b_n as m D_n / mu (with conj(mu) for the time factor).
"""

from __future__ import annotations

import numpy as np

from . import C0, EPS0, MU0


def mie_coefficients(m, x, mu=1.0):
    """a_n, b_n for relative refractive index m, size parameter x and relative permeability
    mu of the sphere (Bohren & Huffman's convention; mu = 1 for a non-magnetic sphere)."""
    nstop = int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    mx = m * x
    nmx = int(max(nstop, abs(mx))) + 16
    D = np.zeros(nmx + 1, dtype=complex)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    psi_m1, psi_0 = np.cos(x), np.sin(x)
    chi_m1, chi_0 = -np.sin(x), np.cos(x)
    xi_m1 = psi_m1 - 1j * chi_m1
    xi_0 = psi_0 - 1j * chi_0
    a, b = [], []
    for n in range(1, nstop + 1):
        psi = (2.0 * n - 1.0) / x * psi_0 - psi_m1
        chi = (2.0 * n - 1.0) / x * chi_0 - chi_m1
        xi = psi - 1j * chi
        ta = mu * D[n] / m + n / x
        tb = D[n] * m / mu + n / x
        a.append((ta * psi - psi_0) / (ta * xi - xi_0))
        b.append((tb * psi - psi_0) / (tb * xi - xi_0))
        psi_m1, psi_0 = psi_0, psi
        chi_m1, chi_0 = chi_0, chi
        xi_m1, xi_0 = xi_0, xi
    return np.array(a), np.array(b)


def cross_sections(eps, radius, freq, mu=1.0):
    """(C_ext, C_sca, C_abs) in m^2 for relative permittivity eps and permeability mu
    (exp(+i omega t) convention)."""
    k0 = 2.0 * np.pi * freq / C0
    mub = np.conj(complex(mu))
    m = np.sqrt(np.conj(complex(eps)) * mub)
    x = k0 * radius
    a, b = mie_coefficients(m, x, mub)
    n = np.arange(1, a.size + 1)
    cext = 2.0 * np.pi / k0**2 * np.sum((2 * n + 1) * np.real(a + b))
    csca = 2.0 * np.pi / k0**2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return cext, csca, cext - csca


def absorbed_power(eps_real, sigma, radius, freq, e0=1.0, mu=1.0):
    """Absorbed power (W) of a sphere in a plane wave of amplitude e0 (V/m); mu = mu' - i mu''."""
    omega = 2.0 * np.pi * freq
    eps = eps_real - 1j * sigma / (omega * EPS0)
    eta0 = np.sqrt(MU0 / EPS0)
    return cross_sections(eps, radius, freq, mu)[2] * abs(e0) ** 2 / (2.0 * eta0)
