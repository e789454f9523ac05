"""Quadrature rules on the unit interval, square and cube (oracle; test infrastructure only).

* `gauss01(n)`: n-point Gauss-Legendre rule mapped to [0, 1].
* `duffy_cube(nt, ns)`: rule for integrals over [0,1]^3 of functions with an
  integrable 1/|eta| point singularity at the vertex eta = 0.  The cube is cut
  into three pyramids with apex at the vertex, each mapped to the unit cube by
  the Duffy transform (M. G. Duffy, SIAM J. Numer. Anal. 19 (1982) 1260):
  eta = tau * (e_m + zeta_1 e_j + zeta_2 e_k), Jacobian tau^2, which cancels the
  1/|eta| singularity; tensor Gauss-Legendre is then used in (tau, zeta).
* `duffy_square(nt, ns)`: the 2-D analogue (two triangles, Jacobian tau).
"""

from functools import lru_cache

import numpy as np
from numpy.polynomial.legendre import leggauss


@lru_cache(maxsize=None)
def gauss01(n):
    x, w = leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


@lru_cache(maxsize=None)
def duffy_cube(nt, ns):
    """Nodes eta (M, 3) in [0,1]^3 and weights (M,) for a vertex singularity at 0."""
    t, wt = gauss01(nt)
    s, ws = gauss01(ns)
    T, S1, S2 = np.meshgrid(t, s, s, indexing="ij")
    W = (wt[:, None, None] * ws[None, :, None] * ws[None, None, :]) * T * T
    T, S1, S2, W = T.ravel(), S1.ravel(), S2.ravel(), W.ravel()
    nodes, weights = [], []
    for m in range(3):
        eta = np.empty((T.size, 3))
        others = [a for a in range(3) if a != m]
        eta[:, m] = T
        eta[:, others[0]] = T * S1
        eta[:, others[1]] = T * S2
        nodes.append(eta)
        weights.append(W)
    return np.concatenate(nodes), np.concatenate(weights)


@lru_cache(maxsize=None)
def duffy_square(nt, ns):
    """Nodes eta (M, 2) in [0,1]^2 and weights (M,) for a vertex singularity at 0."""
    t, wt = gauss01(nt)
    s, ws = gauss01(ns)
    T, S = np.meshgrid(t, s, indexing="ij")
    W = (wt[:, None] * ws[None, :]) * T
    T, S, W = T.ravel(), S.ravel(), W.ravel()
    nodes, weights = [], []
    for m in range(2):
        eta = np.empty((T.size, 2))
        eta[:, m] = T
        eta[:, 1 - m] = T * S
        nodes.append(eta)
        weights.append(W)
    return np.concatenate(nodes), np.concatenate(weights)
