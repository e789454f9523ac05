"""Galerkin entries of the N and K operators for PWL functions on voxels (oracle; test infrastructure only).

What is computed (Section III-B/C, Eq. 25, Eq. 32-34, Eq. 42-43):

    N^{pl,ql'}_{m,n} = < f_m^{pl}, N f_n^{ql'} >,   N u = curl curl S u,   S u = int g u,
    g(r) = exp(-i k0 |r|) / (4 pi |r|)  (Eq. 8-10, time factor exp(i omega t)),

for the PWL functions f^{pl}_n = N^l_n p-hat (Eq. 20-22) on a uniform grid.  The
entry depends on d = m - n only (Eq. 42); the oracle returns it for any list of
offsets, positive and negative, for all 144 pairs of components, with no
symmetry shortcut.

Reduction of the singular 6-D integrals (the paper reduces them to surface
integrals and defers their evaluation to external cubature codes, Section
III-C; this file uses an equivalent reduction written out here).  Because
(lap + k0^2) g = -delta (Eq. 10), inside the support

    N u = grad div S u + k0^2 S u + u,

and div S u = S (Div u), where Div u is the distributional divergence of u,
which includes the surface jump of u on the voxel faces.  Testing with f_m and
integrating by parts once more gives, for component indices alpha = (p, l),
beta = (q, l'):

    N^{alpha beta}(d) = delta_{d,0} delta_{alpha beta} G^l            (Gram, Eq. 33)
                      + k0^2 delta_{pq} S^{l l'}(d)
                      - Q^{alpha beta}(d),
    S^{l l'}(d)        = int int N^l_m(r) g(r - r') N^{l'}_n(r') dr dr',
    Q^{alpha beta}(d)  = int int (Div f_m^{alpha})(r) g(r - r') (Div f_n^{beta})(r') dr dr'.

In the voxel coordinate s in [-1/2, 1/2]^3 (r = r_n + Delta * s) the densities
N^l and Div f^{pl} = (1/Delta_p) d/ds_p [N^l P] are sums of products of
one-dimensional factors: an interval with weight 1 or s, or a point mass on a
face s_p = +-1/2.  For product densities A(s) = prod_i a_i(s_i) and
B(s') = prod_i b_i(s'_i),

    int int A(s) B(s') g(Delta (d + s - s')) ds ds' = int prod_i W_i(t_i) g(Delta (d + t)) dt,
    W_i(t) = int a_i(s) b_i(s - t) ds                       (1-D correlation),

and every W_i is, on each unit cell of the t-lattice, a polynomial of degree
<= 3 (or a point mass when both factors are points).  All breakpoints are
integers, so every integral is a sum over unit cells (or unit squares, for a
pair of parallel faces) of g times a polynomial, and the singularity u = 0
only ever sits at a cell vertex.  Those cell integrals ("moments") are done
with tensor Gauss-Legendre rules away from the origin and with the Duffy
transform (quadrature.py) on the cells that touch it.
"""

from __future__ import annotations

from math import comb

import numpy as np
from numpy.polynomial import Polynomial

from .quadrature import duffy_cube, duffy_square, gauss01

NCOMP = 12


def comp(p, l):
    """Component index alpha = 4 p + (l - 1); p in {0,1,2} = x,y,z; l in {1,2,3,4} (Eq. 19-22)."""
    return 4 * p + (l - 1)


def lin_axis(l):
    """Axis along which the scalar PWL function N^l is linear (Eq. 20); None for l = 1."""
    return None if l == 1 else l - 2


def gram(l, dV):
    """Diagonal Gram entry (Eq. 33): DV for l = 1, DV / 12 for l = 2, 3, 4."""
    return dV if l == 1 else dV / 12.0


# ---------------------------------------------------------------------------
# One-dimensional factors and their correlations
#   ("I", k)     : interval s in [-1/2, 1/2] with weight s**k, k in {0, 1}
#   ("P", sigma) : point mass at s = sigma / 2, sigma in {-1, +1}
# ---------------------------------------------------------------------------


def basis_factors(l):
    """Per-axis factors of N^l(s) P(s) (Eq. 20)."""
    return tuple(("I", 1 if lin_axis(l) == i else 0) for i in range(3))


def divergence_pieces(p, l):
    """Div of N^l p-hat in voxel coordinates: d/ds_p [N^l(s) P(s)] as a list of (coef, factors).

    Volume part: d N^l / ds_p = 1 if N^l is linear along p, else 0.
    Face parts:  N^l(s) * dP/ds_p with dP/ds_p = delta(s_p + 1/2) - delta(s_p - 1/2),
    i.e. coefficient -sigma on the face s_p = sigma/2, times the value of the
    p-factor of N^l there (sigma/2 if linear along p, else 1).
    The physical divergence is this divided by Delta_p.
    """
    pieces = []
    la = lin_axis(l)
    if la == p:
        pieces.append((1.0, (("I", 0),) * 3))
    for sigma in (-1, 1):
        value = sigma / 2.0 if la == p else 1.0
        f = [("I", 1 if la == i else 0) for i in range(3)]
        f[p] = ("P", sigma)
        pieces.append((-sigma * value, tuple(f)))
    return pieces


def _poly4(p):
    c = np.zeros(4)
    pc = np.asarray(p.coef, dtype=float)
    c[: pc.size] = pc
    if pc.size > 4 and np.any(np.abs(pc[4:]) > 0):
        raise ValueError("correlation degree exceeds 3")
    return c


def correlation_1d(fa, fb):
    """W(t) = int a(s) b(s - t) ds for two 1-D factors.

    Returns a list of pieces:
      ("cell", lo, c)  : W(t) = sum_k c[k] (t - lo)**k on t in [lo, lo + 1]
      ("point", t0, w) : W(t) = w delta(t - t0)
    """
    t = Polynomial([0.0, 1.0])
    ka, kb = fa[1], fb[1]
    if fa[0] == "I" and fb[0] == "I":
        out = []
        for lo in (-1, 0):
            # s ranges over [-1/2, 1/2] intersected with [t - 1/2, t + 1/2]
            if lo == 0:
                s_lo, s_hi = t - 0.5, Polynomial([0.5])
            else:
                s_lo, s_hi = Polynomial([-0.5]), t + 0.5
            # integrand s**ka (s - t)**kb = sum_j C(kb, j) (-t)**(kb - j) s**(ka + j)
            W = Polynomial([0.0])
            for j in range(kb + 1):
                e = ka + j + 1
                W = W + comb(kb, j) * (-t) ** (kb - j) * (s_hi**e - s_lo**e) / e
            out.append(("cell", lo, _poly4(W(Polynomial([float(lo), 1.0])))))
        return out
    if fa[0] == "P" and fb[0] == "I":
        sig = fa[1]
        # W(t) = b(sigma/2 - t) for |sigma/2 - t| <= 1/2
        lo = 0 if sig == 1 else -1
        W = (Polynomial([sig / 2.0]) - t) ** kb
        return [("cell", lo, _poly4(W(Polynomial([float(lo), 1.0]))))]
    if fa[0] == "I" and fb[0] == "P":
        sig = fb[1]
        # W(t) = a(t + sigma'/2) for |t + sigma'/2| <= 1/2
        lo = -1 if sig == 1 else 0
        W = (t + sig / 2.0) ** ka
        return [("cell", lo, _poly4(W(Polynomial([float(lo), 1.0]))))]
    # two points: W(t) = delta(t - (sigma - sigma')/2)
    return [("point", (fa[1] - fb[1]) // 2, 1.0)]


# ---------------------------------------------------------------------------
# Moments of g over unit cells of the lattice u = Delta * v, v in Z^3 + [0,1]^3
# ---------------------------------------------------------------------------

_OFF = 1 << 20
_B = 1 << 21


def _code(K):
    K = np.asarray(K, dtype=np.int64)
    return ((K[:, 0] + _OFF) * _B + (K[:, 1] + _OFF)) * _B + (K[:, 2] + _OFF)


def gauss_order(ratio):
    """Gauss-Legendre points per axis for a unit cell whose distance from the
    singular point is `ratio` cell sizes (chosen by self-convergence to ~1e-15)."""
    return np.where(ratio < 1.5, 16, np.where(ratio < 3.0, 12, np.where(ratio < 6.0, 10, 8)))


class Moments:
    """mu3[k][a,b,c] = int_{[0,1]^3} g(Delta (k + xi)) xi_x^a xi_y^b xi_z^c dxi  and
    mu2[i][(lev, kj, kk)][a,b] = int_{[0,1]^2} g(Delta v) xi_j^a xi_k^b with v_i = lev,
    v_j = kj + xi_j, v_k = kk + xi_k (j < k the two other axes)."""

    DUFFY_T = 12
    DUFFY_S = 16

    def __init__(self, delta, k0):
        self.delta = np.asarray(delta, dtype=float)
        self.k0 = float(k0)
        self.codes3 = None
        self.mu3 = None
        self.codes2 = [None, None, None]
        self.mu2 = [None, None, None]
        self._memo = {}

    def g(self, r):
        return np.exp(-1j * self.k0 * r) / (4.0 * np.pi * r)

    # -- 3-D cells ---------------------------------------------------------
    def _cells3(self, K):
        out = np.empty((len(K), 4, 4, 4), dtype=complex)
        d = self.delta
        touching = np.all((K == 0) | (K == -1), axis=1)
        dist = np.maximum(np.maximum(K, -K - 1), 0) * d
        ratio = np.sqrt((dist**2).sum(1)) / d.max()
        order = gauss_order(ratio)
        for n in np.unique(order[~touching]):
            sel = np.nonzero((order == n) & ~touching)[0]
            x, w = gauss01(int(n))
            V = x[:, None] ** np.arange(4)[None, :]
            chunk = max(1, 4_000_000 // n**3)
            for c0 in range(0, sel.size, chunk):
                s = sel[c0 : c0 + chunk]
                ux = d[0] * (K[s, 0][:, None] + x[None, :])
                uy = d[1] * (K[s, 1][:, None] + x[None, :])
                uz = d[2] * (K[s, 2][:, None] + x[None, :])
                r = np.sqrt(ux[:, :, None, None] ** 2 + uy[:, None, :, None] ** 2 + uz[:, None, None, :] ** 2)
                G = self.g(r) * (w[:, None, None] * w[None, :, None] * w[None, None, :])
                out[s] = np.einsum("cijk,ia,jb,kd->cabd", G, V, V, V, optimize=True)
        eta, wq = duffy_cube(self.DUFFY_T, self.DUFFY_S)
        for idx in np.nonzero(touching)[0]:
            k = K[idx]
            r = np.sqrt(((eta * d[None, :]) ** 2).sum(1))
            xi = np.where(k[None, :] == 0, eta, 1.0 - eta)
            G = self.g(r) * wq
            P = xi[:, :, None] ** np.arange(4)[None, None, :]
            out[idx] = np.einsum("n,na,nb,nc->abc", G, P[:, 0], P[:, 1], P[:, 2])
        return out

    def prepare3(self, K):
        K = np.unique(np.asarray(K, dtype=np.int64), axis=0)
        codes = _code(K)
        order = np.argsort(codes)
        self.codes3 = codes[order]
        self.mu3 = self._cells3(K[order])

    def shifted3(self, D, shift):
        """Moments of the cells D + shift, memoised per (D, shift)."""
        key = (D.shape, hash(D.tobytes()), shift)
        if key not in self._memo:
            self._memo[key] = self.get3(D + np.array(shift, dtype=np.int64))
        return self._memo[key]

    def shifted2(self, D, axis, shift):
        """Moments of the faces (D_axis + shift[0], D_j + shift[1], D_k + shift[2])."""
        key = (D.shape, hash(D.tobytes()), axis, shift)
        if key not in self._memo:
            j, k = [a for a in range(3) if a != axis]
            F = np.stack([D[:, axis] + shift[0], D[:, j] + shift[1], D[:, k] + shift[2]], axis=1)
            self._memo[key] = self.get2(axis, F)
        return self._memo[key]

    def get3(self, K):
        c = _code(K)
        i = np.searchsorted(self.codes3, c)
        if np.any(i >= self.codes3.size) or np.any(self.codes3[np.minimum(i, self.codes3.size - 1)] != c):
            raise KeyError("3-D cell moment not prepared")
        return self.mu3[i]

    # -- 2-D faces -------------------------------------------------------------
    def _faces2(self, axis, F):
        """F rows are (lev, kj, kk)."""
        j, k = [a for a in range(3) if a != axis]
        d = self.delta
        out = np.empty((len(F), 4, 4), dtype=complex)
        touching = (F[:, 0] == 0) & np.all((F[:, 1:] == 0) | (F[:, 1:] == -1), axis=1)
        dj = np.maximum(np.maximum(F[:, 1], -F[:, 1] - 1), 0) * d[j]
        dk = np.maximum(np.maximum(F[:, 2], -F[:, 2] - 1), 0) * d[k]
        ratio = np.sqrt((F[:, 0] * d[axis]) ** 2 + dj**2 + dk**2) / d.max()
        order = gauss_order(ratio)
        for n in np.unique(order[~touching]):
            sel = np.nonzero((order == n) & ~touching)[0]
            x, w = gauss01(int(n))
            V = x[:, None] ** np.arange(4)[None, :]
            ui = d[axis] * F[sel, 0].astype(float)
            uj = d[j] * (F[sel, 1][:, None] + x[None, :])
            uk = d[k] * (F[sel, 2][:, None] + x[None, :])
            r = np.sqrt(ui[:, None, None] ** 2 + uj[:, :, None] ** 2 + uk[:, None, :] ** 2)
            G = self.g(r) * (w[:, None] * w[None, :])
            out[sel] = np.einsum("cij,ia,jb->cab", G, V, V, optimize=True)
        eta, wq = duffy_square(self.DUFFY_T, self.DUFFY_S)
        dd = np.array([d[j], d[k]])
        for idx in np.nonzero(touching)[0]:
            kk = F[idx, 1:]
            r = np.sqrt(((eta * dd[None, :]) ** 2).sum(1))
            xi = np.where(kk[None, :] == 0, eta, 1.0 - eta)
            G = self.g(r) * wq
            P = xi[:, :, None] ** np.arange(4)[None, None, :]
            out[idx] = np.einsum("n,na,nb->ab", G, P[:, 0], P[:, 1])
        return out

    def prepare2(self, axis, F):
        F = np.unique(np.asarray(F, dtype=np.int64), axis=0)
        codes = _code(F)
        order = np.argsort(codes)
        self.codes2[axis] = codes[order]
        self.mu2[axis] = self._faces2(axis, F[order])

    def get2(self, axis, F):
        c = _code(F)
        tab = self.codes2[axis]
        i = np.searchsorted(tab, c)
        if np.any(i >= tab.size) or np.any(tab[np.minimum(i, tab.size - 1)] != c):
            raise KeyError("2-D face moment not prepared")
        return self.mu2[axis][i]


def prepare_moments(delta, k0, D):
    """Moments of every lattice cell and face needed by the offsets D (n, 3) = (dx, dy, dz)."""
    D = np.asarray(D, dtype=np.int64)
    mom = Moments(delta, k0)
    sig = np.array([[a, b, c] for a in (-1, 0) for b in (-1, 0) for c in (-1, 0)])
    mom.prepare3((D[:, None, :] + sig[None, :, :]).reshape(-1, 3))
    for axis in range(3):
        j, k = [a for a in range(3) if a != axis]
        rows = []
        for t0 in (-1, 0, 1):
            for a in (-1, 0):
                for b in (-1, 0):
                    rows.append(np.stack([D[:, axis] + t0, D[:, j] + a, D[:, k] + b], axis=1))
        mom.prepare2(axis, np.concatenate(rows))
    return mom


def pair_integral(fa, fb, D, mom):
    """I(d) = int prod_i W_i(t_i) g(Delta (d + t)) dt for product densities with factors fa, fb."""
    D = np.asarray(D, dtype=np.int64)
    per_axis = [correlation_1d(fa[i], fb[i]) for i in range(3)]
    points = [i for i in range(3) if per_axis[i][0][0] == "point"]
    val = np.zeros(len(D), dtype=complex)
    if not points:
        for px in per_axis[0]:
            for py in per_axis[1]:
                for pz in per_axis[2]:
                    mu = mom.shifted3(D, (px[1], py[1], pz[1]))
                    w = np.einsum("a,b,c->abc", px[2], py[2], pz[2]).ravel()
                    val += mu.reshape(len(D), 64) @ w
        return val
    if len(points) > 1:
        raise ValueError("two point axes cannot occur")
    axis = points[0]
    j, k = [a for a in range(3) if a != axis]
    t0, w = per_axis[axis][0][1], per_axis[axis][0][2]
    for pj in per_axis[j]:
        for pk in per_axis[k]:
            mu = mom.shifted2(D, axis, (t0, pj[1], pk[1]))
            val += w * (mu.reshape(len(D), 16) @ np.outer(pj[2], pk[2]).ravel())
    return val


def n_entries(delta, k0, D, mom=None):
    """All 144 Galerkin entries N^{alpha beta}(d) for offsets D (n, 3) = (dx, dy, dz) in voxels.

    Returns complex array (12, 12, n).  Includes the Gram term at d = 0.
    """
    D = np.asarray(D, dtype=np.int64).reshape(-1, 3)
    delta = np.asarray(delta, dtype=float)
    if mom is None:
        mom = prepare_moments(delta, k0, D)
    dV = float(np.prod(delta))
    cache = {}

    def I(fa, fb):
        key = (fa, fb)
        if key not in cache:
            cache[key] = pair_integral(fa, fb, D, mom)
        return cache[key]

    zero = np.all(D == 0, axis=1).astype(float)
    T = np.zeros((NCOMP, NCOMP, len(D)), dtype=complex)
    for p in range(3):
        for l in range(1, 5):
            a = comp(p, l)
            for q in range(3):
                for lp in range(1, 5):
                    b = comp(q, lp)
                    v = np.zeros(len(D), dtype=complex)
                    if p == q:
                        v += k0 * k0 * dV * dV * I(basis_factors(l), basis_factors(lp))
                    Qv = np.zeros(len(D), dtype=complex)
                    for ca, fa in divergence_pieces(p, l):
                        for cb, fb in divergence_pieces(q, lp):
                            Qv += ca * cb * I(fa, fb)
                    v -= dV * dV / (delta[p] * delta[q]) * Qv
                    if a == b:
                        v += zero * gram(l, dV)
                    T[a, b] = v
    return T


def s_entries(delta, k0, D, mom=None):
    """The 16 volume integrals S^{l l'}(d) (in m^5), returned as complex array (4, 4, n)."""
    D = np.asarray(D, dtype=np.int64).reshape(-1, 3)
    delta = np.asarray(delta, dtype=float)
    if mom is None:
        mom = prepare_moments(delta, k0, D)
    dV = float(np.prod(delta))
    S = np.zeros((4, 4, len(D)), dtype=complex)
    for l in range(1, 5):
        for lp in range(1, 5):
            S[l - 1, lp - 1] = dV * dV * pair_integral(basis_factors(l), basis_factors(lp), D, mom)
    return S


def q_entries(delta, k0, D, mom=None):
    """Q^{alpha beta}(d) (in m^3), complex array (12, 12, n)."""
    D = np.asarray(D, dtype=np.int64).reshape(-1, 3)
    delta = np.asarray(delta, dtype=float)
    if mom is None:
        mom = prepare_moments(delta, k0, D)
    dV = float(np.prod(delta))
    Q = np.zeros((NCOMP, NCOMP, len(D)), dtype=complex)
    for p in range(3):
        for l in range(1, 5):
            for q in range(3):
                for lp in range(1, 5):
                    v = np.zeros(len(D), dtype=complex)
                    for ca, fa in divergence_pieces(p, l):
                        for cb, fb in divergence_pieces(q, lp):
                            v += ca * cb * pair_integral(fa, fb, D, mom)
                    Q[comp(p, l), comp(q, lp)] = dV * dV / (delta[p] * delta[q]) * v
    return Q


# ---------------------------------------------------------------------------
# K operator (Eq. 8: K u = curl S u), for the magnetic field h = h_inc + K j (Section II total fields)
# ---------------------------------------------------------------------------

LEVI_CIVITA = np.zeros((3, 3, 3))
for _i, _j, _k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
    LEVI_CIVITA[_i, _j, _k] = 1.0
    LEVI_CIVITA[_i, _k, _j] = -1.0


def k_entries(delta, k0, D, mom=None):
    """All 144 Galerkin entries K^{alpha beta}(d) = < f_m^{pl}, K f_n^{ql'} > (Eq. 25) for offsets
    D (n, 3) = (dx, dy, dz) in voxels; complex array (12, 12, n).

    (K u)_p = (curl S u)_p = sum_{j,q} eps_{pjq} d_j S u_q, so with d_j acting on g(r - r'),

        K^{(p,l),(q,l')}(d) = sum_j eps_{pjq} int int N^l_m(r) d_j g(r - r') N^{l'}_n(r') dr dr'
                            = - sum_j eps_{pjq} int int (D_j N^l_m)(r) g(r - r') N^{l'}_n(r') dr dr',

    integrating by parts in r over the testing function's support: D_j N^l is its distributional
    derivative (the volume part and the point masses of its jumps on the faces s_j = +-1/2),
    i.e. divergence_pieces(j, l) / Delta_j.  The kernel d_j g is only weakly singular; after this
    step every term is g times polynomials, evaluated by the same cell moments as N.
    """
    D = np.asarray(D, dtype=np.int64).reshape(-1, 3)
    delta = np.asarray(delta, dtype=float)
    if mom is None:
        mom = prepare_moments(delta, k0, D)
    dV = float(np.prod(delta))
    # P[j][l][l'] = int int (D_j N^l) g N^{l'} (physical units)
    P = np.zeros((3, 4, 4, len(D)), dtype=complex)
    for j in range(3):
        for l in range(1, 5):
            for lp in range(1, 5):
                v = np.zeros(len(D), dtype=complex)
                for c, fa in divergence_pieces(j, l):
                    v += c * pair_integral(fa, basis_factors(lp), D, mom)
                P[j, l - 1, lp - 1] = dV * dV / delta[j] * v
    T = np.zeros((NCOMP, NCOMP, len(D)), dtype=complex)
    for p in range(3):
        for q in range(3):
            for j in range(3):
                e = LEVI_CIVITA[p, j, q]
                if e == 0.0:
                    continue
                for l in range(1, 5):
                    for lp in range(1, 5):
                        T[comp(p, l), comp(q, lp)] -= e * P[j, l - 1, lp - 1]
    return T


def all_offsets(nx, ny, nz):
    """Every offset d in (-N, N)^3 as an (n, 3) array (dx, dy, dz), dz slowest."""
    dz, dy, dx = np.meshgrid(
        np.arange(-nz + 1, nz), np.arange(-ny + 1, ny), np.arange(-nx + 1, nx), indexing="ij"
    )
    return np.stack([dx.ravel(), dy.ravel(), dz.ravel()], axis=1)


def toeplitz_tensors(grid, k0):
    """Toeplitz defining tensors (Eq. 43) for every offset: complex (12, 12, 2Nz-1, 2Ny-1, 2Nx-1),
    offset d stored at index d + N - 1 along each axis (z, y, x order)."""
    D = all_offsets(grid.nx, grid.ny, grid.nz)
    T = n_entries((grid.dx, grid.dy, grid.dz), k0, D)
    return T.reshape(NCOMP, NCOMP, 2 * grid.nz - 1, 2 * grid.ny - 1, 2 * grid.nx - 1)


def k_toeplitz_tensors(grid, k0):
    """Toeplitz defining tensors of K for every offset, laid out as toeplitz_tensors."""
    D = all_offsets(grid.nx, grid.ny, grid.nz)
    T = k_entries((grid.dx, grid.dy, grid.dz), k0, D)
    return T.reshape(NCOMP, NCOMP, 2 * grid.nz - 1, 2 * grid.ny - 1, 2 * grid.nx - 1)
