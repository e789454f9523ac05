"""Pin of the oracle's Galerkin entries of N at touching voxels (|d|_inf = 1), all 144 entries,
by a route that shares nothing with the oracle's reduction.

The oracle integrates by parts onto the PWL functions (their divergence with face jumps) and
evaluates volume/face moments of g.  Here the entry is taken from its plain definition instead:
for voxels that do not overlap, the Galerkin entry (Eq. 25 with N u = grad div S u + k0^2 S u
off the support, Eq. 8-10) is the absolutely convergent 6-D integral

    N^{(p,l),(q,l')}(d) = int_{V_m} int_{V_n} N^l(r) [k0^2 g delta_pq + d_p d_q g](r - r') N^l'(r') dr dr',

with the pointwise dyadic kernel and no reduction.  Its integrand is singular only where the
voxels touch.  Written in the difference variable u = r - r' it becomes a 3-D integral
prod_i Delta_i^2 int c(t) K((d + t) Delta) dt over t in [-1, 1]^3, where c is the product over
the axes of the 1-D cross-correlations of the two voxels' basis factors (piecewise polynomial,
evaluated here by exact Gauss quadrature).  The kernel's singular point t = -d is a vertex of
the sub-boxes that touch it, and there c vanishes at least linearly, so the Duffy transform
(three pyramids per cube, Duffy 1982) leaves a smooth integrand and Gauss-Legendre converges fast;
the other sub-boxes take plain tensor Gauss.  Self-convergence (order n vs n + 8) is checked too.
"""

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from oracle import green as OG

DELTA = np.array([0.004, 0.005, 0.0045])
K0 = 2 * np.pi * 298e6 / 299792458.0


def _gl(n, a, b):
    x, w = leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def _corr(t, lin_a, lin_b):
    """c(t) = int a(s) b(s - t) ds over the overlap of [-1/2, 1/2] and [t - 1/2, t + 1/2];
    a(s) = s if lin_a else 1, b likewise (the degree-2 integrand is exact with 3 points)."""
    lo = np.maximum(-0.5, t - 0.5)
    hi = np.minimum(0.5, t + 0.5)
    x, w = leggauss(3)
    s = 0.5 * (hi + lo)[..., None] + 0.5 * (hi - lo)[..., None] * x
    a = s if lin_a else 1.0
    b = (s - t[..., None]) if lin_b else 1.0
    return 0.5 * (hi - lo) * np.sum(w * a * b, axis=-1)


def _points(d, n):
    """Quadrature points t (m, 3) and weights over [-1, 1]^3, split at t_i = 0, Duffy at t = -d."""
    sing = -np.asarray(d, dtype=float)
    pts, wts = [], []
    for box in np.ndindex(2, 2, 2):
        lo = np.array([-1.0 if b == 0 else 0.0 for b in box])
        hi = lo + 1.0
        corners = [np.where(np.array(c) == 0, lo, hi) for c in np.ndindex(2, 2, 2)]
        vtx = [c for c in corners if np.allclose(c, sing)]
        if not vtx:
            xs = [_gl(n, lo[i], hi[i]) for i in range(3)]
            T = np.stack(np.meshgrid(xs[0][0], xs[1][0], xs[2][0], indexing="ij"), -1).reshape(-1, 3)
            W = (xs[0][1][:, None, None] * xs[1][1][None, :, None] * xs[2][1][None, None, :]).ravel()
            pts.append(T)
            wts.append(W)
            continue
        v = vtx[0]
        direction = np.where(np.isclose(v, lo), 1.0, -1.0)  # from the singular vertex into the box
        tau, wt = _gl(n, 0.0, 1.0)
        s, ws = _gl(n, 0.0, 1.0)
        TT, A, B = np.meshgrid(tau, s, s, indexing="ij")
        Wd = (wt[:, None, None] * ws[None, :, None] * ws[None, None, :]) * TT ** 2  # Jacobian tau^2
        for k in range(3):  # pyramid where local coordinate k is the largest
            xi = np.empty(TT.shape + (3,))
            others = [j for j in range(3) if j != k]
            xi[..., k] = TT
            xi[..., others[0]] = TT * A
            xi[..., others[1]] = TT * B
            pts.append((v + direction * xi).reshape(-1, 3))
            wts.append(Wd.ravel())
    return np.concatenate(pts), np.concatenate(wts)


def _entries(d, n):
    """All 144 entries at offset d (voxels) from the unreduced dyadic kernel, shape (12, 12)."""
    t, w = _points(d, n)
    u = (np.asarray(d)[None, :] + t) * DELTA
    R = np.sqrt((u ** 2).sum(-1))
    uh = u / R[:, None]
    g = np.exp(-1j * K0 * R) / (4 * np.pi * R)
    radial = g * (3 / R ** 2 + 3j * K0 / R - K0 ** 2)  # d_p d_q g = radial uh_p uh_q + iso delta_pq
    iso = -g * (1 / R ** 2 + 1j * K0 / R)
    K = radial[:, None, None] * uh[:, :, None] * uh[:, None, :]
    for p in range(3):
        K[:, p, p] += iso + K0 ** 2 * g
    C = [[[_corr(t[:, i], fa, fb) for fb in (0, 1)] for fa in (0, 1)] for i in range(3)]
    scale = np.prod(DELTA ** 2)
    out = np.zeros((12, 12), dtype=complex)
    for la in range(1, 5):
        for lb in range(1, 5):
            c = np.ones(len(w))
            for i in range(3):
                c = c * C[i][int(la == i + 2)][int(lb == i + 2)]
            M = scale * np.einsum("m,mpq->pq", w * c, K)
            for p in range(3):
                for q in range(3):
                    out[4 * p + la - 1, 4 * q + lb - 1] = M[p, q]
    return out


ADJACENT = [(1, 0, 0), (0, -1, 0), (0, 0, 1), (1, 1, 0), (-1, 0, 1), (0, 1, -1), (1, 1, 1), (-1, 1, -1)]


def test_correlation_weights_brute_force():
    """The 1-D cross-correlations against a fine midpoint rule of their definition."""
    t = np.linspace(-1, 1, 9)
    s = (np.arange(20000) + 0.5) / 20000 - 0.5
    for fa in (0, 1):
        for fb in (0, 1):
            ref = []
            for tt in t:
                sb = s - tt
                m = np.abs(sb) <= 0.5
                ref.append(np.sum(((s if fa else 1.0) * (sb if fb else 1.0) * m)) / s.size)
            assert np.max(np.abs(_corr(t, fa, fb) - np.array(ref))) < 1e-6


def test_adjacent_reference_self_convergence():
    a = _entries((1, 1, 0), 14)
    b = _entries((1, 1, 0), 22)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("d", ADJACENT)
def test_adjacent_entries_vs_unreduced_kernel(d):
    """All 144 oracle entries at a touching offset vs the unreduced dyadic kernel: the p != q
    blocks the trace identity does not constrain, and the p = q ones."""
    ref = _entries(d, 22)
    got = OG.n_entries(DELTA, K0, np.array([d]))[:, :, 0]
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) < 1e-12 * scale
    # the off-diagonal component blocks (p != q) on their own scale
    off = np.array([[a // 4 != b // 4 for b in range(12)] for a in range(12)])
    s_off = np.max(np.abs(ref[off]))
    assert s_off > 0 and np.max(np.abs((got - ref)[off])) < 1e-11 * s_off
