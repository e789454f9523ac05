"""Pins of the oracle's Galerkin entries of N against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks it against an
independent route (closed forms, a different quadrature of the unreduced
kernel, exact identities of the operator, brute-force integration).
"""

import json
import os

import numpy as np
import pytest

from oracle import green as G
from oracle.quadrature import gauss01

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _lin(l):
    return None if l == 1 else l - 2


def test_gram_closed_form():
    """Eq. 33: G = DV (l = 1), DV/12 (l = 2,3,4); checked against Gauss integration of (N^l)^2."""
    delta = np.array([0.003, 0.004, 0.005])
    dV = np.prod(delta)
    x, w = gauss01(4)
    s = x - 0.5
    for l in range(1, 5):
        la = _lin(l)
        val = dV * sum(w[i] * w[j] * w[k] * ((1.0 if la is None else (s[i], s[j], s[k])[la]) ** 2)
                       for i in range(4) for j in range(4) for k in range(4))
        assert abs(G.gram(l, dV) - val) < 1e-15 * dV
    assert G.gram(1, 1.0) == GOLD["gram"]["l1"]
    assert abs(G.gram(2, 1.0) - GOLD["gram"]["l234"]) < 1e-16


@pytest.mark.parametrize("fa,fb", [
    (("I", 0), ("I", 0)), (("I", 1), ("I", 0)), (("I", 0), ("I", 1)), (("I", 1), ("I", 1)),
    (("P", 1), ("I", 0)), (("P", -1), ("I", 1)), (("I", 1), ("P", 1)), (("I", 0), ("P", -1)),
])
def test_correlation_1d_brute_force(fa, fb):
    """W(t) = int a(s) b(s - t) ds vs direct numerical integration on a fine grid."""
    pieces = G.correlation_1d(fa, fb)
    ts = np.linspace(-0.999, 0.999, 38)  # avoids the breakpoint t = 0

    def evalW(t):
        v = 0.0
        for kind, lo, c in pieces:
            if lo <= t < lo + 1:
                v += np.polyval(c[::-1], t - lo)
        return v

    def brute(t):
        if fa[0] == "I" and fb[0] == "I":
            lo, hi = max(-0.5, t - 0.5), min(0.5, t + 0.5)
            x, w = gauss01(8)
            s = lo + (hi - lo) * x
            return (hi - lo) * np.sum(w * s ** fa[1] * (s - t) ** fb[1])
        if fa[0] == "P":
            s0 = fa[1] / 2.0
            return (s0 - t) ** fb[1] if abs(s0 - t) <= 0.5 else 0.0
        s0 = fb[1] / 2.0
        return (t + s0) ** fa[1] if abs(t + s0) <= 0.5 else 0.0

    for t in ts:
        assert abs(evalW(t) - brute(t)) < 1e-14


def test_correlation_points():
    assert G.correlation_1d(("P", 1), ("P", -1)) == [("point", 1, 1.0)]
    assert G.correlation_1d(("P", -1), ("P", -1)) == [("point", 0, 1.0)]
    assert G.correlation_1d(("P", -1), ("P", 1)) == [("point", -1, 1.0)]


OFFSETS = np.array([[0, 0, 0], [1, 0, 0], [0, -1, 0], [1, 1, 0], [-1, 1, -1], [2, -1, 1], [0, 0, 3], [3, 2, -2]])


@pytest.fixture(scope="module")
def near():
    delta = np.array([0.004, 0.005, 0.0045])
    k0 = 9.0
    mom = G.prepare_moments(delta, k0, OFFSETS)
    return dict(delta=delta, k0=k0, mom=mom,
                S=G.s_entries(delta, k0, OFFSETS, mom), Q=G.q_entries(delta, k0, OFFSETS, mom),
                N=G.n_entries(delta, k0, OFFSETS, mom))


def test_trace_identity(near):
    """sum_p Q^{pl,pl'}(d) = k0^2 S^{ll'}(d) + delta_{d0} delta_{ll'} G^l at every offset incl. singular ones.

    From sum_p d_p d_p = Laplacian and (lap + k0^2) g = -delta (Eq. 10), integrating by parts twice."""
    S, Q, delta, k0 = near["S"], near["Q"], near["delta"], near["k0"]
    dV = np.prod(delta)
    zero = np.all(OFFSETS == 0, axis=1)
    for l in range(1, 5):
        for lp in range(1, 5):
            tr = sum(Q[G.comp(p, l), G.comp(p, lp)] for p in range(3))
            rhs = k0 * k0 * S[l - 1, lp - 1] + zero * (l == lp) * G.gram(l, dV)
            assert np.max(np.abs(tr - rhs)) < 1e-13 * dV


def test_cube_self_term():
    """Cubic voxel: Q^{p1,p1}(0) equal for x,y,z (symmetry), so each = (k0^2 S^{11}(0) + DV)/3;
    off-diagonal Q^{p1,q1}(0) = 0 (reflection symmetry); static limit N^{p1,p1}(0) -> 2 DV/3."""
    h = 0.01
    delta = np.array([h, h, h])
    D = np.zeros((1, 3), dtype=int)
    for k0 in (1e-6, 6.0, 20.0):
        mom = G.prepare_moments(delta, k0, D)
        S = G.s_entries(delta, k0, D, mom)[:, :, 0]
        Q = G.q_entries(delta, k0, D, mom)[:, :, 0]
        dV = h ** 3
        target = (k0 * k0 * S[0, 0] + dV) / 3.0
        for p in range(3):
            assert abs(Q[4 * p, 4 * p] - target) < 1e-14 * dV
            for q in range(3):
                if q != p:
                    assert abs(Q[4 * p, 4 * q]) < 1e-14 * dV
        if k0 < 1e-3:
            N = G.n_entries(delta, k0, D, mom)[:, :, 0]
            for p in range(3):
                assert abs(N[4 * p, 4 * p] - 2.0 * dV / 3.0) < 1e-12 * dV


def test_static_cube_self_potential():
    """k0 -> 0: S^{11}(0) = a^5 / (4 pi) * <|r - r'|^-1>_{unit cube}, with the closed form
    2 [(1 + sqrt2 - 2 sqrt3)/5 - pi/3 + ln((1 + sqrt2)(2 + sqrt3))] = 1.88231264438966..."""
    a = 0.007
    delta = np.array([a, a, a])
    D = np.zeros((1, 3), dtype=int)
    S = G.s_entries(delta, 0.0, D)[0, 0, 0]
    c = 2.0 * ((1 + np.sqrt(2) - 2 * np.sqrt(3)) / 5 - np.pi / 3 + np.log((1 + np.sqrt(2)) * (2 + np.sqrt(3))))
    assert abs(S - a ** 5 * c / (4 * np.pi)) < 1e-14 * abs(S)


def test_static_cube_constant_mpmath():
    """Independent check of the closed-form constant above by mpmath quadrature."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 16
    f = lambda u, v: mp.quad(lambda t: (1 - t) * (1 - t * u) * (1 - t * v) * t / mp.sqrt(1 + u * u + v * v), [0, 1])
    val = 24 * mp.quad(lambda u: mp.quad(lambda v: f(u, v), [0, 1]), [0, 1])
    c = 2.0 * ((1 + np.sqrt(2) - 2 * np.sqrt(3)) / 5 - np.pi / 3 + np.log((1 + np.sqrt(2)) * (2 + np.sqrt(3))))
    assert abs(float(val) - c) < 1e-13


def _dyadic_6d(delta, k0, d, n):
    """N^{alpha beta}(d) for separated voxels by plain 6-D Gauss of the pointwise dyadic kernel
    f_m . (k0^2 g I + grad grad g) f_n  (valid for r != r'), no reduction involved."""
    x, w = gauss01(n)
    s = x - 0.5
    S = np.stack(np.meshgrid(s, s, s, indexing="ij"), -1).reshape(-1, 3)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    R = (np.asarray(d)[None, None, :] + S[:, None, :] - S[None, :, :]) * delta
    Rn = np.sqrt((R ** 2).sum(-1))
    Rh = R / Rn[..., None]
    g = np.exp(-1j * k0 * Rn) / (4 * np.pi * Rn)
    a = g * (-1 / Rn ** 2 - 1j * k0 / Rn) + k0 * k0 * g
    c = g * (3 / Rn ** 2 + 3j * k0 / Rn - k0 * k0)
    phi = np.ones((S.shape[0], 4))
    phi[:, 1:] = S
    dV = np.prod(delta)
    out = np.zeros((12, 12), dtype=complex)
    for p in range(3):
        for q in range(3):
            K = c * Rh[..., p] * Rh[..., q] + (a if p == q else 0.0)
            M = np.einsum("i,ia,ij,j,jb->ab", W, phi, K, W, phi, optimize=True) * dV * dV
            for l in range(4):
                for lp in range(4):
                    out[4 * p + l, 4 * q + lp] = M[l, lp]
    return out


@pytest.mark.parametrize("d", [(2, 0, 0), (0, -2, 1), (2, 1, -1), (-3, 2, 1)])
def test_far_entries_vs_dyadic_kernel(d):
    """Reduced evaluation (Q, S pieces) vs the unreduced dyadic kernel on separated voxels, all 144 entries."""
    delta = np.array([0.004, 0.005, 0.0045])
    k0 = 9.0
    N = G.n_entries(delta, k0, np.array([d]))[:, :, 0]
    ref = _dyadic_6d(delta, k0, d, 11)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(N - ref)) < 1e-10 * scale


def _parity(i, a):
    p, l = divmod(a, 4)
    return (-1) ** (int(p == i) + int(_lin(l + 1) == i))


def test_reciprocity_reflection_symmetries(near):
    """T^{ab}(d) = T^{ba}(-d) (reciprocity of the Galerkin form) and
    T^{ab}(R_i d) = s^i_a s^i_b T^{ab}(d) (reflection of axis i flips the p-component and the
    function linear along i), computed by the oracle without using either."""
    delta, k0 = near["delta"], near["k0"]
    D = np.array([[1, 2, 0], [2, -1, 1], [0, 1, 1], [1, 0, 0], [3, 1, 2]])
    Dall = [D, -D]
    for i in range(3):
        Di = D.copy()
        Di[:, i] *= -1
        Dall.append(Di)
    Dall = np.concatenate(Dall)
    T = G.n_entries(delta, k0, Dall)
    n = len(D)
    Tp, Tm = T[:, :, :n], T[:, :, n:2 * n]
    scale = np.max(np.abs(Tp))
    assert np.max(np.abs(Tp - np.transpose(Tm, (1, 0, 2)))) < 1e-13 * scale
    for i in range(3):
        Ti = T[:, :, (2 + i) * n:(3 + i) * n]
        sgn = np.array([[_parity(i, a) * _parity(i, b) for b in range(12)] for a in range(12)])
        assert np.max(np.abs(Ti - sgn[:, :, None] * Tp)) < 1e-13 * scale


def test_sixty_unique_tensors():
    """Exactly 60 of the 144 tensors are distinct up to sign (Section III-C, Section V)."""
    delta = np.array([0.004, 0.005, 0.0045])
    rng = np.random.Generator(np.random.PCG64(5))
    D = rng.integers(-3, 4, size=(24, 3))
    D[0] = 0
    T = G.n_entries(delta, 9.0, D).reshape(144, -1)
    scale = np.max(np.abs(T))
    classes = []
    for a in range(144):
        for c in classes:
            if min(np.max(np.abs(T[a] - T[c])), np.max(np.abs(T[a] + T[c]))) < 1e-12 * scale:
                break
        else:
            classes.append(a)
    assert len(classes) == GOLD["unique_tensors"]["N"]


def test_quadrature_self_convergence(monkeypatch):
    """Raising every Gauss and Duffy order by 4 changes the entries by < 1e-13 of their scale."""
    delta = np.array([0.004, 0.005, 0.0045])
    k0 = 12.0
    D = OFFSETS
    T0 = G.n_entries(delta, k0, D)
    base = G.gauss_order
    monkeypatch.setattr(G, "gauss_order", lambda r: base(r) + 4)
    monkeypatch.setattr(G.Moments, "DUFFY_T", G.Moments.DUFFY_T + 4)
    monkeypatch.setattr(G.Moments, "DUFFY_S", G.Moments.DUFFY_S + 4)
    T1 = G.n_entries(delta, k0, D)
    assert np.max(np.abs(T0 - T1)) < 1e-13 * np.max(np.abs(T0))
