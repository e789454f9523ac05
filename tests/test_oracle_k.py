"""Pins of the oracle's K operator (K u = curl S u, Eq. 8; Eq. 25) and magnetic post-processing.

Each checks the reduced evaluation against an independent route: plain 6-D Gauss of the
unreduced kernel eps_{pjq} d_j g on separated voxels, the integration by parts done on the
source side instead of the testing side (different moments, including the singular
offsets), identities of the operator, and the count of distinct tensors the paper states.
"""

import json
import os

import numpy as np
import pytest

from oracle import EPS0, MU0
from oracle import green as G
from oracle import operator as O
from oracle import post as OP
from oracle import rhs as RHS
from oracle.quadrature import gauss01
from synth import Grid, random_coefficients, random_tissue

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
DELTA = np.array([0.004, 0.005, 0.0045])
K0 = 9.0
EPS = np.zeros((3, 3, 3))
for i, j, k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
    EPS[i, j, k], EPS[i, k, j] = 1.0, -1.0


def _lin(l):
    return None if l == 1 else l - 2


def _parity(i, a):
    p, l = divmod(a, 4)
    return (-1) ** (int(p == i) + int(_lin(l + 1) == i))


def _curl_kernel_6d(delta, k0, d, n):
    """K^{alpha beta}(d) for separated voxels by plain 6-D Gauss of f_m . (grad g x f_n), i.e. the
    kernel eps_{pjq} d_j g(r - r') with d_j g = g (-1/R - i k0) R_j / R, no reduction involved."""
    x, w = gauss01(n)
    s = x - 0.5
    S = np.stack(np.meshgrid(s, s, s, indexing="ij"), -1).reshape(-1, 3)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    R = (np.asarray(d)[None, None, :] + S[:, None, :] - S[None, :, :]) * delta
    Rn = np.sqrt((R ** 2).sum(-1))
    g = np.exp(-1j * k0 * Rn) / (4 * np.pi * Rn)
    dg = g * (-1.0 / Rn - 1j * k0) / Rn  # times R_j gives d_j g
    phi = np.ones((S.shape[0], 4))
    phi[:, 1:] = S
    dV = np.prod(delta)
    out = np.zeros((12, 12), dtype=complex)
    for p in range(3):
        for q in range(3):
            ker = sum(EPS[p, j, q] * dg * R[..., j] for j in range(3))
            if not np.any(ker):
                continue
            M = np.einsum("i,ia,ij,j,jb->ab", W, phi, ker, W, phi, optimize=True) * dV * dV
            out[4 * p:4 * p + 4, 4 * q:4 * q + 4] = M
    return out


@pytest.mark.parametrize("d", [(2, 0, 0), (0, -2, 1), (2, 1, -1), (-3, 2, 1)])
def test_far_entries_vs_curl_kernel(d):
    K = G.k_entries(DELTA, K0, np.array([d]))[:, :, 0]
    ref = _curl_kernel_6d(DELTA, K0, d, 11)
    assert np.max(np.abs(K - ref)) < 1e-10 * np.max(np.abs(ref))


def _k_source_side(delta, k0, D):
    """The same entries with d_j g(r - r') = -d'_j g moved onto the source function:
    K^{(p,l),(q,l')}(d) = + sum_j eps_{pjq} int int N^l_m g (D_j N^{l'}_n)."""
    mom = G.prepare_moments(delta, k0, D)
    dV = float(np.prod(delta))
    T = np.zeros((12, 12, len(D)), dtype=complex)
    for p in range(3):
        for q in range(3):
            for j in range(3):
                if EPS[p, j, q] == 0:
                    continue
                for l in range(1, 5):
                    for lp in range(1, 5):
                        v = np.zeros(len(D), dtype=complex)
                        for c, fb in G.divergence_pieces(j, lp):
                            v += c * G.pair_integral(G.basis_factors(l), fb, D, mom)
                        T[4 * p + l - 1, 4 * q + lp - 1] += EPS[p, j, q] * dV * dV / delta[j] * v
    return T


NEAR = np.array([[0, 0, 0], [1, 0, 0], [0, -1, 0], [0, 0, 1], [1, 1, 0], [-1, 0, 1], [1, -1, 1], [2, 1, 0]])


def test_singular_offsets_both_sides_of_the_integration_by_parts():
    """Coinciding, face-, edge- and vertex-adjacent voxels: derivative on the testing function
    (the oracle) and on the source function agree; a wrong sign or a missing face mass on
    either side breaks it."""
    A = G.k_entries(DELTA, K0, NEAR)
    B = _k_source_side(DELTA, K0, NEAR)
    assert np.max(np.abs(A - B)) < 1e-13 * np.max(np.abs(A))


def test_operator_identities():
    """Diagonal component blocks vanish; swapping p and q flips the sign; reciprocity
    K^{ba}(-d) = K^{ab}(d); reflection of axis i: K^{ab}(R_i d) = -s^i_a s^i_b K^{ab}(d)
    (the curl of a reflected field carries one more sign than N)."""
    D = np.array([[1, 2, 0], [2, -1, 1], [0, 1, 1], [1, 0, 0], [3, 1, 2], [0, 0, 0]])
    Dall = [D, -D]
    for i in range(3):
        Di = D.copy()
        Di[:, i] *= -1
        Dall.append(Di)
    T = G.k_entries(DELTA, K0, np.concatenate(Dall))
    n = len(D)
    Tp, Tm = T[:, :, :n], T[:, :, n:2 * n]
    scale = np.max(np.abs(Tp))
    for p in range(3):
        assert np.max(np.abs(Tp[4 * p:4 * p + 4, 4 * p:4 * p + 4])) == 0.0
        for q in range(3):
            assert np.max(np.abs(Tp[4 * p:4 * p + 4, 4 * q:4 * q + 4] + Tp[4 * q:4 * q + 4, 4 * p:4 * p + 4])) \
                < 1e-13 * scale
    assert np.max(np.abs(Tp - np.transpose(Tm, (1, 0, 2)))) < 1e-13 * scale
    for i in range(3):
        Ti = T[:, :, (2 + i) * n:(3 + i) * n]
        sgn = np.array([[_parity(i, a) * _parity(i, b) for b in range(12)] for a in range(12)])
        assert np.max(np.abs(Ti + sgn[:, :, None] * Tp)) < 1e-13 * scale


def test_thirty_unique_tensors():
    """The 96 non-zero K tensors fall into exactly 30 classes up to sign (Section III-C)."""
    rng = np.random.Generator(np.random.PCG64(7))
    D = rng.integers(-3, 4, size=(24, 3))
    D[0] = 0
    T = G.k_entries(DELTA, K0, D).reshape(144, -1)
    scale = np.max(np.abs(T))
    classes = []
    for a in range(144):
        if np.max(np.abs(T[a])) < 1e-14 * scale:
            continue
        for c in classes:
            if min(np.max(np.abs(T[a] - T[c])), np.max(np.abs(T[a] + T[c]))) < 1e-12 * scale:
                break
        else:
            classes.append(a)
    assert len(classes) == GOLD["unique_tensors"]["K"]
    assert GOLD["unique_tensors"]["N"] + GOLD["unique_tensors"]["K"] == GOLD["unique_tensors"]["total"]


def test_quadrature_self_convergence(monkeypatch):
    """Raising every Gauss and Duffy order by 4 changes the K entries by < 1e-13 of their scale."""
    T0 = G.k_entries(DELTA, 12.0, NEAR)
    base = G.gauss_order
    monkeypatch.setattr(G, "gauss_order", lambda r: base(r) + 4)
    monkeypatch.setattr(G.Moments, "DUFFY_T", G.Moments.DUFFY_T + 4)
    monkeypatch.setattr(G.Moments, "DUFFY_S", G.Moments.DUFFY_S + 4)
    T1 = G.k_entries(DELTA, 12.0, NEAR)
    assert np.max(np.abs(T0 - T1)) < 1e-13 * np.max(np.abs(T0))


# ---------------------------------------------------------------------------
# Magnetic field of a dipole, the K operator on a grid, and the magnetic post-processing
# ---------------------------------------------------------------------------

F = 298e6
KF = O.k0_of(F)
R0 = np.array([0.01, -0.02, 0.03])
PM = np.array([0.2, -0.5, 1.0])
PTS = np.array([[0.05, 0.04, -0.02], [0.1, 0.0, 0.0], [0.013, -0.017, 0.09]])


def _g(x):
    d = np.linalg.norm(x - R0)
    return np.exp(-1j * KF * d) / (4 * np.pi * d)


def _richardson(fd, h):
    return (4.0 * fd(h) - fd(2 * h)) / 3.0  # O(h^4) from two central differences


def test_dipole_hfield_matches_finite_differences():
    """h = grad g x p vs central differences of g (no closed-form derivative)."""
    H = RHS.dipole_hfield(PTS, R0, PM, KF)
    for i, ri in enumerate(PTS):
        grad = _richardson(lambda h: np.array([(_g(ri + e * h) - _g(ri - e * h)) / (2 * h) for e in np.eye(3)]), 1e-4)
        ref = np.cross(grad, PM)
        assert np.linalg.norm(H[i] - ref) < 1e-8 * np.linalg.norm(ref)


def test_dipole_fields_obey_faraday():
    """curl e_inc = -i omega mu0 h_inc (time factor exp(i omega t)): the electric field of the
    dipole (pinned separately) and its magnetic field agree in sign and scale."""
    ce = 1j * 2 * np.pi * F * EPS0
    for ri in PTS:
        def curl(h):
            J = np.zeros((3, 3), dtype=complex)  # J[a, b] = d E_a / d x_b
            for b in range(3):
                e = np.eye(3)[b] * h
                J[:, b] = (RHS.dipole_field((ri + e)[None], R0, PM, KF, ce)[0]
                           - RHS.dipole_field((ri - e)[None], R0, PM, KF, ce)[0]) / (2 * h)
            return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
        lhs = _richardson(curl, 1e-4)
        rhs = -1j * 2 * np.pi * F * MU0 * RHS.dipole_hfield(ri[None], R0, PM, KF)[0]
        assert np.linalg.norm(lhs - rhs) < 1e-7 * np.linalg.norm(rhs)


def test_k_operator_fft_equals_dense_product():
    """K x by circulant embedding + FFT equals the dense Galerkin matrix of K applied to x."""
    g = Grid(3, 2, 4, 0.004, 0.005, 0.0045)
    T = G.k_toeplitz_tensors(g, KF)
    x = random_coefficients(g, 2, seed=3)
    Kop = O.KOperator(g, KF, T)
    y = Kop.apply(x)
    M = O.dense_N(g, T)  # entry (m alpha, n beta) = T^{alpha beta}(m - n), any operator
    ref = (M @ x.reshape(2, -1).T).T.reshape(x.shape)
    assert np.max(np.abs(y - ref)) < 1e-13 * np.max(np.abs(ref))


def test_magnetic_energy_is_the_integral_of_the_pwl_field():
    """W_m from the Gram-weighted coefficients equals 1/4 mu0 int |sum_l h_l N^l|^2 over the tissue
    voxels by direct quadrature of the PWL field; b1+ is mu0 (h_x + i h_y) of the voxel averages."""
    g = Grid(3, 3, 2, 0.004, 0.005, 0.0045)
    eps, sig = random_tissue(g, seed=8, air_fraction=0.4)
    prob = O.Problem(g, F, eps, sig)
    h = random_coefficients(g, 1, seed=9)[0]
    w, W = OP.magnetic_energy(prob, h)
    x, wq = gauss01(4)
    s = x - 0.5
    ref = 0.0
    for iz in range(g.nz):
        for iy in range(g.ny):
            for ix in range(g.nx):
                if prob.chi[iz, iy, ix] == 0:
                    continue
                for a, wa in zip(s, wq):
                    for b, wb in zip(s, wq):
                        for c, wc in zip(s, wq):
                            phi = np.array([1.0, a, b, c])
                            v = np.array([h[4 * p:4 * p + 4, iz, iy, ix] @ phi for p in range(3)])
                            ref += wa * wb * wc * prob.dV * 0.25 * MU0 * np.sum(np.abs(v) ** 2)
    assert abs(W - ref) < 1e-12 * ref
    assert np.all(w[prob.chi == 0] == 0)
    b1 = OP.b1_plus(h)
    assert np.allclose(b1, MU0 * (h[0] + 1j * h[4]), rtol=0, atol=0)
