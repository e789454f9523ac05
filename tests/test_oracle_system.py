"""Pins of the oracle's MoM system, solver, sources, post-processing and Mie series."""

import json
import os

import numpy as np
import pytest

from oracle import C0, EPS0, MU0
from oracle import mie
from oracle import operator as O
from oracle import post as P
from oracle import rhs as R
from oracle import solver as S
from oracle.green import NCOMP
from synth import Grid, random_coefficients, random_tissue, sphere_phantom

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def test_paper_dof_and_memory_tables():
    """Tables II, IV, VI, VII: DoFs = 12 N_V (PWL), 3 N_V (PWC); memory 96 N_V / 24 N_V complex128."""
    for r in GOLD["rows"]:
        nx, ny, nz = r["n"]
        nv = nx * ny * nz
        assert round(NCOMP * nv / 1e6, 2) == pytest.approx(r["dofs_pwl"], abs=0.011)
        assert round(3 * nv / 1e6, 2) == pytest.approx(r["dofs_pwc"], abs=0.011)
        assert round(8 * NCOMP * nv * 16 / 2 ** 30, 3) == pytest.approx(r["mem_pwl"], abs=1.1e-3)
        assert round(8 * 3 * nv * 16 / 2 ** 30, 3) == pytest.approx(r["mem_pwc"], abs=1.1e-3)


@pytest.fixture(scope="module")
def tiny():
    g = Grid(3, 2, 4, 0.004, 0.005, 0.0045)
    eps, sig = random_tissue(g, seed=3)
    prob = O.Problem(g, 298e6, eps, sig)
    Nop = O.NOperator(g, prob.k0)
    return g, prob, Nop


def test_fft_matvec_equals_dense(tiny):
    """Circulant embedding + FFT (Section IV-A) reproduces the dense MoM product (Eq. 24)."""
    g, prob, Nop = tiny
    x = random_coefficients(g, 2, seed=11)
    A = O.dense_A(prob, Nop.T)
    for r in range(2):
        ref = (A @ x[r].ravel()).reshape(x[r].shape)
        y = O.apply_A(prob, Nop, x[r])
        assert np.linalg.norm(y - ref) < 1e-13 * np.linalg.norm(ref)
    # batched form
    yb = O.apply_A(prob, Nop, x)
    assert np.linalg.norm(yb[1] - O.apply_A(prob, Nop, x[1])) == 0.0


def test_galerkin_matrix_complex_symmetric(tiny):
    """Reciprocity: the Galerkin N matrix is complex symmetric (not Hermitian)."""
    g, prob, Nop = tiny
    N = O.dense_N(g, Nop.T)
    assert np.max(np.abs(N - N.T)) < 1e-14 * np.max(np.abs(N))
    assert np.max(np.abs(N - N.conj().T)) > 1e-6 * np.max(np.abs(N))


def test_gmres_matches_direct_solve(tiny):
    g, prob, Nop = tiny
    e = R.planewave_tested(g, prob.k0)
    b = R.rhs(prob, e)
    A = O.dense_A(prob, Nop.T)
    xd = S.direct_solve(A, b)
    x, info = S.gmres(lambda v: O.apply_PA(prob, Nop, v), O.apply_Pinv(prob, b), tol=1e-12, restart=20, maxit=50)
    assert info["converged"]
    assert np.linalg.norm(x - xd) < 1e-10 * np.linalg.norm(xd)
    # restarted run (restart shorter than the iteration count) converges to the same solution
    x2, info2 = S.gmres(lambda v: O.apply_PA(prob, Nop, v), O.apply_Pinv(prob, b), tol=1e-12, restart=5, maxit=200)
    assert info2["restarts"] > 1
    assert np.linalg.norm(x2 - xd) < 1e-9 * np.linalg.norm(xd)


def test_preconditioned_operator_identity_in_air():
    """P^-1 A = I - M_tau G^-1 N (Eq. 17): in air voxels (chi = 0) it is the identity row."""
    g = Grid(3, 3, 3, 0.004, 0.004, 0.004)
    eps, sig = random_tissue(g, seed=4, air_fraction=0.5)
    prob = O.Problem(g, 128e6, eps, sig)
    Nop = O.NOperator(g, prob.k0)
    x = random_coefficients(g, 1, seed=5)[0]
    y = O.apply_PA(prob, Nop, x)
    air = np.broadcast_to(prob.chi == 0, x.shape)
    assert np.allclose(y[air], x[air], rtol=0, atol=1e-14 * np.abs(x).max())
    G = prob.gram_vector()[:, None, None, None]
    alt = x - prob.tau * Nop.apply(x) / G
    assert np.linalg.norm(y - alt) < 1e-13 * np.linalg.norm(y)


def test_planewave_closed_form_vs_quadrature():
    g = Grid(3, 4, 5, 0.02, 0.015, 0.03)
    k0 = O.k0_of(298e6) * 3.0
    d = np.array([0.3, -0.4, 0.866])
    d /= np.linalg.norm(d)
    pol = np.cross(d, [1.0, 0.0, 0.0])
    pol /= np.linalg.norm(pol)
    e_cf = R.planewave_tested(g, k0, pol, d)
    e_q = R.tested_field_quadrature(g, lambda r: pol * np.exp(-1j * k0 * (r @ d))[..., None], n=10)
    assert np.max(np.abs(e_cf - e_q)) < 1e-13 * np.max(np.abs(e_cf))


def test_dipole_field_matches_finite_differences():
    """e = (1/c_e)(k0^2 g p + grad(p . grad g)) vs central differences of g (no closed-form second derivatives)."""
    k0 = O.k0_of(298e6)
    ce = 1j * 2 * np.pi * 298e6 * EPS0
    r0 = np.array([0.01, -0.02, 0.03])
    p = np.array([0.2, -0.5, 1.0])
    r = np.array([[0.05, 0.04, -0.02], [0.1, 0.0, 0.0], [0.013, -0.017, 0.09]])
    E = R.dipole_field(r, r0, p, k0, ce)
    g = lambda x: np.exp(-1j * k0 * np.linalg.norm(x - r0)) / (4 * np.pi * np.linalg.norm(x - r0))
    def hessian(ri, h):
        H = np.zeros((3, 3), dtype=complex)
        for a in range(3):
            for b in range(3):
                ea, eb = np.eye(3)[a] * h, np.eye(3)[b] * h
                H[a, b] = (g(ri + ea + eb) - g(ri + ea - eb) - g(ri - ea + eb) + g(ri - ea - eb)) / (4 * h * h)
        return H

    for i, ri in enumerate(r):
        H = (4.0 * hessian(ri, 1e-4) - hessian(ri, 2e-4)) / 3.0  # Richardson, O(h^4)
        ref = (k0 * k0 * g(ri) * p + H @ p) / ce
        assert np.linalg.norm(E[i] - ref) < 1e-8 * np.linalg.norm(ref)


def test_constants():
    assert abs(1.0 / np.sqrt(MU0 * EPS0) - C0) < 1e-6
    assert abs(MU0 / (4e-7 * np.pi) - 1.0) < 1e-9


def test_post_power_identities():
    """At the solution: (a) in tissue the field from the extra matvec equals x / (c_e chi) (the equation
    itself rearranged); (b) P_abs of Eq. 44 equals sum over tissue of (sigma/2) sum_alpha |e_alpha|^2 G_alpha."""
    g = Grid(4, 4, 4, 0.01, 0.01, 0.01)
    eps, sig = random_tissue(g, seed=8, air_fraction=0.3)
    prob = O.Problem(g, 128e6, eps, sig)
    Nop = O.NOperator(g, prob.k0)
    e_inc = R.planewave_tested(g, prob.k0)
    b = R.rhs(prob, e_inc)
    x, info = S.gmres(lambda v: O.apply_PA(prob, Nop, v), O.apply_Pinv(prob, b), tol=1e-13, restart=60, maxit=20)
    e = P.fields(prob, Nop, x, e_inc)
    tissue = np.broadcast_to(prob.chi != 0, x.shape)
    ej = np.where(prob.chi != 0, x / np.where(prob.chi != 0, prob.ce * prob.chi, 1.0), 0)
    assert np.linalg.norm((e - ej)[tissue]) < 1e-9 * np.linalg.norm(e[tissue])
    p, Pabs = P.absorbed_power(prob, x)
    G = prob.gram_vector()[:, None, None, None]
    ref = 0.5 * np.sum(sig * (np.abs(e) ** 2 * G).sum(0) * (prob.chi != 0))
    assert abs(Pabs - ref) < 1e-9 * abs(ref)
    assert np.all(p[prob.chi == 0] == 0) and np.all(p >= 0)


def test_mie_rayleigh_limit():
    """k0 a |eps| -> 0: P_abs -> (sigma/2) |3/(eps+2)|^2 |E0|^2 (4/3 pi a^3) (quasi-static sphere;
    the eddy-current term is of relative order (k0 a |eps|)^2 and is negligible here)."""
    f, a = 298e6, 1e-5
    for er, s in ((50.0, 0.5), (5.0, 0.05), (80.0, 2.0)):
        eps = er - 1j * s / (2 * np.pi * f * EPS0)
        ref = 0.5 * s * abs(3.0 / (eps + 2.0)) ** 2 * (4.0 / 3.0) * np.pi * a ** 3
        assert abs(mie.absorbed_power(er, s, a, f) - ref) < 1e-4 * ref


def test_mie_positivity_and_lossless():
    for er, s, a, f in ((64.0, 0.51, 0.075, 298.06e6), (227.0, 0.25, 0.075, 21.29e6), (50.0, 0.5, 0.1, 298e6)):
        eps = er - 1j * s / (2 * np.pi * f * EPS0)
        cext, csca, cabs = mie.cross_sections(eps, a, f)
        assert csca > 0 and cabs > 0 and cext > cabs
    cext, csca, cabs = mie.cross_sections(9.0 + 0j, 0.05, 298e6)
    assert abs(cabs) < 1e-12 * csca


@pytest.mark.slow
def test_sphere_absorbed_power_vs_mie():
    """Section V-A: absorbed power of a homogeneous sphere vs the Mie series, PWL and PWC.
    PWL: a discretisation-error pin (staircase sphere), a few per cent at 12.5 mm voxels and
    decreasing under refinement.  PWC (the l = 1 sub-block): several times the PWL error, the
    factor growing under refinement (the paper finds about 12 at 5 mm and finer)."""
    Pm = mie.absorbed_power(50.0, 0.5, 0.1, 298e6)
    errs, errs_pwc = [], []
    for n in (16, 20):
        h = 0.2 / n
        g = Grid(n, n, n, h, h, h)
        eps, sig = sphere_phantom(g, 0.1, 50.0, 0.5)
        prob = O.Problem(g, 298e6, eps, sig)
        Nop = O.NOperator(g, prob.k0)
        b = R.rhs(prob, R.planewave_tested(g, prob.k0))
        x, info = S.gmres(lambda v: O.apply_PA(prob, Nop, v), O.apply_Pinv(prob, b), tol=1e-6, restart=50, maxit=20)
        assert info["converged"]
        _, Pabs = P.absorbed_power(prob, x)
        errs.append(abs(Pabs - Pm) / Pm)
        m = O.pwc_mask()
        xc, info = S.gmres(lambda v: O.apply_PA_pwc(prob, Nop, v), m * O.apply_Pinv(prob, b), tol=1e-6, restart=50,
                           maxit=20)
        assert info["converged"]
        assert np.all(xc * (1 - m) == 0)  # the iteration stays in the PWC unknowns
        _, Pabs_c = P.absorbed_power(prob, xc)
        errs_pwc.append(abs(Pabs_c - Pm) / Pm)
    assert errs[0] < 0.15 and errs[1] < errs[0]
    ratios = [c / l for c, l in zip(errs_pwc, errs)]
    assert ratios[0] > 2.5 and ratios[1] > ratios[0]


def test_planewave_voxel_integrals_vs_mpmath():
    """The 1-D voxel integrals of Eq. 30 for a plane wave, int s^k exp(-i kappa s) ds, vs mpmath quadrature
    across the switch between the Taylor series and the closed form."""
    mp = pytest.importorskip("mpmath")
    for kap in (1e-6, 1e-3, 0.07, 0.2499, 0.25, 0.3, 1.3, 4.0):
        for k, f in ((0, R._f0), (1, R._f1)):
            ref = complex(mp.quad(lambda s: s ** k * mp.exp(-1j * kap * s), [-0.5, 0.5]))
            assert abs(complex(f(np.array(kap))) - ref) <= 1e-13 * abs(ref)


def _mie_direct(m, x, n_terms):
    """a_n, b_n of Bohren & Huffman (Eq. 4.53) straight from the Riccati-Bessel functions
    psi_n(z) = z j_n(z), xi_n(z) = z h_n^(1)(z) of scipy.special (no logarithmic derivative,
    no recurrence of the oracle's)."""
    from scipy.special import spherical_jn, spherical_yn

    n = np.arange(1, n_terms + 1)
    mx = m * x

    def psi(z):
        return z * spherical_jn(n, z)

    def dpsi(z):
        return spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)

    def xi(z):
        return z * (spherical_jn(n, z) + 1j * spherical_yn(n, z))

    def dxi(z):
        h = spherical_jn(n, z) + 1j * spherical_yn(n, z)
        dh = spherical_jn(n, z, derivative=True) + 1j * spherical_yn(n, z, derivative=True)
        return h + z * dh

    a = (m * psi(mx) * dpsi(x) - psi(x) * dpsi(mx)) / (m * psi(mx) * dxi(x) - xi(x) * dpsi(mx))
    b = (psi(mx) * dpsi(x) - m * psi(x) * dpsi(mx)) / (psi(mx) * dxi(x) - m * xi(x) * dpsi(mx))
    return a, b


@pytest.mark.parametrize("er,s,a,f", [(50.0, 0.5, 0.1, 298e6), (80.0, 2.0, 0.01, 447e6), (5.0, 0.05, 0.064, 447e6),
                                       (40.0, 0.6, 0.09, 128e6)])
def test_mie_coefficients_vs_direct_bessel(er, s, a, f):
    """The oracle's a_n, b_n (downward logarithmic-derivative recurrence) against a direct
    evaluation with spherical Bessel functions, at the sizes and materials of the workloads
    (the Mie-check sphere: k0 a = 0.62, |m| k0 a = 4.4)."""
    eps = er - 1j * s / (2 * np.pi * f * EPS0)
    m = np.sqrt(np.conj(eps))
    x = 2 * np.pi * f / 299792458.0 * a
    ao, bo = mie.mie_coefficients(m, x)
    ad, bd = _mie_direct(m, x, len(ao))
    assert np.max(np.abs(ao - ad)) <= 1e-10 * np.max(np.abs(ad))
    assert np.max(np.abs(bo - bd)) <= 1e-10 * np.max(np.abs(bd))
    # and the cross-sections the oracle forms from them
    k0 = 2 * np.pi * f / 299792458.0
    n = np.arange(1, len(ad) + 1)
    cext = 2 * np.pi / k0 ** 2 * np.sum((2 * n + 1) * np.real(ad + bd))
    csca = 2 * np.pi / k0 ** 2 * np.sum((2 * n + 1) * (np.abs(ad) ** 2 + np.abs(bd) ** 2))
    ce, cs, ca = mie.cross_sections(eps, a, f)
    assert abs(ce - cext) <= 1e-10 * abs(cext) and abs(cs - csca) <= 1e-10 * abs(csca)


def test_mie_published_example():
    """The sample output of Bohren & Huffman's BHMIE (Appendix A): Q_ext, Q_sca and Q_back of a
    sphere of radius 0.525 um, m = 1.55, in light of 0.6328 um, printed to six digits."""
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mie_published.json")))
    x = 2 * np.pi * ref["radius_um"] / ref["wavelength_um"]
    m = complex(*ref["refractive_index"])
    f = 298e6  # any frequency: only the size parameter k0 a enters
    a = x / (2 * np.pi * f / 299792458.0)
    cext, csca, _ = mie.cross_sections(np.conj(m) ** 2, a, f)
    area = np.pi * a * a
    half_ulp = 0.5 * 10.0 ** (1 - ref["digits"])
    assert abs(cext / area - ref["Q_ext"]) <= half_ulp * 1.01
    assert abs(csca / area - ref["Q_sca"]) <= half_ulp * 1.01
    an, bn = mie.mie_coefficients(m, x)
    n = np.arange(1, len(an) + 1)
    qback = abs(np.sum((2 * n + 1) * (-1.0) ** n * (an - bn))) ** 2 / x ** 2
    assert abs(qback - ref["Q_back"]) <= half_ulp * 1.01
    # the rounded size parameter the table prints gives a visibly different Q_ext: the pin is sharp
    cext2, _, _ = mie.cross_sections(np.conj(m) ** 2, 5.213 / (2 * np.pi * f / 299792458.0), f)
    assert abs(cext2 / (np.pi * (5.213 / (2 * np.pi * f / 299792458.0)) ** 2) - ref["Q_ext"]) > 1e-4


def test_dense_N_from_absolute_positions():
    """The dense Galerkin matrix assembled pair by pair from the voxels' absolute centre positions
    (each pair's entries computed on their own) equals the one indexed from the Toeplitz tensor
    T[m - n] (translation invariance of the Galerkin entries, Eq. 42-43)."""
    from oracle import green as OG

    g = Grid(3, 2, 4, 0.004, 0.005, 0.0045)
    k0 = O.k0_of(298e6)
    xx, yy, zz = g.centres()
    pos = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1)
    delta = np.array([g.dx, g.dy, g.dz])
    nv = g.nv
    D = np.rint((pos[:, None, :] - pos[None, :, :]) / delta).astype(np.int64).reshape(-1, 3)
    E = OG.n_entries(delta, k0, D).reshape(12, 12, nv, nv)
    M = np.transpose(E, (0, 2, 1, 3)).reshape(12 * nv, 12 * nv)
    T = OG.toeplitz_tensors(g, k0)
    ref = O.dense_N(g, T)
    assert np.max(np.abs(M - ref)) <= 1e-14 * np.max(np.abs(ref))
