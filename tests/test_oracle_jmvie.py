"""Pins of the oracle's full JM-VIE (Eq. 13-15) and of the magnetic Mie series.

The JM system is tied to things outside itself:
  * mu = 1 leaves the dielectric system of Eq. 16 (pinned elsewhere) and a zero magnetization;
  * electromagnetic duality: a purely magnetic scatterer (eps = 1, mu) in the incident field
    (e, h) carries m' = j of the dielectric scatterer eps = mu in the field (eta0 h, -e / eta0),
    with e = -eta0 h' and h = e' / eta0 for the fields -- which fixes the scale factors i k0
    and eta0 of the second row and of the field formulas against the dielectric path;
  * reciprocity: diag(1/chi_e, -1/chi_m) A is complex symmetric, which fixes the signs and
    factors of the two coupling blocks relative to each other;
  * a magnetodielectric sphere's absorbed power against the Mie series (discretisation error);
  * the Mie series with mu against a direct spherical-Bessel evaluation, its eps <-> mu duality
    and its quasi-static limit.
"""

import numpy as np
import pytest

from oracle import EPS0, MU0
from oracle import green as OG
from oracle import jmvie as J
from oracle import mie
from oracle import operator as O
from oracle import post as P
from oracle import rhs as R
from oracle import solver as S
from synth import Grid, random_coefficients, random_permeability, random_tissue, sphere_phantom

F = 298e6
K0 = O.k0_of(F)


def _tiny_problem(air_fraction=0.0, seed=5):
    g = Grid(3, 2, 2, 0.004, 0.005, 0.0045)
    eps, sig = random_tissue(g, seed, air_fraction=air_fraction)
    mr, mi = random_permeability(g, seed + 1, nonmagnetic_fraction=air_fraction)
    return J.MagProblem(g, F, eps, sig, mr, mi)


def _ops(g):
    TN = OG.toeplitz_tensors(g, K0)
    TK = OG.k_toeplitz_tensors(g, K0)
    return TN, TK, O.NOperator(g, K0, TN), O.KOperator(g, K0, TK)


def test_nonmagnetic_reduces_to_eq16():
    """mu = 1: the second row is G m', so m' = 0 at the solution, and on m' = 0 the first row is
    the dielectric operator of Eq. 24."""
    g = Grid(4, 3, 5, 0.004, 0.005, 0.0045)
    eps, sig = random_tissue(g, 3)
    prob = J.MagProblem(g, F, eps, sig)
    _, _, Nop, Kop = _ops(g)
    x = random_coefficients(g, 4, seed=9).reshape(2, 2, 12, *g.shape)
    G = prob.gram_vector()[:, None, None, None]
    y = J.apply_A(prob, Nop, Kop, x)
    assert np.max(np.abs(y[:, 1] - G * x[:, 1])) == 0.0
    x[:, 1] = 0.0
    y = J.apply_A(prob, Nop, Kop, x)
    assert np.max(np.abs(y[:, 0] - O.apply_A(prob, Nop, x[:, 0]))) == 0.0
    assert np.max(np.abs(y[:, 1])) == 0.0


def test_fft_matvec_equals_dense():
    prob = _tiny_problem(air_fraction=0.2)
    TN, TK, Nop, Kop = _ops(prob.grid)
    x = random_coefficients(prob.grid, 4, seed=2).reshape(2, 2, 12, *prob.grid.shape)
    y = J.apply_A(prob, Nop, Kop, x)
    A = J.dense_A(prob, TN, TK)
    ref = (A @ x.reshape(2, -1).T).T.reshape(x.shape)
    assert np.max(np.abs(y - ref)) < 1e-13 * np.max(np.abs(ref))


def test_reciprocity_symmetry():
    """diag(1/chi_e, -1/chi_m) A = [[(eps/chi_e) G - N, i k0 K], [i k0 K, N - (mu/chi_m) G]] is
    complex symmetric; the unscaled A is not (the check is not vacuous)."""
    prob = _tiny_problem(air_fraction=0.0)
    TN, TK, _, _ = _ops(prob.grid)
    A = J.dense_A(prob, TN, TK)
    d = np.concatenate([np.tile(1.0 / prob.chi.ravel(), 12), np.tile(-1.0 / prob.chim.ravel(), 12)])
    DA = d[:, None] * A
    scale = np.max(np.abs(DA))
    assert np.max(np.abs(DA - DA.T)) < 1e-12 * scale
    assert np.max(np.abs(A - A.T)) > 1e-3 * np.max(np.abs(A))
    # a coupling block with the other sign breaks it
    n = A.shape[0] // 2
    B = DA.copy()
    B[n:, :n] *= -1
    assert np.max(np.abs(B - B.T)) > 1e-3 * scale


def test_duality_magnetic_scatterer():
    """eps = 1, mu = mu_s in (e, h)  <->  eps = mu_s, mu = 1 in (eta0 h, -e / eta0): m' = j, and
    the magnetic problem's fields are e = -eta0 h', h = e' / eta0 (dense solves)."""
    g = Grid(3, 2, 2, 0.004, 0.005, 0.0045)
    mr, mi = random_permeability(g, 11, nonmagnetic_fraction=0.2)
    one = np.ones(g.shape)
    mag = J.MagProblem(g, F, one, 0.0 * one, mr, mi)
    # the dielectric twin: eps = mr - i mi, i.e. sigma = mi omega eps0
    diel = O.Problem(g, F, mr, mi * (2 * np.pi * F * EPS0))
    TN, TK, Nop, Kop = _ops(g)
    rng = np.random.Generator(np.random.PCG64(4))
    shp = (12,) + g.shape
    e_t = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    h_t = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / J.ETA0
    b = J.rhs(mag, e_t, h_t)
    x = S.direct_solve(J.dense_A(mag, TN, TK), b)
    e2, h2 = J.ETA0 * h_t, -e_t / J.ETA0
    xd = S.direct_solve(O.dense_A(diel, TN), R.rhs(diel, e2))
    scale = np.max(np.abs(xd))
    assert np.max(np.abs(x[0])) < 1e-13 * scale  # no polarization current without chi_e
    assert np.max(np.abs(x[1] - xd)) < 1e-11 * scale
    e_mag, h_mag = J.fields(mag, Nop, Kop, x, e_t, h_t)
    e_d = P.fields(diel, Nop, xd, e2)
    h_d = P.magnetic_fields(diel, Kop, xd, h2)
    assert np.max(np.abs(e_mag + J.ETA0 * h_d)) < 1e-11 * np.max(np.abs(e_mag))
    assert np.max(np.abs(h_mag - e_d / J.ETA0)) < 1e-11 * np.max(np.abs(h_mag))
    # the absorbed power: magnetic loss of the one equals the dielectric loss of the other
    _, Pm = J.absorbed_power(mag, x)
    _, Pd = P.absorbed_power(diel, xd)
    assert abs(Pm - Pd) < 1e-11 * abs(Pd) and Pd > 0


def test_gmres_matches_direct_solve():
    prob = _tiny_problem(air_fraction=0.2, seed=8)
    TN, TK, Nop, Kop = _ops(prob.grid)
    rng = np.random.Generator(np.random.PCG64(6))
    shp = (2, 12) + prob.grid.shape
    b = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    xref = S.direct_solve(J.dense_A(prob, TN, TK), b)
    x, info = S.gmres(lambda v: J.apply_PA(prob, Nop, Kop, v), J.apply_Pinv(prob, b), tol=1e-12, restart=200,
                      maxit=5)
    assert info["converged"]
    assert np.linalg.norm(x - xref) < 1e-9 * np.linalg.norm(xref)


def _mie_direct(m, x, mu, n_terms):
    """a_n, b_n of Bohren & Huffman's Eq. 4.53 (sphere permeability mu, medium 1) from
    scipy.special's spherical Bessel functions; no recurrence of the oracle's."""
    from scipy.special import spherical_jn, spherical_yn

    n = np.arange(1, n_terms + 1)
    mx = m * x
    jx, jmx = spherical_jn(n, x), spherical_jn(n, mx)
    djx, djmx = spherical_jn(n, x, derivative=True), spherical_jn(n, mx, derivative=True)
    hx = jx + 1j * spherical_yn(n, x)
    dhx = djx + 1j * spherical_yn(n, x, derivative=True)
    xj = jx + x * djx  # [x j_n(x)]'
    xh = hx + x * dhx  # [x h_n(x)]'
    mxj = jmx + mx * djmx  # [mx j_n(mx)]' with respect to mx
    a = (m * m * jmx * xj - mu * jx * mxj) / (m * m * jmx * xh - mu * hx * mxj)
    b = (mu * jmx * xj - jx * mxj) / (mu * jmx * xh - hx * mxj)
    return a, b


@pytest.mark.parametrize("eps,mu,a,f", [(50 - 30j, 2.0 - 0.3j, 0.1, 298e6), (1.0, 3.0 - 1.0j, 0.05, 298e6),
                                        (5.0 - 1j, 1.5 - 0.2j, 0.064, 447e6)])
def test_magnetic_mie_vs_direct_bessel(eps, mu, a, f):
    k0 = 2 * np.pi * f / 299792458.0
    mub = np.conj(mu)
    m = np.sqrt(np.conj(eps) * mub)
    ao, bo = mie.mie_coefficients(m, k0 * a, mub)
    ad, bd = _mie_direct(m, k0 * a, mub, len(ao))
    assert np.max(np.abs(ao - ad)) <= 1e-10 * np.max(np.abs(ad))
    assert np.max(np.abs(bo - bd)) <= 1e-10 * np.max(np.abs(bd))


def test_magnetic_mie_duality_and_rayleigh_limit():
    """Swapping eps and mu swaps a_n and b_n (so the cross-sections stay); a small sphere with
    eps = 1 absorbs P = 1/2 omega mu0 mu'' |3/(mu+2)|^2 |H0|^2 (4/3 pi a^3) (quasi-static
    magnetic dipole), H0 = E0 / eta0."""
    f, a = 298e6, 0.05
    eps, mu = 20.0 - 5.0j, 3.0 - 1.0j
    k0 = 2 * np.pi * f / 299792458.0
    m = np.sqrt(np.conj(eps) * np.conj(mu))
    a1, b1 = mie.mie_coefficients(m, k0 * a, np.conj(mu))
    a2, b2 = mie.mie_coefficients(m, k0 * a, np.conj(eps))
    assert np.max(np.abs(a1 - b2)) < 1e-12 * np.max(np.abs(a1))
    assert np.max(np.abs(b1 - a2)) < 1e-12 * np.max(np.abs(b1))
    c1, c2 = mie.cross_sections(eps, a, f, mu), mie.cross_sections(mu, a, f, eps)
    assert np.allclose(c1, c2, rtol=1e-12, atol=0)
    a = 1e-5
    eta0 = np.sqrt(MU0 / EPS0)
    ref = 0.5 * 2 * np.pi * f * MU0 * 1.0 * abs(3.0 / (mu + 2.0)) ** 2 * (1.0 / eta0) ** 2 * 4.0 / 3.0 * np.pi * a ** 3
    assert abs(mie.absorbed_power(1.0, 0.0, a, f, mu=mu) - ref) < 1e-4 * ref


@pytest.mark.slow
def test_magnetodielectric_sphere_vs_mie():
    """A sphere with eps_r = 50, sigma = 0.5 S/m and mu_r = 2 - 0.5 i in an x-polarised plane wave
    along z (h = y / eta0): the JM-VIE absorbed power (electric + magnetic loss) against the Mie
    series, a discretisation-error pin that shrinks under refinement, with K coupling both currents."""
    mu_s = 2.0 - 0.5j
    Pm = mie.absorbed_power(50.0, 0.5, 0.1, F, mu=mu_s)
    errs = []
    for n in (16, 20):
        h = 0.2 / n
        g = Grid(n, n, n, h, h, h)
        eps, sig = sphere_phantom(g, 0.1, 50.0, 0.5)
        inside = eps != 1.0
        prob = J.MagProblem(g, F, eps, sig, np.where(inside, mu_s.real, 1.0), np.where(inside, -mu_s.imag, 0.0))
        Nop, Kop = O.NOperator(g, prob.k0), O.KOperator(g, prob.k0)
        e_t = R.planewave_tested(g, prob.k0, pol=(1.0, 0.0, 0.0))
        h_t = R.planewave_tested(g, prob.k0, pol=(0.0, 1.0 / J.ETA0, 0.0))
        b = J.rhs(prob, e_t, h_t)
        x, info = S.gmres(lambda v: J.apply_PA(prob, Nop, Kop, v), J.apply_Pinv(prob, b), tol=1e-6, restart=50,
                          maxit=20)
        assert info["converged"]
        _, Pabs = J.absorbed_power(prob, x)
        errs.append(abs(Pabs - Pm) / Pm)
    assert errs[0] < 0.15 and errs[1] < errs[0], errs
