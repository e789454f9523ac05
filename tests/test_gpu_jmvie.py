"""Parity of the full JM-VIE on the GPU (vie_jm_*, Eq. 13-15) with the FP64 oracle (oracle/jmvie.py).

Tolerances: matvec, right-hand side, fields and absorbed power <= 1e-12 relative (FP64 against
FP64, each side with its own Green tensors); solutions <= 1e-8 relative at a 1e-11 residual.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import EPS0  # noqa: E402
from oracle import jmvie as J  # noqa: E402
from oracle import mie  # noqa: E402
from oracle import operator as O  # noqa: E402
from oracle import rhs as OR  # noqa: E402
from oracle import solver as OS  # noqa: E402
from synth import Grid, random_coefficients, random_permeability, random_tissue, sphere_phantom  # noqa: E402

F = 298e6


@pytest.fixture(scope="module")
def vie():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_02196_gb300 as v

    v.build()
    return v


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def handle(vie, g, eps, sig, mr=None, mi=None):
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), F, eps, sig)
    if mr is not None:
        vie.vie_set_permeability(h, np.ascontiguousarray(mr, dtype=np.float64),
                                 np.ascontiguousarray(mi, dtype=np.float64))
    return h


def problem(g, seed):
    eps, sig = random_tissue(g, seed)
    mr, mi = random_permeability(g, seed + 100)
    return eps, sig, mr, mi, J.MagProblem(g, F, eps, sig, mr, mi)


def ops(g):
    k0 = O.k0_of(F)
    return O.NOperator(g, k0), O.KOperator(g, k0)


@pytest.mark.parametrize("shape,nrhs", [((7, 5, 4), 2), ((9, 6, 11), 1), ((20, 18, 9), 3)])
def test_jm_matvec_parity(vie, shape, nrhs):
    """A x and P^-1 A x of the JM system on ragged grids, random materials (with air and
    non-magnetic voxels) and random currents: FP64 within 1e-12 and FP32 (the operator of the
    mixed solve's inner GMRES) within 1e-5 of the oracle, on the fused and the line xy paths."""
    g = Grid(*shape, 0.004, 0.005, 0.0045)
    eps, sig, mr, mi, prob = problem(g, sum(shape))
    Nop, Kop = ops(g)
    x = random_coefficients(g, 2 * nrhs, seed=7).reshape(nrhs, 2, 12, *g.shape)
    h = handle(vie, g, eps, sig, mr, mi)
    for op, ref in ((vie.VIE_OP_A, J.apply_A(prob, Nop, Kop, x)), (vie.VIE_OP_PA, J.apply_PA(prob, Nop, Kop, x))):
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        yd = torch.empty_like(xd)
        torch.cuda.synchronize()  # the library's stream does not wait for torch's
        vie.vie_jm_matvec(h, xd, yd, op)
        torch.cuda.synchronize()
        assert rel(yd.cpu().numpy(), ref) <= 1e-12
        yh = np.empty_like(x)  # host buffers take the same path
        vie.vie_jm_matvec(h, x, yh, op)
        assert np.array_equal(yh, yd.cpu().numpy())
        x32 = np.ascontiguousarray(x.astype(np.complex64))
        y32 = np.empty_like(x32)
        vie.vie_jm_matvec(h, x32, y32, op, precision=vie.VIE_FP32)
        assert rel(y32, ref) <= 1e-5
    with pytest.raises(vie.VieError) as e:
        vie.vie_jm_matvec(h, x.astype(np.complex64), np.empty(x.shape, np.complex64), precision=vie.VIE_BF16X3)
    assert e.value.code == vie.VIE_EINVAL
    h.close()


def test_jm_rhs_fields_and_power_parity(vie):
    g = Grid(6, 5, 7, 0.006, 0.005, 0.007)
    eps, sig, mr, mi, prob = problem(g, 31)
    Nop, Kop = ops(g)
    rng = np.random.Generator(np.random.PCG64(12))
    shp = (2, 12) + g.shape
    e_t = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    h_t = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / J.ETA0
    x = random_coefficients(g, 4, seed=8).reshape(2, 2, 12, *g.shape) * 1e-3
    h = handle(vie, g, eps, sig, mr, mi)
    b = np.empty((2, 2, 12) + g.shape, dtype=np.complex128)
    vie.vie_jm_rhs(h, e_t, h_t, b)
    assert rel(b, J.rhs(prob, e_t, h_t)) <= 1e-12
    ec = np.empty(shp, dtype=np.complex128)
    hc = np.empty(shp, dtype=np.complex128)
    p = np.empty((2,) + g.shape)
    P = vie.vie_jm_fields(h, x, e_t, h_t, ec, hc, p)
    h.close()
    er, hr = J.fields(prob, Nop, Kop, x, e_t, h_t)
    pr, Pr = J.absorbed_power(prob, x)
    assert rel(ec, er) <= 1e-12 and rel(hc, hr) <= 1e-12
    assert rel(p, pr) <= 1e-12
    assert np.allclose(P, Pr, rtol=1e-12, atol=0)


@pytest.mark.parametrize("mode", ["fp64", "fp32_refine"])
def test_jm_solve_parity_dense(vie, mode):
    """vie_jm_solve at a 1e-13 preconditioned residual against the oracle's dense LU solve of the same
    system (the unpreconditioned residual is within the condition number of P = diag(eps G, mu G),
    about 1e3 here, of the preconditioned one).  The mixed mode reaches the same FP64 bound through
    its refinement sweeps, its inner products all FP32."""
    g = Grid(5, 4, 3, 0.004, 0.005, 0.0045)
    eps, sig, mr, mi, prob = problem(g, 44)
    from oracle import green as OG

    k0 = O.k0_of(F)
    A = J.dense_A(prob, OG.toeplitz_tensors(g, k0), OG.k_toeplitz_tensors(g, k0))
    rng = np.random.Generator(np.random.PCG64(3))
    shp = (3, 2, 12) + g.shape
    b = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    ref = np.stack([OS.direct_solve(A, b[r]) for r in range(3)])
    h = handle(vie, g, eps, sig, mr, mi)
    x = np.empty_like(b)
    m = vie.VIE_SOLVE_FP64 if mode == "fp64" else vie.VIE_SOLVE_FP32_REFINE
    rc, info = vie.vie_jm_solve(h, b, x, tol=1e-13, restart=80, maxit=20, mode=m, true_resid=True)
    h.close()
    assert rc == vie.VIE_OK and all(i["converged"] for i in info)
    assert all(i["true_resid"] < 1e-9 for i in info), [i["true_resid"] for i in info]
    assert rel(x, ref) <= 1e-9
    if mode == "fp32_refine":
        assert info[0]["fp32_matvecs"] > info[0]["fp64_matvecs"] and info[0]["refinements"] >= 2, info[0]


@pytest.mark.parametrize("mode", ["fp64", "fp32_refine"])
def test_jm_graph_replay_matches_direct_launches(vie, mode):
    """The JM solve's Arnoldi chunks replayed as CUDA graphs give the same bits and counts as the
    same steps launched kernel by kernel (flags bit 3)."""
    g = Grid(9, 8, 7, 0.005, 0.005, 0.005)
    eps, sig, mr, mi, _ = problem(g, 61)
    h = handle(vie, g, eps, sig, mr, mi)
    rng = np.random.Generator(np.random.PCG64(62))
    shp = (2, 2, 12) + g.shape
    b = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    m = vie.VIE_SOLVE_FP64 if mode == "fp64" else vie.VIE_SOLVE_FP32_REFINE
    out = []
    for graph in (True, False):
        x = np.empty_like(b)
        rc, info = vie.vie_jm_solve(h, b, x, tol=1e-10, restart=16, maxit=60, mode=m, graph=graph)
        assert rc == vie.VIE_OK, info
        out.append((x, info))
    h.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_jm_nonmagnetic_equals_dielectric_solve(vie):
    """mu = 1: the magnetization stays exactly zero and j equals vie_solve's FP64 solution."""
    g = Grid(8, 7, 6, 0.005, 0.005, 0.005)
    eps, sig = random_tissue(g, 5)
    h = handle(vie, g, eps, sig)
    pos = np.array([[0.0, 0.06, 0.0], [0.05, -0.04, 0.01]])
    mom = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    shp = (2, 12) + g.shape
    e_t = np.empty(shp, dtype=np.complex128)
    b = np.empty(shp, dtype=np.complex128)
    vie.vie_rhs_dipoles(h, pos, mom, e_t, b)
    h_t = np.empty(shp, dtype=np.complex128)
    vie.vie_rhs_dipoles_h(h, pos, mom, h_t)
    bj = np.empty((2, 2, 12) + g.shape, dtype=np.complex128)
    vie.vie_jm_rhs(h, e_t, h_t, bj)
    assert rel(bj[:, 0], b) <= 1e-15 and not np.any(bj[:, 1])  # c_e chi e_inc up to the product's rounding order
    xj = np.empty_like(bj)
    rc, _ = vie.vie_jm_solve(h, bj, xj, tol=1e-11, restart=60, maxit=20)
    assert rc == vie.VIE_OK
    x = np.empty_like(b)
    rc, _ = vie.vie_solve(h, b, x, tol=1e-11, restart=60, maxit=20, mode=vie.VIE_SOLVE_FP64)
    h.close()
    assert rc == vie.VIE_OK
    assert not np.any(xj[:, 1])
    assert rel(xj[:, 0], x) <= 1e-9


def test_jm_duality_on_the_gpu(vie):
    """A purely magnetic scatterer (eps = 1, mu) in (e, h) carries m' = j of the dielectric scatterer
    eps = mu in (eta0 h, -e / eta0): the GPU JM solve against the GPU dielectric solve."""
    g = Grid(7, 6, 5, 0.005, 0.005, 0.005)
    mr, mi = random_permeability(g, 61, nonmagnetic_fraction=0.2)
    one = np.ones(g.shape)
    hm = handle(vie, g, one, 0.0 * one, mr, mi)
    hd = handle(vie, g, mr, mi * (2 * np.pi * F * EPS0))
    rng = np.random.Generator(np.random.PCG64(9))
    shp = (1, 12) + g.shape
    e_t = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    h_t = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / J.ETA0
    bj = np.empty((1, 2, 12) + g.shape, dtype=np.complex128)
    vie.vie_jm_rhs(hm, e_t, h_t, bj)
    xj = np.empty_like(bj)
    rc, _ = vie.vie_jm_solve(hm, bj, xj, tol=1e-11, restart=60, maxit=20)
    assert rc == vie.VIE_OK
    # b = c_e chi e2 of the dielectric twin (mu = 1: the first half of its JM right-hand side)
    e2 = np.ascontiguousarray(J.ETA0 * h_t)
    bt = np.empty_like(bj)
    vie.vie_jm_rhs(hd, e2, np.zeros_like(e2), bt)
    bd = np.ascontiguousarray(bt[:, 0])
    xd = np.empty_like(bd)
    rc, _ = vie.vie_solve(hd, bd, xd, tol=1e-11, restart=60, maxit=20, mode=vie.VIE_SOLVE_FP64)
    hm.close()
    hd.close()
    assert rc == vie.VIE_OK
    assert np.max(np.abs(xj[:, 0])) == 0.0
    assert rel(xj[:, 1], xd) <= 1e-9


@pytest.mark.parametrize("mode", ["fp64", "fp32_refine"])
def test_jm_solve_matches_oracle_gmres_on_a_sphere(vie, mode):
    """A magnetodielectric sphere (eps_r 50, sigma 0.5 S/m, mu_r 2 - 0.5 i) at 10^3 in a plane wave:
    the GPU solution (FP64, or FP32 inner solves with FP64 refinement), fields and absorbed power
    against the oracle's GMRES at the same tolerance."""
    n = 10
    hgt = 0.2 / n
    g = Grid(n, n, n, hgt, hgt, hgt)
    eps, sig = sphere_phantom(g, 0.1, 50.0, 0.5)
    inside = eps != 1.0
    mr, mi = np.where(inside, 2.0, 1.0), np.where(inside, 0.5, 0.0)
    prob = J.MagProblem(g, F, eps, sig, mr, mi)
    Nop, Kop = ops(g)
    k0 = prob.k0
    e_t = OR.planewave_tested(g, k0, pol=(1.0, 0.0, 0.0))[None]
    h_t = OR.planewave_tested(g, k0, pol=(0.0, 1.0 / J.ETA0, 0.0))[None]
    b = J.rhs(prob, e_t, h_t)
    xr, info = OS.gmres(lambda v: J.apply_PA(prob, Nop, Kop, v), J.apply_Pinv(prob, b), tol=1e-10, restart=100,
                        maxit=10)
    assert info["converged"]
    h = handle(vie, g, eps, sig, mr, mi)
    x = np.empty_like(b)
    m = vie.VIE_SOLVE_FP64 if mode == "fp64" else vie.VIE_SOLVE_FP32_REFINE
    rc, _ = vie.vie_jm_solve(h, np.ascontiguousarray(b), x, tol=1e-10, restart=100, maxit=10 if mode == "fp64" else 30,
                             mode=m)
    assert rc == vie.VIE_OK
    ec = np.empty_like(e_t)
    hc = np.empty_like(h_t)
    P = vie.vie_jm_fields(h, x, np.ascontiguousarray(e_t), np.ascontiguousarray(h_t), ec, hc)
    h.close()
    assert rel(x, xr) <= 1e-8
    er, hr = J.fields(prob, Nop, Kop, xr, e_t, h_t)
    assert rel(ec, er) <= 1e-8 and rel(hc, hr) <= 1e-8
    _, Pr = J.absorbed_power(prob, xr)
    assert abs(P[0] - Pr[0]) <= 1e-8 * abs(Pr[0])


def test_jm_sphere_absorbed_power_vs_mie(vie):
    """Section V-A's sphere check for the full JM-VIE: a magnetodielectric sphere's absorbed power
    (electric + magnetic loss) against the Mie series, the error shrinking under refinement."""
    mu_s = 2.0 - 0.5j
    Pm = mie.absorbed_power(50.0, 0.5, 0.1, F, mu=mu_s)
    errs = []
    for n in (16, 24, 32):
        hgt = 0.2 / n
        g = Grid(n, n, n, hgt, hgt, hgt)
        eps, sig = sphere_phantom(g, 0.1, 50.0, 0.5)
        inside = eps != 1.0
        h = handle(vie, g, eps, sig, np.where(inside, mu_s.real, 1.0), np.where(inside, -mu_s.imag, 0.0))
        shp = (1, 12) + g.shape
        e_t = np.empty(shp, dtype=np.complex128)
        h_t = np.empty(shp, dtype=np.complex128)
        vie.vie_rhs_planewave(h, [1.0, 0.0, 0.0], [0.0, 0.0, 1.0], e_t[0], None)
        vie.vie_rhs_planewave(h, [0.0, 1.0 / J.ETA0, 0.0], [0.0, 0.0, 1.0], h_t[0], None)
        b = np.empty((1, 2, 12) + g.shape, dtype=np.complex128)
        vie.vie_jm_rhs(h, e_t, h_t, b)
        x = np.empty_like(b)
        rc, _ = vie.vie_jm_solve(h, b, x, tol=1e-7, restart=60, maxit=20)
        assert rc == vie.VIE_OK
        P = vie.vie_jm_fields(h, x, e_t, h_t)
        h.close()
        errs.append(abs(P[0] - Pm) / Pm)
    assert errs[0] < 0.15 and errs[1] < errs[0] and errs[2] < errs[1], errs


def test_jm_invalid_arguments(vie):
    g = Grid(4, 4, 4, 0.005, 0.005, 0.005)
    eps, sig = random_tissue(g, 2)
    h = handle(vie, g, eps, sig)
    bad = np.ones(g.shape)
    with pytest.raises(vie.VieError):
        vie.vie_set_permeability(h, -bad, 0 * bad)  # mu' <= 0
    with pytest.raises(vie.VieError):
        vie.vie_set_permeability(h, bad, -bad)  # mu'' < 0
    x = np.zeros((1, 2, 12) + g.shape, dtype=np.complex128)
    with pytest.raises(vie.VieError):
        vie.vie_jm_matvec(h, x, x.copy(), vie.VIE_OP_NSCAT)
    x[0, 0, 0, 1, 1, 1] = 1.0
    with pytest.raises(vie.VieError) as e:  # the K block has no BF16x3 z pass
        vie.vie_jm_solve(h, x, x.copy(), mode=vie.VIE_SOLVE_BF16X3_REFINE)
    assert e.value.code == vie.VIE_EINVAL
    h.close()
    hp = vie.vie_setup((4, 4, 4, 0.005, 0.005, 0.005), F, eps, sig, vie.VIE_SETUP_PWC)
    with pytest.raises(vie.VieError):
        vie.vie_set_permeability(hp, bad, 0 * bad)
    hp.close()
