"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (stated per result): FP64 Green tensors and FP64 matvec <= 1e-12 relative
(2-norm over all entries); FP32 matvec <= 1e-5 relative; solutions <= 1e-6 relative
in the current coefficients, fields and absorbed-power maps.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import green as OG  # noqa: E402
from oracle import operator as O  # noqa: E402
from oracle import post as OP  # noqa: E402
from oracle import rhs as OR  # noqa: E402
from oracle import solver as OS  # noqa: E402
from synth import Grid, head_phantom, random_coefficients, random_tissue, ring_dipoles, sphere_phantom  # noqa: E402


@pytest.fixture(scope="module")
def vie():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_02196_gb300 as v

    v.build()
    return v


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def setup(vie, g, freq, eps, sig):
    return vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), freq, eps, sig)


def gpu_matvec(vie, h, x, precision, op):
    dt = torch.complex128 if precision == vie.VIE_FP64 else torch.complex64  # FP32 and BF16X3: complex64
    xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)
    yd = torch.empty_like(xd)
    vie.vie_matvec(h, xd, yd, precision, op)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


PQ = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
LL = [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (2, 4), (3, 3), (3, 4), (4, 4)]


@pytest.mark.parametrize("shape,delta", [((5, 4, 6), (0.004, 0.005, 0.0045)), ((8, 8, 8), (0.003, 0.003, 0.003))])
def test_green_toeplitz_parity(vie, shape, delta):
    """The 60 unique Toeplitz tensors of N - G computed on the GPU vs all-144 oracle entries at every d >= 0."""
    g = Grid(*shape, *delta)
    eps = np.ones(g.shape)
    sig = np.zeros(g.shape)
    freq = 298e6
    h = setup(vie, g, freq, eps, sig)
    out = np.zeros((60,) + g.shape, dtype=np.complex128)
    vie.vie_green_toeplitz(h, out)
    h.close()
    dz, dy, dx = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    D = np.stack([dx.ravel(), dy.ravel(), dz.ravel()], 1)
    T = OG.n_entries(delta, O.k0_of(freq), D)
    dV = np.prod(delta)
    zero = np.all(D == 0, 1)
    ref = np.zeros((60, D.shape[0]), dtype=complex)
    for pqi, (p, q) in enumerate(PQ):
        for lli, (la, lb) in enumerate(LL):
            a, b = 4 * p + la - 1, 4 * q + lb - 1
            v = T[a, b].copy()
            if a == b:
                v -= zero * OG.gram(la, dV)
            ref[10 * pqi + lli] = v
    got = out.reshape(60, -1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape,delta", [((5, 4, 6), (0.004, 0.005, 0.0045)), ((8, 8, 8), (0.003, 0.003, 0.003))])
def test_green_toeplitz_k_parity(vie, shape, delta):
    """The 30 Toeplitz tensors of the K operator computed on the GPU vs the oracle's K entries at
    every d >= 0: P_{10 j + ll}(d) = -eps_pjq K^{(p,la),(q,lb)}(d) for (p, j, q) a permutation."""
    g = Grid(*shape, *delta)
    freq = 298e6
    h = setup(vie, g, freq, np.ones(g.shape), np.zeros(g.shape))
    out = np.zeros((30,) + g.shape, dtype=np.complex128)
    vie.vie_green_toeplitz_k(h, out)
    h.close()
    dz, dy, dx = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    D = np.stack([dx.ravel(), dy.ravel(), dz.ravel()], 1)
    T = OG.k_entries(delta, O.k0_of(freq), D)
    ref = np.zeros((30, D.shape[0]), dtype=complex)
    for j in range(3):
        p, q = (j + 1) % 3, (j + 2) % 3  # eps_{p j q} = -1 for this cyclic choice
        for lli, (la, lb) in enumerate(LL):
            ref[10 * j + lli] = T[4 * p + la - 1, 4 * q + lb - 1]  # -eps_pjq K = +K
    got = out.reshape(30, -1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape,nrhs", [((4, 4, 4), 1), ((7, 5, 9), 2), ((12, 5, 6), 2), ((16, 16, 20), 2),
                                         ((40, 40, 9), 1), ((3, 4, 70), 1)])
def test_k_matvec_parity(vie, shape, nrhs):
    """y = K x (VIE_OP_K, FP64 and FP32: the N operator's transforms with the K block on the octant
    K spectra) vs the oracle's K operator (its own K tensors, circulant + FFT), on grids that take the
    fused xy kernels (16 x 16 x 20, 40 x 40 x 9) and the line transforms (Lz = 256 for 3 x 4 x 70)."""
    g = Grid(*shape, 0.004, 0.005, 0.0045)
    eps, sig = random_tissue(g, seed=sum(shape) + 1)
    freq = 298e6
    h = setup(vie, g, freq, eps, sig)
    x = random_coefficients(g, nrhs, seed=21 + nrhs)
    y = gpu_matvec(vie, h, x, vie.VIE_FP64, vie.VIE_OP_K)
    y32 = gpu_matvec(vie, h, x, vie.VIE_FP32, vie.VIE_OP_K)
    with pytest.raises(vie.VieError) as e:
        gpu_matvec(vie, h, x, vie.VIE_BF16X3, vie.VIE_OP_K)
    assert e.value.code == vie.VIE_EINVAL
    h.close()
    ref = O.KOperator(g, O.k0_of(freq)).apply(x)
    assert rel(y, ref) <= 1e-12
    assert rel(y32, ref) <= 1e-5


@pytest.mark.parametrize("shape", [(6, 5, 4), (9, 7, 6)])
def test_magnetic_post_parity(vie, shape):
    """Tested dipole h_inc, the magnetic field coefficients h = (h_inc + K x) / G, b1+ and W_m vs the
    oracle's (Section II total fields; Section V-D definitions)."""
    g = Grid(*shape, 0.006, 0.005, 0.007)
    eps, sig = random_tissue(g, seed=sum(shape) + 5, air_fraction=0.3)
    freq = 298e6
    prob = O.Problem(g, freq, eps, sig)
    pos, mom = ring_dipoles(2, 0.05)
    h = setup(vie, g, freq, eps, sig)
    hinc = np.zeros((2, 12) + g.shape, dtype=complex)
    vie.vie_rhs_dipoles_h(h, pos, mom, hinc)
    x = random_coefficients(g, 2, seed=sum(shape))
    hc = np.zeros((2, 12) + g.shape, dtype=complex)
    b1 = np.zeros((2,) + g.shape, dtype=complex)
    W = vie.vie_hfields(h, x, hinc, hc, b1)
    h.close()
    hinc_ref = OR.dipoles_tested_h(g, prob.k0, pos, mom)
    assert rel(hinc, hinc_ref) <= 1e-12
    hc_ref = OP.magnetic_fields(prob, O.KOperator(g, prob.k0), x, hinc_ref)
    assert rel(hc, hc_ref) <= 1e-12
    assert rel(b1, OP.b1_plus(hc_ref)) <= 1e-12
    _, W_ref = OP.magnetic_energy(prob, hc_ref)
    assert np.max(np.abs(np.asarray(W) - W_ref) / np.abs(W_ref)) <= 1e-12


# (12, 5, 6) has Lx != Ly (line transforms along x and y), (5, 6, 70) has Lz = 256 and
# (3, 2, 130) Lz = 512 (the FP32 z pass with 2-column tiles); (100, 6, 5) and (6, 100, 5) take the
# two-pass line kernels at length 256 along x, resp. y (the body grid's length), (3, 2, 130) the
# radix-4 line kernel along y (Ly = 4)
# FFT lengths (Lx, Ly, Lz): (8, 8, 8), (16, 16, 32), (32, 32, 16), (32, 32, 32), (32, 16, 16), (16, 16, 256),
# (8, 4, 512), (16, 16, 64), (16, 16, 128), (16, 8, 128), (256, 16, 16), (16, 256, 16): the z-pass
# kernels at every length and tile width, on the fused xy path (square xy circulant) and the line path
CASES = [((4, 4, 4), 1), ((7, 5, 9), 2), ((12, 10, 6), 3), ((16, 16, 16), 1), ((12, 5, 6), 2), ((5, 6, 70), 1),
         ((3, 2, 130), 1), ((6, 5, 20), 2), ((6, 6, 36), 2), ((5, 4, 40), 1), ((100, 6, 5), 2), ((6, 100, 5), 2)]


@pytest.fixture(scope="module")
def cases(vie):
    out = {}
    for shape, R in CASES:
        g = Grid(*shape, 0.004, 0.005, 0.0045)
        eps, sig = random_tissue(g, seed=sum(shape))
        prob = O.Problem(g, 298e6, eps, sig)
        Nop = O.NOperator(g, prob.k0)
        h = setup(vie, g, 298e6, eps, sig)
        x = random_coefficients(g, R, seed=7 + R)
        out[shape] = (g, prob, Nop, h, x)
    yield out
    for v in out.values():
        v[3].close()


@pytest.mark.parametrize("shape", [c[0] for c in CASES])
@pytest.mark.parametrize("op", ["A", "PA", "NSCAT"])
def test_matvec_fp64_parity(vie, cases, shape, op):
    g, prob, Nop, h, x = cases[shape]
    G = prob.gram_vector()[:, None, None, None]
    if op == "A":
        ref, code = O.apply_A(prob, Nop, x), vie.VIE_OP_A
    elif op == "PA":
        ref, code = O.apply_PA(prob, Nop, x), vie.VIE_OP_PA
    else:
        ref, code = Nop.apply(x) - G * x, vie.VIE_OP_NSCAT
    y = gpu_matvec(vie, h, x, vie.VIE_FP64, code)
    assert rel(y, ref) <= 1e-12


@pytest.mark.parametrize("shape", [c[0] for c in CASES])
def test_matvec_fp32_parity(vie, cases, shape):
    g, prob, Nop, h, x = cases[shape]
    G = prob.gram_vector()[:, None, None, None]
    for op, code in (("A", vie.VIE_OP_A), ("PA", vie.VIE_OP_PA), ("NSCAT", vie.VIE_OP_NSCAT)):
        if op == "A":
            ref = O.apply_A(prob, Nop, x)
        elif op == "PA":
            ref = O.apply_PA(prob, Nop, x)
        else:
            ref = Nop.apply(x) - G * x
        y = gpu_matvec(vie, h, x, vie.VIE_FP32, code)
        assert rel(y, ref) <= 1e-5


# BF16x3 block product: each real product within 3 * 2^-16 of exact (bf16 hi/lo splits of both
# operands, the lo x lo term dropped), FP32 transforms and accumulation; bound on the matvec's
# relative 2-norm error: 5e-5
BF16X3_TOL = 5e-5


@pytest.mark.parametrize("shape", [c[0] for c in CASES])
def test_matvec_bf16x3_parity(vie, cases, shape):
    g, prob, Nop, h, x = cases[shape]
    G = prob.gram_vector()[:, None, None, None]
    for op, code in (("A", vie.VIE_OP_A), ("PA", vie.VIE_OP_PA), ("NSCAT", vie.VIE_OP_NSCAT)):
        if op == "A":
            ref = O.apply_A(prob, Nop, x)
        elif op == "PA":
            ref = O.apply_PA(prob, Nop, x)
        else:
            ref = Nop.apply(x) - G * x
        y = gpu_matvec(vie, h, x, vie.VIE_BF16X3, code)
        assert rel(y, ref) <= BF16X3_TOL


def test_matvec_host_buffers_equal_device_buffers(vie, cases):
    g, prob, Nop, h, x = cases[(7, 5, 9)]
    yh = np.zeros_like(x)
    vie.vie_matvec(h, np.ascontiguousarray(x), yh, vie.VIE_FP64, vie.VIE_OP_A)
    yd = gpu_matvec(vie, h, x, vie.VIE_FP64, vie.VIE_OP_A)
    assert np.array_equal(yh, yd)


def test_planewave_and_dipole_rhs_parity(vie):
    g = Grid(6, 7, 5, 0.01, 0.009, 0.011)
    eps, sig = random_tissue(g, seed=31)
    prob = O.Problem(g, 128e6, eps, sig)
    h = setup(vie, g, 128e6, eps, sig)
    d = np.array([0.2, -0.3, 0.93])
    d /= np.linalg.norm(d)
    pol = np.cross(d, [0.0, 1.0, 0.0])
    e = np.zeros((12,) + g.shape, dtype=complex)
    b = np.zeros_like(e)
    vie.vie_rhs_planewave(h, pol, d, e, b)
    e_ref = OR.planewave_tested(g, prob.k0, pol, d)
    assert rel(e, e_ref) <= 1e-12
    assert rel(b, OR.rhs(prob, e_ref)) <= 1e-12
    pos, mom = ring_dipoles(3, 0.06, z=0.01)
    mom[1] = [0.3, -0.2, 0.5]
    ed = np.zeros((3, 12) + g.shape, dtype=complex)
    bd = np.zeros_like(ed)
    vie.vie_rhs_dipoles(h, pos, mom, ed, bd)
    ed_ref = OR.dipoles_tested(g, prob.k0, prob.ce, pos, mom)
    assert rel(ed, ed_ref) <= 1e-12
    assert rel(bd, OR.rhs(prob, ed_ref)) <= 1e-12
    h.close()


@pytest.fixture(scope="module")
def sphere(vie):
    """Config of the Mie check: 16^3 sphere r = 0.1 m, 12.5 mm voxels, eps' = 50, sigma = 0.5, 298 MHz, plane wave."""
    g = Grid(16, 16, 16, 0.0125, 0.0125, 0.0125)
    eps, sig = sphere_phantom(g, 0.1, 50.0, 0.5)
    prob = O.Problem(g, 298e6, eps, sig)
    Nop = O.NOperator(g, prob.k0)
    e_inc = OR.planewave_tested(g, prob.k0)
    b = OR.rhs(prob, e_inc)
    xo, info = OS.gmres(lambda v: O.apply_PA(prob, Nop, v), O.apply_Pinv(prob, b), tol=1e-11, restart=100, maxit=40)
    h = setup(vie, g, 298e6, eps, sig)
    yield g, prob, Nop, e_inc, b, xo, h
    h.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed", "bf16x3"])
def test_solve_parity_sphere(vie, sphere, mode):
    g, prob, Nop, e_inc, b, xo, h = sphere
    bd = torch.from_numpy(b[None].copy()).cuda()
    xd = torch.empty_like(bd)
    m = {"fp64": vie.VIE_SOLVE_FP64, "mixed": vie.VIE_SOLVE_FP32_REFINE, "bf16x3": vie.VIE_SOLVE_BF16X3_REFINE}[mode]
    rc, info = vie.vie_solve(h, bd, xd, tol=1e-8, restart=50, maxit=40, mode=m)
    assert rc == vie.VIE_OK, info
    assert info[0]["resid"] <= 1e-8
    x = xd.cpu().numpy()[0]
    assert rel(x, xo) <= 1e-6
    # fields and absorbed power of the GPU solution vs the oracle post-processing of the same solution
    ed = torch.from_numpy(e_inc[None].copy()).cuda()
    ef = torch.empty_like(ed)
    pa = torch.empty((1,) + g.shape, dtype=torch.float64, device="cuda")
    P = vie.vie_fields(h, xd, ed, ef, pa)
    e_ref = OP.fields(prob, Nop, x, e_inc)
    p_ref, P_ref = OP.absorbed_power(prob, x)
    # FP64 mode: the product at the returned x is the solver's last FP64 one.  Mixed mode: the
    # FP64 product at the refinement point plus the FP32 product of the later correction d,
    # an error of at most about 1e-6 |d| / |x| <= 1e-9, three orders below the 1e-6 field
    # tolerance.
    # (BF16x3 mode: the same FP32 correction of the field map as the mixed mode)
    assert rel(ef.cpu().numpy()[0], e_ref) <= (1e-12 if mode == "fp64" else 1e-9)
    assert rel(pa.cpu().numpy()[0], p_ref) <= 1e-12
    assert abs(P[0] - P_ref) <= 1e-12 * abs(P_ref)
    # and the solution's physics against the oracle solution's
    _, P_or = OP.absorbed_power(prob, xo)
    assert abs(P[0] - P_or) <= 1e-6 * abs(P_or)


def fields_launches(vie, h, x, e, nrhs, shape):
    """vie_fields with the field map; returns (field map, p_abs, P_abs, launches per kernel name)."""
    ef = torch.empty_like(e)
    pa = torch.empty((nrhs,) + shape, dtype=torch.float64, device="cuda")
    vie.vie_stats_reset(0)
    P = vie.vie_fields(h, x, e, ef, pa)
    torch.cuda.synchronize()
    _, st = vie.vie_stats_read()
    return ef, pa, P, {k: v[0] for k, v in st.items()}


def f64_matvec_launches(st):
    return sum(n for k, n in st.items() if k.endswith("_f64"))


@pytest.mark.parametrize("shape", [(12, 10, 8), (9, 7, 6)])
def test_fields_reuse_the_solver_product(vie, shape):
    """vie_fields after vie_solve takes (N - G) x from the solver's last FP64 residual matvec
    (plus the FP32 product of x - x1 when x moved after it) instead of a new FP64 matvec, when
    |x - x1| <= 1e-3 |x| for every right-hand side and nrhs matches; otherwise the FP64 matvec.
    Reference: a second handle of the same problem that never solved (always the FP64 matvec)."""
    g = Grid(*shape, 0.006, 0.005, 0.007)
    eps, sig = random_tissue(g, seed=sum(shape), air_fraction=0.3)
    h, h2 = setup(vie, g, 128e6, eps, sig), setup(vie, g, 128e6, eps, sig)
    R = 3
    pos, mom = ring_dipoles(R, 0.05)
    e = torch.zeros((R, 12) + g.shape, dtype=torch.complex128, device="cuda")
    b = torch.zeros_like(e)
    vie.vie_rhs_dipoles(h, pos, mom, e, b)
    x = torch.zeros_like(b)

    # mixed solve: the field map is the cached FP64 product plus an FP32 correction
    rc, _ = vie.vie_solve(h, b, x, tol=1e-7, restart=30, maxit=40, mode=vie.VIE_SOLVE_FP32_REFINE)
    assert rc == vie.VIE_OK
    ef, pa, P, st = fields_launches(vie, h, x, e, R, g.shape)
    ef2, pa2, P2, st2 = fields_launches(vie, h2, x, e, R, g.shape)
    assert st.get("fields_diff") == 1 and f64_matvec_launches(st) == 0, st
    assert "fields_diff" not in st2 and f64_matvec_launches(st2) > 0, st2
    assert rel(ef.cpu().numpy(), ef2.cpu().numpy()) <= 1e-9  # FP32 term: <= ~1e-6 |d| / |x|, |d| <= 1e-3 |x|
    assert torch.equal(pa, pa2) and P == P2  # the absorbed power depends on x alone

    # x moved by more than 1e-3 |x|: the FP64 matvec, the same bits as the reference handle
    x3 = x * 1.01
    ef, _, _, st = fields_launches(vie, h, x3, e, R, g.shape)
    ef2, _, _, _ = fields_launches(vie, h2, x3, e, R, g.shape)
    assert st.get("fields_diff") == 1 and f64_matvec_launches(st) > 0, st
    assert torch.equal(ef, ef2)

    # a solve that keeps no point (flags bit 2): the FP64 matvec, the same bits as the reference
    x4 = torch.zeros_like(b)
    rc, _ = vie.vie_solve(h, b, x4, tol=1e-7, restart=30, maxit=40, mode=vie.VIE_SOLVE_FP32_REFINE,
                          keep_point=False)
    assert rc == vie.VIE_OK and rel(x4.cpu().numpy(), x.cpu().numpy()) <= 1e-6  # both meet tol 1e-7
    ef, _, _, st = fields_launches(vie, h, x4, e, R, g.shape)
    ef2, _, _, _ = fields_launches(vie, h2, x4, e, R, g.shape)
    assert "fields_diff" not in st and f64_matvec_launches(st) > 0, st
    assert torch.equal(ef, ef2)

    # another number of right-hand sides: the FP64 matvec
    rc, _ = vie.vie_solve(h, b, x, tol=1e-7, restart=30, maxit=40, mode=vie.VIE_SOLVE_FP32_REFINE)
    xs, es = x[:2].contiguous(), e[:2].contiguous()
    ef, _, _, st = fields_launches(vie, h, xs, es, 2, g.shape)
    ef2, _, _, _ = fields_launches(vie, h2, xs, es, 2, g.shape)
    assert "fields_diff" not in st and f64_matvec_launches(st) > 0, st
    assert torch.equal(ef, ef2)

    # FP64 solve: its last FP64 residual is at the returned x, so the cached product is used as is
    rc, _ = vie.vie_solve(h, b, x, tol=1e-7, restart=30, maxit=40, mode=vie.VIE_SOLVE_FP64)
    assert rc == vie.VIE_OK
    ef, _, _, st = fields_launches(vie, h, x, e, R, g.shape)
    ef2, _, _, _ = fields_launches(vie, h2, x, e, R, g.shape)
    assert st.get("fields_diff") == 1 and f64_matvec_launches(st) == 0, st
    assert not any(k.endswith("_f32") for k in st), st  # no correction term
    assert rel(ef.cpu().numpy(), ef2.cpu().numpy()) <= 1e-13
    h.close()
    h2.close()


def test_batch_independence_and_guess(vie):
    """A right-hand side gives the same bits alone and inside a batch; a converged guess returns at once."""
    g = Grid(8, 8, 8, 0.005, 0.005, 0.005)
    eps, sig = random_tissue(g, seed=41, air_fraction=0.3)
    h = setup(vie, g, 128e6, eps, sig)
    prob = O.Problem(g, 128e6, eps, sig)
    pos, mom = ring_dipoles(3, 0.05)
    b = np.zeros((3, 12) + g.shape, dtype=complex)
    vie.vie_rhs_dipoles(h, pos, mom, None, b)
    bd = torch.from_numpy(b).cuda()
    xb = torch.empty_like(bd)
    rc, info = vie.vie_solve(h, bd, xb, tol=1e-7, restart=30, maxit=30, mode=vie.VIE_SOLVE_FP32_REFINE)
    assert rc == vie.VIE_OK
    x1 = torch.empty_like(bd[1:2])
    rc1, info1 = vie.vie_solve(h, bd[1:2].contiguous(), x1, tol=1e-7, restart=30, maxit=30,
                               mode=vie.VIE_SOLVE_FP32_REFINE)
    assert torch.equal(x1[0], xb[1])
    rc2, info2 = vie.vie_solve(h, bd, xb, tol=1e-6, restart=30, maxit=30, mode=vie.VIE_SOLVE_FP32_REFINE, guess=True)
    assert rc2 == vie.VIE_OK and all(i["iterations"] == 0 for i in info2)
    h.close()


@pytest.mark.parametrize("case", ["b_zero_in_air", "b_in_air", "guess_in_air"])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_solve_on_support(vie, case, mode):
    """The solver works on each row's span of the voxels where chi, b or the guess is non-zero
    (air elsewhere): solutions match the oracle's GMRES on the full grid to 1e-6, and the
    solution is exactly zero outside the span.  The map has an air slab (x < 2), an air
    plane (z = 0, so whole rows are empty) and scattered air voxels."""
    g = Grid(7, 5, 4, 0.004, 0.005, 0.0045)
    eps, sig = random_tissue(g, seed=77, air_fraction=0.15)
    eps[:, :, :2], sig[:, :, :2] = 1.0, 0.0
    eps[0], sig[0] = 1.0, 0.0
    prob = O.Problem(g, 298e6, eps, sig)
    Nop = O.NOperator(g, prob.k0)
    rng = np.random.Generator(np.random.PCG64(5))
    R = 2
    b = (rng.standard_normal((R, 12) + g.shape) + 1j * rng.standard_normal((R, 12) + g.shape))
    air = prob.chi == 0
    if case != "b_in_air":
        b = b * (~air)
    else:
        b[:, :, 0, 1, 0] = 0.3 + 0.2j  # one air voxel with a source, inside an empty row
    h = setup(vie, g, 298e6, eps, sig)
    m = vie.VIE_SOLVE_FP64 if mode == "fp64" else vie.VIE_SOLVE_FP32_REFINE
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    guess = case == "guess_in_air"
    if guess:
        xd[:, :, 0, 2, 1] = 0.5j  # a guess that is non-zero in an air voxel of an empty row
    rc, info = vie.vie_solve(h, bd, xd, tol=1e-9, restart=40, maxit=60, mode=m, guess=guess)
    h.close()
    assert rc == vie.VIE_OK, info
    x = xd.cpu().numpy()
    for r in range(R):
        xo, oi = OS.gmres(lambda v: O.apply_PA(prob, Nop, v), O.apply_Pinv(prob, b[r]), tol=1e-12, restart=200,
                          maxit=20)
        assert oi["converged"]
        assert rel(x[r], xo) <= 1e-6
    if case == "b_zero_in_air":
        # rows with no tissue carry no unknowns: the solution there is exactly zero
        assert np.all(x[:, :, 0] == 0) and np.all(x[:, :, :, :, :2] == 0)


def test_full_size_fp32_matvec_sampled(vie):
    """64^3 head phantom, 3 mm, 298 MHz, 16 right-hand sides (the benchmark's batched FP32 matvec):
    x has a few non-zero voxels per right-hand side; y at sampled voxels from oracle Galerkin entries."""
    g = Grid(64, 64, 64, 0.003, 0.003, 0.003)
    eps, sig = head_phantom(g)
    prob = O.Problem(g, 298e6, eps, sig)
    h = setup(vie, g, 298e6, eps, sig)
    rng = np.random.Generator(np.random.PCG64(99))
    R = 16
    x = np.zeros((R, 12) + g.shape, dtype=np.complex64)
    src = []
    for r in range(R):
        vox = rng.integers(0, 64, size=(2, 3))
        src.append(vox)
        for v in vox:
            x[r, :, v[2], v[1], v[0]] = (rng.standard_normal(12) + 1j * rng.standard_normal(12)).astype(np.complex64)
    y = gpu_matvec(vie, h, x, vie.VIE_FP32, vie.VIE_OP_A)
    h.close()
    G = prob.gram_vector()
    for r in (0, 7, 15):
        ms = rng.integers(0, 64, size=(12, 3))
        ms = np.concatenate([ms, src[r][:1]])  # include a source voxel (self term)
        D = np.array([m - n for m in ms for n in src[r]])
        T = OG.n_entries((g.dx, g.dy, g.dz), prob.k0, D).reshape(12, 12, len(ms), len(src[r]))
        ref = np.zeros((len(ms), 12), dtype=complex)
        for i, m in enumerate(ms):
            nx = sum(T[:, :, i, k] @ x[r, :, n[2], n[1], n[0]].astype(complex) for k, n in enumerate(src[r]))
            xm = x[r, :, m[2], m[1], m[0]].astype(complex)
            ref[i] = prob.eps[m[2], m[1], m[0]] * G * xm - prob.chi[m[2], m[1], m[0]] * nx
        got = np.array([y[r, :, m[2], m[1], m[0]] for m in ms])
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_body_matvec_sampled(vie, precision):
    """128 x 128 x 256 body stack, 5 mm, 128 MHz (circulant 256 x 256 x 512: line transforms along x
    and y, the 512-point z pass): a few non-zero voxels per right-hand side, y at sampled voxels
    from oracle Galerkin entries; 1e-5 (FP32) / 1e-12 (FP64) relative."""
    from synth import body_phantom

    g = Grid(128, 128, 256, 0.005, 0.005, 0.005)
    eps, sig = body_phantom(g)
    prob = O.Problem(g, 128e6, eps, sig)
    h = setup(vie, g, 128e6, eps, sig)
    rng = np.random.Generator(np.random.PCG64(17))
    R = 2
    dt = np.complex64 if precision == "fp32" else np.complex128
    x = np.zeros((R, 12) + g.shape, dtype=dt)
    src = []
    for r in range(R):
        vox = np.stack([rng.integers(0, 128, 2), rng.integers(0, 128, 2), rng.integers(0, 256, 2)], 1)
        src.append(vox)
        for v in vox:
            x[r, :, v[2], v[1], v[0]] = (rng.standard_normal(12) + 1j * rng.standard_normal(12)).astype(dt)
    y = gpu_matvec(vie, h, x, vie.VIE_FP32 if precision == "fp32" else vie.VIE_FP64, vie.VIE_OP_A)
    h.close()
    G = prob.gram_vector()
    tol = 1e-5 if precision == "fp32" else 1e-12
    for r in range(R):
        ms = np.stack([rng.integers(0, 128, 8), rng.integers(0, 128, 8), rng.integers(0, 256, 8)], 1)
        ms = np.concatenate([ms, src[r][:1]])
        D = np.array([m - n for m in ms for n in src[r]])
        T = OG.n_entries((g.dx, g.dy, g.dz), prob.k0, D).reshape(12, 12, len(ms), len(src[r]))
        ref = np.zeros((len(ms), 12), dtype=complex)
        for i, m in enumerate(ms):
            nx = sum(T[:, :, i, k] @ x[r, :, n[2], n[1], n[0]].astype(complex) for k, n in enumerate(src[r]))
            xm = x[r, :, m[2], m[1], m[0]].astype(complex)
            ref[i] = prob.eps[m[2], m[1], m[0]] * G * xm - prob.chi[m[2], m[1], m[0]] * nx
        got = np.array([y[r, :, m[2], m[1], m[0]] for m in ms])
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


def test_invalid_arguments(vie):
    g = Grid(3, 3, 3, 0.01, 0.01, 0.01)
    eps, sig = random_tissue(g, seed=1)
    with pytest.raises(vie.VieError) as e:
        vie.vie_setup((3, 3, 0, 0.01, 0.01, 0.01), 1e8, eps, sig)
    assert e.value.code == vie.VIE_EINVAL
    bad = eps.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(vie.VieError):
        vie.vie_setup((3, 3, 3, 0.01, 0.01, 0.01), 1e8, bad, sig)
    h = setup(vie, g, 1e8, eps, sig)
    x = np.zeros((1, 12) + g.shape, dtype=complex)
    with pytest.raises(vie.VieError):
        vie.vie_matvec(h, x, x, vie.VIE_FP64, vie.VIE_OP_A)
    with pytest.raises(vie.VieError):
        vie.vie_matvec(h, x, np.zeros_like(x), 7, vie.VIE_OP_A)
    with pytest.raises(vie.VieError):
        vie.vie_solve(h, x, np.zeros_like(x), tol=2.0)
    h.close()
