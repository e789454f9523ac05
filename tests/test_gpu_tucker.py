"""Tucker compression of the Green tensors on the GPU (vie_green_tucker) against the oracle's truncated
HOSVD (oracle/tucker.py) and the exact operator.

What is unique and compared: the error bound ||T - T~|| <= tol ||T|| per tensor (checked on the host
from the reconstruction the library returns), ranks at least the truncated-SVD ranks of the same
criterion (which are minimal) and close to them, and the matvec / solve with the compressed Green
function within a small multiple of tol of the exact ones.  The factors themselves are not unique.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import operator as O  # noqa: E402
from oracle import tucker as OT  # noqa: E402
from synth import Grid, random_coefficients, random_tissue, sphere_phantom  # noqa: E402

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


def handle(vie, g, eps, sig):
    return vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), F, eps, sig)


@pytest.mark.parametrize("shape,tol", [((12, 12, 12), 1e-6), ((9, 7, 11), 1e-4), ((20, 16, 24), 1e-7)])
def test_tucker_bound_and_ranks(vie, shape, tol):
    g = Grid(*shape, 0.004, 0.005, 0.0045)
    eps, sig = random_tissue(g, 3)
    h = handle(vie, g, eps, sig)
    T = np.empty((60,) + g.shape, dtype=np.complex128)
    vie.vie_green_toeplitz(h, T)
    _, b0 = vie.vie_info(h)
    ranks, err, nbytes = vie.vie_green_tucker(h, tol, apply=True)
    _, b1 = vie.vie_info(h)  # (before the copy below, which stages through handle memory)
    R = np.empty_like(T)
    vie.vie_green_toeplitz(h, R)  # now the reconstruction
    h.close()
    for t in range(60):
        e = np.linalg.norm(R[t] - T[t]) / np.linalg.norm(T[t])
        assert e <= tol, (t, e)
        assert abs(e - err[t]) <= 1e-3 * tol + 1e-14  # the library's own error report
        _, Us = OT.hosvd(T[t], tol)
        r_svd = [Us[2].shape[1], Us[1].shape[1], Us[0].shape[1]]  # (x, y, z)
        assert all(ranks[t][k] >= r_svd[k] for k in range(3)), (t, ranks[t], r_svd)
        assert all(ranks[t][k] <= r_svd[k] + 3 for k in range(3)), (t, ranks[t], r_svd)
    nz, ny, nx = g.shape
    expect = 16 * sum(int(rx * ry * rz + nx * rx + ny * ry + nz * rz) for rx, ry, rz in ranks)
    assert nbytes == expect
    assert b1 == b0 - 60 * g.nv * 16 + nbytes


def test_tucker_matvec_and_solve(vie):
    """The FP64 matvec with the compressed Green function against the oracle's exact operator, and a
    sphere solve before and after compression."""
    n = 16
    hgt = 0.2 / n
    g = Grid(n, n, n, hgt, hgt, hgt)
    eps, sig = sphere_phantom(g, 0.1, 50.0, 0.5)
    tol = 1e-6
    h = handle(vie, g, eps, sig)
    e_inc = np.empty((1, 12) + g.shape, dtype=np.complex128)
    b = np.empty_like(e_inc)
    vie.vie_rhs_planewave(h, [1.0, 0.0, 0.0], [0.0, 0.0, 1.0], e_inc[0], b[0])
    x0 = np.empty_like(b)
    rc, _ = vie.vie_solve(h, b, x0, tol=1e-10, restart=80, maxit=20, mode=vie.VIE_SOLVE_FP64)
    assert rc == vie.VIE_OK
    ranks, err, nbytes = vie.vie_green_tucker(h, tol, apply=True)
    assert np.all(err <= tol)
    v = random_coefficients(g, 2, seed=4)
    y = np.empty_like(v)
    vie.vie_matvec(h, v, y, vie.VIE_FP64, vie.VIE_OP_NSCAT)
    x1 = np.empty_like(b)
    rc, _ = vie.vie_solve(h, b, x1, tol=1e-10, restart=80, maxit=20, mode=vie.VIE_SOLVE_FP64)
    h.close()
    assert rc == vie.VIE_OK
    prob = O.Problem(g, F, eps, sig)
    Nop = O.NOperator(g, prob.k0)
    G = prob.gram_vector()[:, None, None, None]
    ref = Nop.apply(v) - G * v
    assert rel(y, ref) <= 10 * tol
    assert rel(x1, x0) <= 100 * tol
    assert nbytes < 0.5 * 60 * g.nv * 16  # at 16^3 the form is already smaller than the table


def test_tucker_recompress_pwc_and_arguments(vie):
    """A second compression starts from the first one's reconstruction (the table is gone after
    VIE_TUCKER_APPLY) and keeps the bound against the original within the sum of the tolerances; a
    PWC handle's matvec runs on the compressed tensors; out-of-range tolerances are refused."""
    g = Grid(10, 9, 11, 0.005, 0.005, 0.005)
    eps, sig = random_tissue(g, 8)
    h = handle(vie, g, eps, sig)
    T = np.empty((60,) + g.shape, dtype=np.complex128)
    vie.vie_green_toeplitz(h, T)
    vie.vie_green_tucker(h, 1e-6, apply=True)
    ranks2, err2, _ = vie.vie_green_tucker(h, 1e-4, apply=True)
    R = np.empty_like(T)
    vie.vie_green_toeplitz(h, R)
    for t in range(60):
        assert np.linalg.norm(R[t] - T[t]) <= (1e-4 + 1e-6) * np.linalg.norm(T[t])
    for bad in (0.0, 1e-8, 1.0, float("nan")):
        with pytest.raises(vie.VieError) as e:
            vie.vie_green_tucker(h, bad)
        assert e.value.code == vie.VIE_EINVAL
    h.close()
    # PWC: the l = 1 sub-block of the compressed Green function against the oracle's exact operator
    tol = 1e-6
    hp = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), F, eps, sig, vie.VIE_SETUP_PWC)
    vie.vie_green_tucker(hp, tol, apply=True)
    x = random_coefficients(g, 2, seed=9, ncomp=3)
    y = np.empty_like(x)
    vie.vie_matvec(hp, x, y, vie.VIE_FP64, vie.VIE_OP_PA)
    hp.close()
    prob = O.Problem(g, F, eps, sig)
    Nop = O.NOperator(g, prob.k0)
    xf = np.zeros((2, 12) + g.shape, dtype=complex)
    xf[:, 0::4] = x
    ref = O.apply_PA_pwc(prob, Nop, xf)[:, 0::4]
    assert rel(y, ref) <= 10 * tol
