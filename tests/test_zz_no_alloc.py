"""vie_matvec_noalloc: the matvec for callers that cannot allocate GPU memory at call time.

It must give the same result as vie_matvec (the tolerances of the parity tests:
1e-12 relative in FP64, 1e-5 in FP32) on two calls in a row, since the static
scratch array keeps the previous call's contents; and it must refuse, without
touching anything, calls whose scratch would not fit or whose buffers are on the host.
The file name makes pytest collect it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import Grid, random_coefficients, random_tissue  # noqa: E402


@pytest.fixture(scope="module")
def vie():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_02196_gb300 as v

    v.build()
    return v


def rel(a, b):
    return float((a - b).abs().norm() / b.abs().norm())


@pytest.mark.parametrize("shape,nrhs,precision", [((7, 6, 9), 2, "fp64"), ((16, 16, 16), 3, "fp32"),
                                                  ((12, 10, 6), 2, "fp32")])
def test_noalloc_matches_matvec_twice(vie, shape, nrhs, precision):
    g = Grid(*shape, 0.004, 0.005, 0.0045)
    eps, sig = random_tissue(g, seed=sum(shape) + nrhs)
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), 298e6, eps, sig)
    prec = vie.VIE_FP64 if precision == "fp64" else vie.VIE_FP32
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    tol = 1e-12 if precision == "fp64" else 1e-5
    for op in (vie.VIE_OP_A, vie.VIE_OP_PA):
        xs = [torch.from_numpy(random_coefficients(g, nrhs, seed=s)).to("cuda", dt) for s in (3, 4)]
        for x in xs:  # two calls in a row, different inputs
            ref = torch.empty_like(x)
            vie.vie_matvec(h, x, ref, prec, op)
            out = torch.full_like(x, float("nan"))
            vie.vie_matvec_noalloc(h, x, out, prec, op)
            torch.cuda.synchronize()
            assert torch.isfinite(torch.view_as_real(out)).all()
            assert rel(out, ref) <= tol
    h.close()


def test_noalloc_rejects_oversize_and_host_buffers(vie):
    g = Grid(32, 32, 32, 0.004, 0.004, 0.004)
    eps, sig = random_tissue(g, seed=5)
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), 128e6, eps, sig)
    big = torch.zeros((8, 12) + g.shape, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(big)
    with pytest.raises(vie.VieError) as e:
        vie.vie_matvec_noalloc(h, big, out, vie.VIE_FP64, vie.VIE_OP_A)
    assert e.value.code == vie.VIE_EINVAL and "static scratch" in str(e.value)
    xh = np.zeros((1, 12) + g.shape, dtype=np.complex128)
    with pytest.raises(vie.VieError) as e:
        vie.vie_matvec_noalloc(h, xh, np.zeros_like(xh), vie.VIE_FP64, vie.VIE_OP_A)
    assert e.value.code == vie.VIE_EINVAL
    # a call that fits still works after the refusals
    x = torch.ones((1, 12) + g.shape, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    ref = torch.empty_like(x)
    vie.vie_matvec_noalloc(h, x, y, vie.VIE_FP32, vie.VIE_OP_A)
    vie.vie_matvec(h, x, ref, vie.VIE_FP32, vie.VIE_OP_A)
    torch.cuda.synchronize()
    assert rel(y, ref) <= 1e-5
    h.close()


def test_noalloc_just_under_the_limit(vie):
    """The scratch check counts only the spectrum the call's path uses: on the fused xy path
    (square xy circulant <= 128) that is nrhs * 12 * nz * Ly * Lx values.  16 x 16 x 31 voxels
    (circulant 32 x 32 x 64), FP32: 22 right-hand sides need 682 * 12 * 32 * 32 * 8 + 256 bytes,
    just under 64 MiB, and run; 23 do not fit and are refused."""
    g = Grid(16, 16, 31, 0.004, 0.004, 0.004)
    eps, sig = random_tissue(g, seed=9)
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), 298e6, eps, sig)
    need = 22 * 31 * 12 * 32 * 32 * 8 + 256
    assert need <= 64 << 20 < need + 31 * 12 * 32 * 32 * 8
    x = torch.from_numpy(random_coefficients(g, 22, seed=12)).to("cuda", torch.complex64)
    for _ in range(2):
        out = torch.full_like(x, float("nan"))
        ref = torch.empty_like(x)
        vie.vie_matvec_noalloc(h, x, out, vie.VIE_FP32, vie.VIE_OP_PA)
        vie.vie_matvec(h, x, ref, vie.VIE_FP32, vie.VIE_OP_PA)
        torch.cuda.synchronize()
        assert rel(out, ref) <= 1e-5
    x23 = torch.zeros((23, 12) + g.shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(vie.VieError) as e:
        vie.vie_matvec_noalloc(h, x23, torch.zeros_like(x23), vie.VIE_FP32, vie.VIE_OP_PA)
    assert e.value.code == vie.VIE_EINVAL and "static scratch" in str(e.value)
    h.close()
