"""Dense-input parity of the batched matvec at the benchmark's kernel shapes, with the Green
tensors both computed on the GPU (vie_setup) and supplied by the oracle
(vie_setup_green_external), so that a fault in the matvec and a fault in the Green setup
are told apart.

Each case runs 16 right-hand sides of N(0,1) + iN(0,1) coefficients at every unknown, on
grids whose FFT lengths instantiate the kernels of the 64^3 benchmark: the 128-point fused xy
transforms (Lx = Ly = 128), the 128-point z pass (Lz = 128) and the 64-point xy transforms.
Tolerances (relative 2-norm over all entries): FP64 <= 1e-12, FP32 <= 1e-5.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import green as OG  # noqa: E402
from oracle import operator as O  # noqa: E402
from synth import Grid, random_coefficients, random_tissue  # noqa: E402

R = 16
# (shape (nx, ny, nz), FFT lengths): (33, 33, 4) -> (128, 128, 8); (4, 4, 33) -> (8, 8, 128);
# (32, 32, 5) -> (64, 64, 16); (17, 20, 9) -> (64, 64, 32) with a ragged xy tail (nx != ny)
SHAPES = [(33, 33, 4), (4, 4, 33), (32, 32, 5), (17, 20, 9)]


@pytest.fixture(scope="module")
def vie():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_02196_gb300 as v

    v.build()
    return v


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: "x".join(map(str, s)))
def case(vie, request):
    shape = request.param
    g = Grid(*shape, 0.003, 0.0035, 0.004)
    freq = 298e6
    eps, sig = random_tissue(g, seed=sum(shape) + 100, air_fraction=0.1)
    prob = O.Problem(g, freq, eps, sig)
    T = OG.toeplitz_tensors(g, prob.k0)
    Nop = O.NOperator(g, prob.k0, T)
    grid = (g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)
    h_dev = vie.vie_setup(grid, freq, eps, sig)
    h_ext = vie.vie_setup_green_external(grid, freq, eps, sig, np.ascontiguousarray(T.reshape((144,) + T.shape[2:])))
    x = random_coefficients(g, R, seed=sum(shape) + 7)
    G = prob.gram_vector()[:, None, None, None]
    refs = {"A": O.apply_A(prob, Nop, x), "PA": O.apply_PA(prob, Nop, x), "NSCAT": Nop.apply(x) - G * x}
    yield g, x, refs, h_dev, h_ext
    h_dev.close()
    h_ext.close()


def gpu_matvec(vie, h, x, precision, op):
    dt = torch.complex128 if precision == vie.VIE_FP64 else torch.complex64
    xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)
    yd = torch.empty_like(xd)
    vie.vie_matvec(h, xd, yd, precision, op)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


def test_fft_lengths(vie, case):
    g, _, _, h_dev, h_ext = case
    L = vie.vie_info(h_dev)[0]
    assert L == vie.vie_info(h_ext)[0]
    assert all(Li >= 2 * n - 1 for Li, n in zip(L, (g.nx, g.ny, g.nz)))


@pytest.mark.parametrize("green", ["device", "oracle"])
@pytest.mark.parametrize("op", ["A", "PA", "NSCAT"])
def test_dense_matvec_fp64(vie, case, green, op):
    g, x, refs, h_dev, h_ext = case
    code = {"A": vie.VIE_OP_A, "PA": vie.VIE_OP_PA, "NSCAT": vie.VIE_OP_NSCAT}[op]
    y = gpu_matvec(vie, h_dev if green == "device" else h_ext, x, vie.VIE_FP64, code)
    assert rel(y, refs[op]) <= 1e-12


@pytest.mark.parametrize("green", ["device", "oracle"])
@pytest.mark.parametrize("op", ["A", "PA", "NSCAT"])
def test_dense_matvec_fp32(vie, case, green, op):
    g, x, refs, h_dev, h_ext = case
    code = {"A": vie.VIE_OP_A, "PA": vie.VIE_OP_PA, "NSCAT": vie.VIE_OP_NSCAT}[op]
    y = gpu_matvec(vie, h_dev if green == "device" else h_ext, x, vie.VIE_FP32, code)
    err = rel(y, refs[op])
    assert err <= 1e-5, err
    # every right-hand side on its own, not only the batch norm
    for r in range(R):
        assert rel(y[r], refs[op][r]) <= 1e-5


@pytest.mark.parametrize("op", ["A", "PA", "NSCAT"])
def test_dense_matvec_bf16x3(vie, case, op):
    """The BF16x3 tensor-core block product (bound 5e-5, from 3 * 2^-16 per real product)."""
    g, x, refs, h_dev, h_ext = case
    code = {"A": vie.VIE_OP_A, "PA": vie.VIE_OP_PA, "NSCAT": vie.VIE_OP_NSCAT}[op]
    y = gpu_matvec(vie, h_ext, x, vie.VIE_BF16X3, code)
    err = rel(y, refs[op])
    print(f"bf16x3 {g.nx}x{g.ny}x{g.nz} {op}: {err:.2e}")
    assert err <= 5e-5, err
    for r in range(R):
        assert rel(y[r], refs[op][r]) <= 5e-5


def test_external_green_toeplitz_roundtrip(vie, case):
    """The 60 tensors the external handle keeps are the oracle's representative entries (N - G)."""
    g, _, _, h_dev, h_ext = case
    a = np.zeros((60,) + g.shape, dtype=np.complex128)
    b = np.zeros_like(a)
    vie.vie_green_toeplitz(h_ext, a)
    vie.vie_green_toeplitz(h_dev, b)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
