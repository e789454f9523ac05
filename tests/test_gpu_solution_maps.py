"""Field and absorbed-power maps of a heterogeneous head solve at the benchmark's tolerance,
against the oracle's converged solution.

Workload: the head phantom generator of the 64^3 benchmark on 32^3 voxels of 6 mm (192 mm box),
298 MHz, four z-directed unit dipoles on the 15 cm ring.  The GPU solves with GMRES(50) to a
preconditioned relative residual of 1e-6 (the benchmark's stopping rule) and to 1e-7,
in mixed precision (FP32 GMRES inside FP64 refinement) and in plain FP64; the oracle's solution was
taken to 1e-11 (tests/golden/make_head32_solution.py, oracle only).  Compared per right-hand side,
as relative 2-norms over the tissue voxels: the voxel-average (l = 1) field coefficients of the
three components (the field map) and the absorbed-power density (the SAR map); and the total
absorbed power (Eq. 44).  The 1e-6 map target needs the 1e-7 residual.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import Grid, head_phantom, ring_dipoles  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "head32_ring4_solution.npz")
N, FREQ, R = 32, 298e6, 4


@pytest.fixture(scope="module")
def vie():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_02196_gb300 as v

    v.build()
    return v


@pytest.fixture(scope="module")
def problem(vie):
    h = 0.192 / N
    g = Grid(N, N, N, h, h, h)
    eps, sig = head_phantom(g)
    pos, mom = ring_dipoles(R, 0.15)
    hd = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), FREQ, eps, sig)
    e = torch.zeros((R, 12) + g.shape, dtype=torch.complex128, device="cuda")
    b = torch.zeros_like(e)
    vie.vie_rhs_dipoles(hd, pos, mom, e, b)
    tissue = ((eps != 1.0) | (sig != 0.0)).ravel()
    ref = np.load(GOLDEN)
    yield g, hd, e, b, tissue, ref
    hd.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solve_maps(vie, problem, mode, tol):
    g, hd, e, b, tissue, ref = problem
    m = vie.VIE_SOLVE_FP32_REFINE if mode == "mixed" else vie.VIE_SOLVE_FP64
    x = torch.zeros_like(b)
    rc, info = vie.vie_solve(hd, b, x, tol=tol, restart=50, maxit=200, mode=m)
    assert rc == vie.VIE_OK, info
    assert all(i["resid"] <= tol for i in info), info
    ef = torch.empty_like(e)
    pa = torch.empty((R,) + g.shape, dtype=torch.float64, device="cuda")
    P = vie.vie_fields(hd, x, e, ef, pa)
    fmap = ef.cpu().numpy()[:, [0, 4, 8]].reshape(R, 3, -1)[:, :, tissue]
    pabs = pa.cpu().numpy().reshape(R, -1)[:, tissue]
    out = []
    for r in range(R):
        ef_err = rel(fmap[r], ref["field_l1"][r].astype(np.complex128))
        pa_err = rel(pabs[r], ref["p_abs"][r].astype(np.float64))
        P_err = abs(P[r] - ref["P_abs"][r]) / abs(ref["P_abs"][r])
        print(f"{mode} tol {tol:.0e} rhs {r}: field map {ef_err:.2e}, p_abs {pa_err:.2e}, P_abs {P_err:.2e}, "
              f"resid {info[r]['resid']:.2e}, err_est {info[r]['err_est']:.2e}, iterations {info[r]['iterations']}")
        out.append((ef_err, pa_err, P_err, info[r]))
    return out


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_head32_maps_tolerance_chain(vie, problem, mode):
    """Residual -> map error on this phantom: at the benchmark's 1e-6 residual the maps carry an
    error several times the residual (about 4e-6), which the solver's err_est reports within a
    factor 3; a 1e-7 residual delivers maps within 1e-6 of the oracle's converged solution."""
    for ef_err, pa_err, P_err, info in solve_maps(vie, problem, mode, 1e-6):
        assert ef_err <= 1e-5 and pa_err <= 1e-5
        assert ef_err / 3 <= info["err_est"] <= 3 * ef_err
    for ef_err, pa_err, P_err, info in solve_maps(vie, problem, mode, 1e-7):
        assert ef_err <= 1e-6
        assert pa_err <= 1e-6
        assert P_err <= 1e-6
        assert info["err_est"] <= 1e-6
