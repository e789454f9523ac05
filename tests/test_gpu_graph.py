"""The solver's restart cycles run without host round trips, replayed as CUDA graphs.

* A cycle replayed from its graph gives the same bits as the same cycle launched kernel by
  kernel (flags bit 3), in every mode: the graph only changes how the launches are issued.
* Launch accounting under graphs: every replay is counted, the launches whose active list was
  empty are not, so the FP32 z pass shows exactly the solver's inner matvec count, and with
  timing on the replayed kernels carry device time.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import Grid, random_tissue, ring_dipoles  # noqa: E402


@pytest.fixture(scope="module")
def vie():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_02196_gb300 as v

    v.build()
    return v


@pytest.fixture(scope="module")
def prob(vie):
    g = Grid(12, 10, 9, 0.006, 0.005, 0.007)
    eps, sig = random_tissue(g, seed=55, air_fraction=0.25)
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), 298e6, eps, sig)
    R = 5
    pos, mom = ring_dipoles(R, 0.07)
    b = torch.zeros((R, 12) + g.shape, dtype=torch.complex128, device="cuda")
    vie.vie_rhs_dipoles(h, pos, mom, None, b)
    yield g, h, b
    h.close()


MODES = ["fp64", "mixed", "bf16x3"]


def mode_of(vie, name):
    return {"fp64": vie.VIE_SOLVE_FP64, "mixed": vie.VIE_SOLVE_FP32_REFINE, "bf16x3": vie.VIE_SOLVE_BF16X3_REFINE}[name]


@pytest.mark.parametrize("mode", MODES)
def test_graph_replay_matches_direct_launches(vie, prob, mode):
    g, h, b = prob
    out = []
    for graph in (True, False):
        x = torch.zeros_like(b)
        rc, info = vie.vie_solve(h, b, x, tol=1e-8, restart=12, maxit=80, mode=mode_of(vie, mode), graph=graph)
        assert rc == vie.VIE_OK, info
        out.append((x, info))
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("graph", [True, False])
def test_launch_accounting_under_graphs(vie, prob, graph):
    g, h, b = prob
    x = torch.zeros_like(b)
    vie.vie_stats_reset(True)
    rc, info = vie.vie_solve(h, b, x, tol=1e-8, restart=12, maxit=80, mode=vie.VIE_SOLVE_FP32_REFINE, graph=graph)
    total, st = vie.vie_stats_read()
    vie.vie_stats_reset(False)
    assert rc == vie.VIE_OK
    n32 = info[0]["fp32_matvecs"]
    # every inner FP32 matvec and the refinement's FP32 residual update run the z pass once
    assert st["zpass_block_f32"][0] == n32, (st["zpass_block_f32"], info[0])
    assert st["zpass_block_f32"][1] > 0 and st["zpass_block_f32"][2] > 0
    assert st["gs_dots"][0] > 0 and st["gs_dots"][1] > 0
    # total_launches also holds the launches that found an empty active list
    assert total >= sum(v[0] for v in st.values())


def test_autotuner_reports_its_choice(vie):
    """The first matvec on a new grid shape measures the z pass's tile widths and keeps the fastest;
    the report names the shape, every width with its time, and the choice."""
    g = Grid(9, 7, 11, 0.004, 0.004, 0.004)  # a shape the other tests do not use
    eps, sig = random_tissue(g, seed=8)
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), 128e6, eps, sig)
    (Lx, Ly, Lz), _ = vie.vie_info(h)
    key = f"Lz={Lz} Lx={Lx} Ly={Ly} nz={g.nz} R<=2:"
    x = torch.zeros((2, 12) + g.shape, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for prec, name in ((vie.VIE_FP32, "zpass_block_f32"), (vie.VIE_BF16X3, "zpass_block_bf16x3")):
        vie.vie_matvec(h, x, y, prec, vie.VIE_OP_PA)
        lines = [ln for ln in vie.vie_tuning() if ln.startswith(name + " ") and key in ln]
        assert len(lines) == 1, vie.vie_tuning()
        assert "TB=4" in lines[0] and "TB=8" in lines[0] and "->" in lines[0]
    torch.cuda.synchronize()
    h.close()
