"""Host arithmetic of bench.py's roofline line (no GPU): the algorithmic byte and FLOP model
of the z pass, its affine dependence on the right-hand sides a launch transforms (used to
recover that count from the library's byte counters), and the scaling of the recorded ncu
traffic to the timed launches."""

import importlib.util
import math
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


GRID, L = (64, 64, 64), (128, 128, 128)


def test_zpass_model_head64():
    b = load_bench()
    by, fl = b.kernel_model("zpass_block_f32", GRID, L, 16)
    # spectrum read + written once (16 RHS x 12 x 64 planes x 128 x 128, 8-byte complex) + octant Green
    assert by == 2 * 16 * 12 * 64 * 128 * 128 * 8 + 60 * 65**3 * 8
    # two length-128 transforms per line (5 N log2 N) + 144 complex multiply-adds per point
    assert fl == 2 * 5 * 128 * 7 * (16 * 12 * 128 * 128) + 144 * 8 * 16 * 128**3
    assert abs(fl / 1e9 - 66.840428544) < 1e-9
    # above the FP32 ridge point (80.5 TFLOP/s over 6.69 TB/s): the ALU floor is the larger
    assert fl / 80.54784e12 > by / 6688.8e9


def test_rhs_count_recovered_from_bytes():
    b = load_bench()
    b0, _ = b.kernel_model("zpass_block_f32", GRID, L, 0)
    b1, f1 = b.kernel_model("zpass_block_f32", GRID, L, 1)
    for R in (1, 7, 15.27, 16):
        bR = b0 + R * (b1 - b0)
        assert math.isclose((bR - b0) / (b1 - b0), R)
    # flops are linear in R with no constant term
    assert b.kernel_model("zpass_block_f32", GRID, L, 0)[1] == 0
    assert math.isclose(b.kernel_model("zpass_block_f32", GRID, L, 16)[1], 16 * f1)


def test_matvec_bytes_head64():
    b = load_bench()
    assert b.matvec_alg_bytes(GRID, L, 16, 8) == 7782230496


def test_traffic_scaling(monkeypatch):
    b = load_bench()
    full, _ = b.kernel_model("zpass_block_f32", GRID, L, b.NRHS)
    monkeypatch.setattr(b, "measured_traffic", lambda k: 3.4e9)
    assert math.isclose(b.scaled_traffic("zpass_block_f32", GRID, L, full), 3.4e9)
    assert math.isclose(b.scaled_traffic("zpass_block_f32", GRID, L, full / 2), 1.7e9)
    monkeypatch.setattr(b, "measured_traffic", lambda k: None)
    assert b.scaled_traffic("zpass_block_f32", GRID, L, full) is None
