"""Request loop with continuous batching (vie_server_*, vie_submit, vie_poll) on one GPU.

Tolerance: a request's outputs (solution, absorbed-power map and totals) are bitwise the
same alone, in a mix of concurrent requests, and through the direct calls vie_setup +
vie_rhs_dipoles + vie_solve + vie_fields: every request runs the same kernels on its
own stream with deterministic reductions.
"""

import re

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


# (shape, voxel, frequency, right-hand sides, tissue seed); requests 0 and 2 share (grid, voxel, frequency)
SPECS = [((12, 12, 12), 0.005, 298e6, 2, 11), ((14, 10, 9), 0.006, 128e6, 3, 12), ((12, 12, 12), 0.005, 298e6, 1, 13),
         ((10, 12, 8), 0.007, 64e6, 2, 14)]


def requests():
    out = []
    for shape, d, f, R, seed in SPECS:
        g = Grid(*shape, d, d, d)
        eps, sig = random_tissue(g, seed=seed, air_fraction=0.3)
        pos, mom = ring_dipoles(R, 0.06 + 0.01 * R)
        out.append((g, f, eps, sig, pos, mom))
    return out


def grid_tuple(g):
    return (g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)


def wait(server, ticket, limit_s=120.0):
    for _ in range(int(limit_s / 0.1)):
        r = server.poll(ticket, timeout_us=100000)
        if r is not None:
            return r
    raise AssertionError("request did not finish")


def run(server, reqs, tol=1e-7):
    tickets, outs = [], []
    for g, f, eps, sig, pos, mom in reqs:
        R = pos.shape[0]
        x = np.zeros((R, 12) + g.shape, dtype=np.complex128)
        pa = np.zeros((R,) + g.shape)
        P = np.zeros(R)
        tickets.append(server.submit(grid_tuple(g), f, eps, sig, pos, mom, tol=tol, restart=30, maxit=40,
                                     x_out=x, p_abs_out=pa, P_abs_out=P))
        outs.append((x, pa, P))
    return [wait(server, t) for t in tickets], outs


def test_mix_equals_alone_and_direct_calls(vie):
    reqs = requests()
    s = vie.Server(max_concurrent=4)
    res_mix, out_mix = run(s, reqs)
    s.close()
    assert all(r["status"] == vie.VIE_OK for r in res_mix), res_mix
    # requests 0 and 2 share one Green cache entry: exactly one of them built it
    assert res_mix[0]["green_cached"] + res_mix[2]["green_cached"] == 1
    assert res_mix[1]["green_cached"] == 0 and res_mix[3]["green_cached"] == 0
    # the requests were on the device at the same time: with four slots, the device spans (CUDA
    # events on each request's stream before its first and after its last kernel) of at least
    # two requests intersect, and so do their host spans
    spans = [(r["dev_start_s"], r["dev_end_s"]) for r in res_mix]
    assert all(0.0 <= a < b for a, b in spans), spans
    pairs = [(i, j) for i in range(4) for j in range(i + 1, 4)
             if max(spans[i][0], spans[j][0]) < min(spans[i][1], spans[j][1])]
    assert pairs, spans
    host = [(r["start_s"], r["end_s"]) for r in res_mix]
    assert any(max(host[i][0], host[j][0]) < min(host[i][1], host[j][1]) for i, j in pairs), host
    for i, req in enumerate(reqs):
        s1 = vie.Server(max_concurrent=1)
        res1, out1 = run(s1, [req])
        s1.close()
        assert res1[0]["status"] == vie.VIE_OK and res1[0]["iterations"] == res_mix[i]["iterations"]
        for a, b in zip(out_mix[i], out1[0]):
            assert np.array_equal(a, b)
    # the direct calls give the same bits
    g, f, eps, sig, pos, mom = reqs[1]
    h = vie.vie_setup(grid_tuple(g), f, eps, sig)
    R = pos.shape[0]
    e = torch.zeros((R, 12) + g.shape, dtype=torch.complex128, device="cuda")
    b = torch.zeros_like(e)
    vie.vie_rhs_dipoles(h, pos, mom, e, b)
    x = torch.zeros_like(b)
    rc, _ = vie.vie_solve(h, b, x, tol=1e-7, restart=30, maxit=40, mode=vie.VIE_SOLVE_FP32_REFINE)
    pa = torch.zeros((R,) + g.shape, dtype=torch.float64, device="cuda")
    P = vie.vie_fields(h, x, e, None, pa)
    torch.cuda.synchronize()
    h.close()
    assert np.array_equal(x.cpu().numpy(), out_mix[1][0])
    assert np.array_equal(pa.cpu().numpy(), out_mix[1][1])
    assert np.array_equal(np.asarray(P), out_mix[1][2])


def need_bytes(vie, req):
    """Device bytes the loop reserves for a request, read from the refusal of a 1-byte budget."""
    g, f, eps, sig, pos, mom = req
    s = vie.Server(hbm_budget_bytes=1, max_concurrent=1)
    with pytest.raises(vie.VieError) as e:
        s.submit(grid_tuple(g), f, eps, sig, pos, mom, restart=30, maxit=40)
    s.close()
    assert e.value.code == vie.VIE_ENOMEM
    return int(re.search(r"needs (\d+) device bytes", str(e.value)).group(1))


def test_budget_admits_one_at_a_time(vie):
    """With room for one request's working set only, the four requests run one after another."""
    reqs = requests()
    budget = int(1.3 * max(need_bytes(vie, r) for r in reqs))
    s = vie.Server(hbm_budget_bytes=budget, max_concurrent=4)
    res, _ = run(s, reqs)
    st = s.stats()
    s.close()
    assert all(r["status"] == vie.VIE_OK for r in res)
    spans = sorted((r["queued_s"], r["queued_s"] + r["run_s"]) for r in res)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 0.05, spans  # submissions are a few ms apart
    assert st["running"] == 0 and st["queued"] == 0


def test_poll_timeout_and_retired_ticket(vie):
    g = Grid(20, 20, 20, 0.005, 0.005, 0.005)
    eps, sig = random_tissue(g, seed=3, air_fraction=0.3)
    pos, mom = ring_dipoles(4, 0.09)
    s = vie.Server(max_concurrent=1)
    t = s.submit(grid_tuple(g), 128e6, eps, sig, pos, mom, tol=1e-7)
    assert s.poll(t, timeout_us=0) is None  # setup alone takes longer than this
    r = wait(s, t)
    assert r["status"] == vie.VIE_OK and r["nrhs"] == 4
    with pytest.raises(vie.VieError) as e:
        s.poll(t, timeout_us=0)
    assert e.value.code == vie.VIE_EINVAL
    with pytest.raises(vie.VieError) as e:
        s.submit(grid_tuple(g), 128e6, eps, sig, pos, mom, restart=0)
    assert e.value.code == vie.VIE_EINVAL
    s.close()


def test_closed_server_returns_its_pool_memory(vie):
    """Requests allocate in stream order from the device's memory pool, which keeps freed memory
    while the loop runs; closing the loop hands it back, so a later loop (or any other allocation)
    sees the device memory it had before."""
    reqs = requests()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    s = vie.Server(max_concurrent=4)
    res, _ = run(s, reqs)
    s.close()
    assert all(r["status"] == vie.VIE_OK for r in res)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20), (free0, free1)
