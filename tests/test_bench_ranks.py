"""Multi-rank host logic of bench.py on the CPU: two gloo ranks (127.0.0.1) take the slowest
rank's time with max_over_ranks and report the whole-job throughput (the units every rank
processed over that time), as the timed steps and the end-to-end leg do under torchrun."""

import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


LOCAL_SECONDS = [3.0, 5.0]


def worker(rank, world_size, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        b = load_bench()
        slowest = b.max_over_ranks(LOCAL_SECONDS[rank])
        value = b.job_throughput(16, world_size, slowest)
        with open(os.path.join(out_dir, f"rank{rank}"), "w") as f:
            f.write(f"{slowest!r} {value!r}")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_job_throughput_two_gloo_ranks(tmp_path):
    mp.spawn(worker, args=(2, free_port(), str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        slowest, value = map(float, (tmp_path / f"rank{rank}").read_text().split())
        assert slowest == 5.0  # every rank sees the slowest rank's time
        assert value == 16 * 2 / 5.0


def test_single_process_is_identity():
    b = load_bench()
    assert not dist.is_initialized()
    assert b.max_over_ranks(2.5) == 2.5
    assert b.job_throughput(16, 1, 2.0) == 8.0
