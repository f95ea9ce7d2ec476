"""Multi-rank path of bench.py on the CPU: N independent replicas (one per rank,
no data-path collective) whose job time is the maximum over the ranks and whose
throughput is N x the node updates of one replica over that time.  Two gloo
ranks on 127.0.0.1."""
import importlib.util
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, updates, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        t_max, value = bench.replica_throughput(torch, times[rank], updates, dist, device="cpu")
        out[rank] = (t_max, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_report_max_time_and_summed_throughput():
    world, updates = 2, 4096 * 4096 * 400
    times = [0.050, 0.047]
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), times, updates, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t_max, value = res[rank]
        assert t_max == max(times)
        assert abs(value - world * updates / max(times) / 1e6) <= 1e-9 * value


def test_single_process_is_one_replica():
    bench = _bench()
    t_max, value = bench.replica_throughput(torch, 0.02, 1_000_000, None)
    assert t_max == 0.02 and abs(value - 50.0) < 1e-12
