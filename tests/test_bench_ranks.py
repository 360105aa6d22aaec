"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2): every rank ends up
with the longest rank's timed region, and the throughput counts the updates of all ranks."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms, value = bench.combine_ranks(10.0 + 5.0 * rank, world, upd_step=1000, steps=4, device="cpu")
    out.put((rank, ms, value))
    tdist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0                                   # the slower rank's region
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)  # both ranks' updates over it


def test_one_rank_is_unchanged():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.combine_ranks(8.0, 1, 500, 2) == (8.0, 500 * 2 / 0.008)
