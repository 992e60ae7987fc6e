"""The multi-rank logic of bench.py on CPU ranks (gloo, world size 2): max-over-ranks
timing, whole-job throughput, independent problems per rank, and the reference arm
running on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    ms, value = bench.job_throughput(10.0 + 5.0 * rank, steps=20, device="cpu")
    out.put((rank, ms, value, bench.rank_seed(0, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, seed in res:
        assert ms == pytest.approx(15.0)                       # the slower rank's time, on every rank
        assert value == pytest.approx(2 * 20 / 0.015)          # both ranks' iterations over that time
    assert res[0][3] != res[1][3]                               # independent problems


def test_single_process_throughput_is_steps_over_time():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_throughput(50.0, steps=10, device="cpu")
    assert ms == 50.0 and value == pytest.approx(200.0)


def test_reference_arm_is_silent_on_other_ranks(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        seed, steps, warmup = 0, 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
