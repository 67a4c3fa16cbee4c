"""The multi-rank path of bench.py on CPU: two gloo ranks (one process per
rank, as under torchrun) agree on the job's time as the maximum over the
ranks, and the whole-job throughput counts every rank's cells; the
reference leg runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, ms, bench.job_mlups(1000, 4, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, ms, v in got:
        assert ms == 15.0
        assert v == pytest.approx(1000 * 4 * 2 / 15e-3 / 1e6)


def test_single_rank_is_its_own_maximum_and_reference_leg_skips_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_mlups(2 ** 21, 10, 1, 1000.0) == pytest.approx(2 ** 21 * 10 / 1e6)
    assert bench.run_reference(None, None, 2, 1) is None
    assert capsys.readouterr().out == ""
