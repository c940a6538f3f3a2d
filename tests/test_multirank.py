"""The multi-rank path of bench.py (one independent propagation per rank, no
data-path collective) on CPU with the gloo backend and two ranks: the ranks
get different problems, the job time is the maximum over ranks, the
throughput counts every rank's steps, and the reference arm runs on rank 0
only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        wl = bench.workload(5, rank)
        ms = bench.max_over_ranks(10.0 * (rank + 1))
        os.environ["RANK"] = str(rank)
        ref = bench.run_reference(bench.parse_args(["--impl", "reference"])) if rank != 0 else None
        out.put((rank, tuple(wl.fields[0].direction), ms, ref))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_ranks_on_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, d0, ms0, _), (r1, d1, ms1, ref1) = res
    assert d0 == (1.0, 0.0, 0.0) and d1 == (0.0, 1.0, 0.0)    # an independent problem per rank
    assert ms0 == ms1 == 20.0                                   # the job's time is the slowest rank's
    assert ref1 == 0                                            # the reference arm does no work off rank 0
    import bench
    assert bench.job_throughput(world, 4, 20.0) == pytest.approx(400.0)
