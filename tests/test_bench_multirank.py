"""The multi-rank bench path on CPU: two gloo ranks, no GPU.  Each rank runs its own shot
(distinct source positions, no data-path collective); the timed region's duration and the
gradient time are reduced with a max over ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank, bench.max_over_ranks(torch, dist, 1.5 * (rank + 1)), bench.rank_shot_offset(rank),
                 bench.max_over_ranks(torch, None, 7.0)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_run_distinct_shots():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [3.0, 3.0]          # max of 1.5 and 3.0 on both ranks
    assert res[0][2] != res[1][2]                     # each rank its own shot position
    assert res[0][3] == 7.0                           # no process group: the value itself
