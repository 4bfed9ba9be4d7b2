"""Host logic of bench.py's multi-GPU launch (replicas, one per rank): the
rank environment and the max-over-ranks step time, on two gloo ranks on the
CPU (the data path has no collective: each rank solves its own seeded
system)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, lr = bench.rank_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    slowest = bench.max_over_ranks(10.0 * (r + 1), dist, device="cpu")
    dist.barrier()
    out.put((r, w, lr, slowest, bench.max_over_ranks(1.5, None)))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_step():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(r[3] == 20.0 and r[4] == 1.5 for r in res)
