"""The bench's multi-rank path on CPU: two gloo ranks combine their figures the
way the GPU ranks do over NCCL (slowest rank's time, summed work), and every
rank walks its own packets under its own key."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.combine_ranks(dist, torch.device("cpu"), 1.0 + rank, 100 * (rank + 1), 7 + rank, 2.0 - rank,
                              50 * (rank + 1))
    q.put((rank, out, bench.rank_seed(1234, rank, 10_000_000)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (o, k)) for r, o, k in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        tsec, trans, esc, e2e_dt, e2e = res[r][0]
        assert tsec == 2.0 and e2e_dt == 2.0          # slowest rank
        assert trans == 300.0 and esc == 15.0 and e2e == 150.0  # summed work
    assert res[0][1] != res[1][1]                      # independent packet streams


def test_single_rank_needs_no_collective():
    import bench
    assert bench.combine_ranks(None, None, 1.5, 10, 2, 0.5, 3) == (1.5, 10.0, 2.0, 0.5, 3.0)
