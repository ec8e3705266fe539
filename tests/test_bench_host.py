"""Host-side logic of bench.py: the multi-rank timing reduction (gloo, world size 2 on CPU),
argument checks and the traffic record lookup."""
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tmax, tsum = bench.reduce_max_sum(dist, world, 10.0 + rank, 100.0 * (rank + 1))
    bench.barrier(dist, world)
    q.put((rank, tmax, tsum))
    dist.destroy_process_group()


def test_reduce_max_sum_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, tsum in out:
        assert tmax == 11.0 and tsum == 300.0


def test_single_rank_reduction_is_identity():
    assert bench.reduce_max_sum(None, 1, 3.5, 7.0) == (3.5, 7.0)


def test_warmup_minimum():
    with pytest.raises(SystemExit):
        bench.main(["--warmup", "2", "--steps", "1"])


def test_traffic_record_tracks_kernel_source():
    # a key that is not recorded gives None (never a stale number)
    assert bench.traffic_per_launch("no_such_kernel") is None
