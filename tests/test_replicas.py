"""bench.py's multi-GPU form runs independent replicas (the correction does not
shard): the only cross-rank steps are a barrier and the max-reduction of the
step time.  They are exercised here with world_size 2 on the gloo backend (CPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
        out[rank] = (ms, bench.replica_throughput(world, 512 ** 3, ms))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(40.0, 55.0), (70.0, 10.0)])
def test_max_over_two_gloo_ranks(times):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        slow = max(times)
        for r in range(2):
            ms, gbs = out[r]
            assert ms == slow
            # whole-job throughput: both replicas' input over the slowest rank's time
            assert gbs == pytest.approx(2 * 4.0 * 512 ** 3 / (slow / 1e3) / 1e9)
