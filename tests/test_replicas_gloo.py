"""The multi-GPU path of bench.py runs independent replicas (one per rank):
the only cross-rank step is timing -- the job's step time is the slowest
rank's, and the whole-job seconds per solve divide it by the number of
replicas.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    got_ws, got_rank, got_local = bench.dist_env()
    t = bench.max_over_ranks(times[rank], ws)
    q.put((rank, got_ws, got_rank, got_local, t, bench.per_solve(t, ws)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_the_slowest_rank():
    ws, times = 2, [0.0125, 0.0375]
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, times, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, got_ws, got_rank, got_local, t, value) in enumerate(out):
        assert (rank, got_ws, got_rank, got_local) == (r, ws, r, r)
        assert t == max(times)
        assert value == max(times) / ws


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.02, 1) == 0.02
    assert bench.per_solve(0.02, 1) == 0.02
