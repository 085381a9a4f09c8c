"""Host logic of the multi-GPU (replicas-only) bench path, run as two gloo ranks on CPU:
barrier, maximum of the timed region over ranks, whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    bench.barrier(dist)
    my_ms = 100.0 + 50.0 * r          # rank 1 is the slow replica
    ms = bench.max_over_ranks(dist, my_ms, device="cpu")
    value = bench.whole_job_mlups(ws, 256 ** 3, 1000, ms)
    q.put((r, ws, local, ms, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for r, ws, local, ms, value in res:
        assert ws == 2 and local == r
        assert ms == 150.0
        assert value == pytest.approx(2 * 256 ** 3 * 1000 / 0.150 / 1e6)
