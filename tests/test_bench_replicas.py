"""The bench's replica path (N > 1) on CPU: two gloo ranks, as torchrun would start them.

Each rank reads its rank from the environment and runs its own seeded problem; the timing
is the slowest rank's (a max all-reduce, which every rank receives); the whole-job value
counts every rank's updates; under torchrun only rank 0 runs the reference arm."""
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        r, w, local = bench.rank_env()
        bench.ranks_barrier(dist)
        slowest = bench.ranks_max(1.5 + r, dist, torch.device("cpu"))
        args = types.SimpleNamespace(gpus=world, steps=1, warmup=3)
        ref_rc = bench.run_reference(args) if r != 0 else None   # rank != 0: returns without work
        bench.ranks_barrier(dist)
        q.put((r, w, local, slowest, bench.replica_seed(r), ref_rc))
        dist.destroy_process_group()
    except Exception as e:   # reported to the parent
        q.put(("error", repr(e)))


def test_two_gloo_replicas():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(o[0] != "error" for o in out), out
    out.sort()
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    assert out[0][3] == out[1][3] == 2.5                 # both ranks see the slowest rank's time
    assert out[0][4] != out[1][4]                        # independent seeded problems
    assert out[1][5] == 0                                # the reference arm runs on rank 0 only


def test_whole_job_value_counts_every_rank():
    import bench
    assert bench.per_update_value(2.0, 4, 2) == 0.25     # 8 updates in the slowest rank's 2 s
    assert bench.per_update_value(2.0, 4, 1) == 0.5
    assert bench.rank_env({}) == (0, 1, 0)
    assert bench.ranks_max(3.0, None, None) == 3.0
