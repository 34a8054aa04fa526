"""The N > 1 path on CPU: two gloo ranks shard the faces and aggregate the timing like the
benchmark does (one rank per GPU, no collective on the data path)."""
import os
import socket

import pytest

from paper_1504_01883_gb300 import replicas


def test_shard_is_a_balanced_partition():
    for n in [0, 1, 5, 4096, 4097]:
        for world in [1, 2, 3, 8]:
            parts = [replicas.shard(n, r, world) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1


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
    from paper_1504_01883_gb300 import replicas as R
    dist.init_process_group("gloo", rank=rank, world_size=world)
    info = R.rank_info()
    faces = R.shard(4096, info.rank, info.world)
    secs = 0.5 + info.rank  # rank 1 is the slowest
    thr = R.job_throughput(len(faces), secs)
    q.put((info.rank, len(faces), R.max_over_ranks(secs), thr))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    import multiprocessing as mp
    pytest.importorskip("torch")
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
    assert [o[1] for o in out] == [2048, 2048]
    assert all(o[2] == 1.5 for o in out)                  # max over ranks
    assert all(abs(o[3] - 4096 / 1.5) < 1e-9 for o in out)  # all units / slowest rank
