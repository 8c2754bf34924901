"""The multi-rank benchmark path on CPU: two gloo ranks (no GPU).

Scenes are independent, so ranks hold their own shards (no data-path
collective); the job's throughput is the summed work over the slowest rank's
time, reduced over the ranks exactly as on the GPUs."""
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    import bench
    ms, n = bench.reduce_over_ranks(dist, [10.0, 25.0][rank], [100, 300][rank], device="cpu")
    q.put((rank, ms, n))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(got) == [(0, 25.0, 400), (1, 25.0, 400)]


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, 12.5, 77) == (12.5, 77)


def test_rank_shards_are_independent():
    import bench
    a, b = bench.rank_scenes(0), bench.rank_scenes(1)
    assert len(a) == len(b) == bench.N_SCENES
    # rank 0 is the benchmark workload itself (seed 2); rank 1 another draw
    assert sum(s.n for s in a) == 5937664
    assert [s.n for s in a] != [s.n for s in b]
