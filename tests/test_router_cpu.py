"""Request routing across GPUs for the continuous-batching server (host logic,
CPU only): one server per rank, the same assignment computed on every rank,
statistics combined on the host over gloo."""
import socket
from dataclasses import dataclass

import pytest

from paper_2609_27342_gb300.serving import combine_stats, route


@dataclass
class _Scene:
    n: int


@dataclass
class _Req:
    scene: _Scene
    n_substeps: int
    arrival_s: float


def _stream(k=40, seed=0):
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(0.02, k))
    return [_Req(_Scene(int(rng.integers(8000, 500000))), int(rng.integers(200, 2000)), float(a))
            for a in t]


def test_route_assigns_each_request_once_and_balances_work():
    reqs = _stream()
    fp = lambda sc: 260 * sc.n  # noqa: E731
    for n_ranks in (1, 2, 3, 8):
        ranks = route(reqs, n_ranks, budget_bytes=1 << 40, footprint_bytes=fp)
        assert len(ranks) == len(reqs) and all(0 <= r < n_ranks for r in ranks)
        work = [sum(q.scene.n * q.n_substeps for q, r in zip(reqs, ranks) if r == k)
                for k in range(n_ranks)]
        biggest = max(q.scene.n * q.n_substeps for q in reqs)
        # greedy least-loaded: the spread never exceeds one request's work
        assert max(work) - min(work) <= biggest
        # deterministic: every rank computes the same assignment
        assert route(reqs, n_ranks, 1 << 40, fp) == ranks
    assert route(reqs, 1, 1 << 40, fp) == [0] * len(reqs)


def test_route_follows_arrival_order_and_refuses_oversize():
    fp = lambda sc: 260 * sc.n  # noqa: E731
    reqs = [_Req(_Scene(1000), 10, 0.3), _Req(_Scene(1000), 10, 0.1), _Req(_Scene(1000), 10, 0.2)]
    # the earliest arrival goes first, to rank 0; the next to rank 1; the third to rank 0
    assert route(reqs, 2, 1 << 30, fp) == [0, 0, 1]
    with pytest.raises(ValueError):
        route([_Req(_Scene(10 ** 6), 10, 0.0)], 2, budget_bytes=1000, footprint_bytes=fp)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    st = [{"requests": 3, "wall_s": 2.0, "particle_substeps": 100, "step_ms_p50": 0.5,
           "step_ms_p99": 0.7, "request_latency_s_p50": 0.4, "request_latency_s_p99": 1.0,
           "queue_latency_s_p50": 0.01, "queue_latency_s_p99": 0.2, "offered_load": 60.0},
          {"requests": 5, "wall_s": 4.0, "particle_substeps": 300, "step_ms_p50": 0.6,
           "step_ms_p99": 0.9, "request_latency_s_p50": 0.3, "request_latency_s_p99": 1.2,
           "queue_latency_s_p50": 0.02, "queue_latency_s_p99": 0.1, "offered_load": 90.0}][rank]
    q.put((rank, combine_stats(st, dist)))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_stats_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        s = got[r]
        assert s["ranks"] == 2 and s["requests"] == 8 and s["wall_s"] == 4.0
        assert s["throughput"] == pytest.approx(400 / 4.0)
        assert s["step_ms_p99"] == 0.9 and s["request_latency_s_p99"] == 1.2
        assert s["queue_latency_s_p99"] == 0.2 and s["offered_load"] == pytest.approx(150.0)
