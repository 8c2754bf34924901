"""Continuous-batching server for cutting rollouts.

Requests (a scene and a substep count) arrive over time.  Every admitted
scene lives in one device batch (packed pools) and is advanced with all other
admitted scenes by CUDA-graph launches; a request that arrives while others
run is admitted as soon as the HBM budget and the pools have room, between
chunks of substeps, so its work overlaps with theirs on the device.  Finished
scenes are read back and their pool ranges freed immediately.

Because every sum in the substep is taken in a fixed order, a scene's result
does not depend on which other scenes share the batch: a rollout served in a
mix is bit-identical to the same rollout run alone.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np

from . import _abi as A
from .sim import Batch, Scene, footprint


@dataclasses.dataclass
class Result:
    request_id: int
    n_particles: int
    n_substeps: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    x: np.ndarray          # final positions (caller order)
    wrench: np.ndarray     # interval-averaged reaction wrench of the last substep
    error_bits: int

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


@dataclasses.dataclass
class _Active:
    rid: int
    scene: Scene
    remaining: int
    total: int
    bytes: int
    arrival_s: float
    admitted_s: float


class Server:
    """HBM-budgeted continuous batching over one GPU.

    ``budget_bytes`` bounds the device memory of admitted scenes (footprints
    from bm_scene_footprint); the batch pools are sized from it once.
    ``max_chunk`` is the number of substeps the batch advances between
    admission points: every admitted scene carries a stop substep
    (bm_scene_set_stop) at its request's length, so a request that ends
    inside a chunk stops there on the device, exactly, and is retired at the
    chunk's end while the others run the whole chunk.  ``node_tile`` and
    ``brick_variant`` are the launch shape (for instance an autotuned one;
    results do not depend on it).  ``allocator`` (a ``TorchAllocator``) makes
    PyTorch's caching allocator own the batch pools.

    While a chunk runs on the GPU the host computes the footprints of queued
    requests (the admission test) in a worker thread, so admission at the
    next chunk boundary only places the scene.
    """

    # pool capacity per budget byte (particles, nodes): a scene's footprint is
    # roughly 260 B per particle and its node count under half its particles
    BYTES_PER_PARTICLE = 260

    def __init__(self, budget_bytes: int, max_scenes: int = 256, max_chunk: int = 16,
                 stream=None, max_particles: Optional[int] = None, node_tile: int = 128,
                 brick_variant: int = 0, allocator=None):
        import torch
        self._torch = torch
        self.budget = int(budget_bytes)
        cap_p = int(max_particles or self.budget // self.BYTES_PER_PARTICLE)
        cap_n = cap_p // 2 + 27 * max_scenes
        self.stream = stream or torch.cuda.Stream()
        self.batch = Batch(max_particles=cap_p, max_nodes=cap_n, max_scenes=max_scenes,
                           graph_chunk=max_chunk, stream=self.stream, allocator=allocator)
        self.batch.set_tiles(max_chunk, node_tile, brick_variant)
        self.max_chunk = max_chunk
        self.queue: List[tuple] = []
        self.active: List[_Active] = []
        self.used = 0
        self.results: Dict[int, Result] = {}
        self.step_ms: List[float] = []      # ms per batched substep, one sample per chunk
        self.step_weight: List[int] = []    # substeps in that chunk
        self.particle_substeps = 0
        self.offered = 0                    # particle-substeps of every submitted request
        self.host_s = {"admit": 0.0, "retire": 0.0, "wait": 0.0}
        self._fp: Dict[int, int] = {}       # request id -> footprint bytes
        self._next_id = 0
        self._pool = None

    # -- requests ----------------------------------------------------------
    def submit(self, scene, n_substeps: int, arrival_s: float = 0.0) -> int:
        rid = self._next_id
        self._next_id += 1
        self.queue.append((arrival_s, rid, scene, int(n_substeps)))
        self.queue.sort(key=lambda t: (t[0], t[1]))
        self.offered += scene.n * int(n_substeps)
        return rid

    def _footprint(self, rid: int, sc) -> int:
        nb = self._fp.get(rid)
        if nb is None:
            nb = self._fp[rid] = footprint(sc)[3]
        return nb

    def _prefetch(self, now: float, horizon_s: float = 0.25) -> None:
        """Footprints of the requests that arrive soon (worker thread)."""
        for arrival, rid, sc, _ in self.queue[:32]:
            if arrival > now + horizon_s:
                break
            self._footprint(rid, sc)

    def _admit(self, now: float) -> None:
        t0 = time.perf_counter()
        while self.queue and self.queue[0][0] <= now:
            arrival, rid, sc, n = self.queue[0]
            nbytes = self._footprint(rid, sc)
            if self.used + nbytes > self.budget:
                break
            try:
                s = Scene.in_batch(self.batch, sc)
            except A.BMError as e:
                if e.code == A.E_CAPACITY:
                    break
                raise
            s.set_stop(n)
            self.queue.pop(0)
            self._fp.pop(rid, None)
            self.used += nbytes
            self.active.append(_Active(rid, s, n, n, nbytes, arrival, now))
        self.host_s["admit"] += time.perf_counter() - t0

    def _retire(self, now: float) -> None:
        t0 = time.perf_counter()
        keep = []
        for a in self.active:
            if a.remaining > 0:
                keep.append(a)
                continue
            # the no-allocation read keeps cudaMalloc/cudaFree (which would stall
            # the other scenes' work) out of the serving loop
            r = a.scene.read_noalloc("x") if a.scene.n * 12 <= (16 << 20) else a.scene.read("x")
            info = a.scene.info()
            assert info.step == a.total, (info.step, a.total)
            self.results[a.rid] = Result(a.rid, a.scene.n, a.total, a.arrival_s, a.admitted_s, now,
                                         r["x"], a.scene.tool_wrench() if a.scene.spec.blade else
                                         np.zeros(6), int(info.error_bits))
            a.scene.close()
            self.used -= a.bytes
        self.active = keep
        self.host_s["retire"] += time.perf_counter() - t0

    # -- main loop -----------------------------------------------------------
    def run(self, realtime: bool = True, timeout_s: float = 3600.0) -> dict:
        """Serve until every submitted request has finished.  With realtime
        the arrival times are honoured against the wall clock; otherwise every
        request counts as already arrived."""
        from concurrent.futures import ThreadPoolExecutor
        torch = self._torch
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        self._pool = ThreadPoolExecutor(max_workers=1)
        try:
            while self.queue or self.active:
                now = time.perf_counter() - t0
                if now > timeout_s:
                    raise TimeoutError("serving loop exceeded its time limit")
                self._admit(now if realtime else float("inf"))
                if not self.active:
                    if self.queue and realtime:
                        self._prefetch(now)
                        time.sleep(max(0.0, min(0.05, self.queue[0][0] - now)))
                        continue
                    if self.queue:
                        raise RuntimeError("a request does not fit the budget or the pools")
                    break
                k = self.max_chunk
                e0.record(self.stream)
                self.batch.step(k)
                e1.record(self.stream)
                # host work that overlaps the chunk: footprints of what arrives next
                fut = self._pool.submit(self._prefetch, now if realtime else float("inf"))
                tw = time.perf_counter()
                e1.synchronize()
                fut.result()
                self.host_s["wait"] += time.perf_counter() - tw
                self.step_ms.append(e0.elapsed_time(e1) / k)
                self.step_weight.append(k)
                for a in self.active:
                    d = min(k, a.remaining)
                    self.particle_substeps += d * a.scene.n
                    a.remaining -= d
                self._retire(time.perf_counter() - t0)
        finally:
            self._pool.shutdown()
            self._pool = None
        wall = time.perf_counter() - t0
        return self.stats(wall)

    def stats(self, wall_s: float) -> dict:
        ms = np.repeat(np.array(self.step_ms), np.array(self.step_weight)) if self.step_ms else \
            np.zeros(1)
        res = list(self.results.values())
        lat = np.array([r.latency_s for r in res]) if res else np.zeros(1)
        queued = np.array([r.admitted_s - r.arrival_s for r in res]) if res else np.zeros(1)
        arrivals = [r.arrival_s for r in res]
        span = (max(arrivals) - min(arrivals)) if len(arrivals) > 1 else 0.0
        return {"requests": len(res), "wall_s": wall_s,
                "throughput": self.particle_substeps / wall_s if wall_s > 0 else 0.0,
                "offered_load": self.offered / span if span > 0 else None,
                "step_ms_p50": float(np.percentile(ms, 50)),
                "step_ms_p99": float(np.percentile(ms, 99)),
                "request_latency_s_p50": float(np.percentile(lat, 50)),
                "request_latency_s_p99": float(np.percentile(lat, 99)),
                "queue_latency_s_p50": float(np.percentile(queued, 50)),
                "queue_latency_s_p99": float(np.percentile(queued, 99)),
                "host_s": dict(self.host_s),
                "particle_substeps": self.particle_substeps}

    def close(self):
        self.batch.close()


# -- several GPUs -------------------------------------------------------------
def route(requests, n_ranks: int, budget_bytes: int, footprint_bytes=None) -> List[int]:
    """Rank of every request when one server per GPU shares a request stream.

    Requests (objects with ``scene``, ``n_substeps`` and ``arrival_s``) are
    taken in arrival order and each goes to the rank with the least work
    assigned so far (particles x substeps) among those whose budget holds its
    footprint; ties go to the lower rank.  The assignment depends only on the
    request stream, so every rank computes the same one on its own: no
    message carries requests and the data path has no collective.  A request
    that fits no rank's budget is refused with ValueError."""
    if footprint_bytes is None:
        footprint_bytes = lambda sc: footprint(sc)[3]  # noqa: E731
    order = sorted(range(len(requests)), key=lambda i: (requests[i].arrival_s, i))
    work = [0] * n_ranks
    out = [-1] * len(requests)
    for i in order:
        r = requests[i]
        nb = footprint_bytes(r.scene)
        if nb > budget_bytes:
            raise ValueError(f"request {i} needs {nb} bytes, more than a rank's budget")
        k = min(range(n_ranks), key=lambda q: (work[q], q))
        out[i] = k
        work[k] += r.scene.n * int(r.n_substeps)
    return out


def serve_sharded(requests, rank: int, n_ranks: int, budget_bytes: int, dist=None, **server_kw) -> dict:
    """Serve this rank's share of a request stream (see ``route``) on its GPU
    and combine the ranks' statistics on the host: the job's throughput is
    the particle-substeps of all ranks over the slowest rank's wall time.
    ``dist`` is ``torch.distributed`` (initialised) or None for one rank."""
    ranks = route(requests, n_ranks, budget_bytes)
    mine = [r for r, k in zip(requests, ranks) if k == rank]
    srv = Server(budget_bytes=budget_bytes, max_scenes=max(1, len(mine)),
                 max_particles=max(1, sum(r.scene.n for r in mine)), **server_kw)
    for r in mine:
        srv.submit(r.scene, r.n_substeps, arrival_s=r.arrival_s)
    st = srv.run(realtime=True, timeout_s=600) if mine else srv.stats(0.0)
    srv.close()
    return combine_stats(st, dist, n_requests=len(mine))


def combine_stats(st: dict, dist=None, n_requests: Optional[int] = None) -> dict:
    """Job-wide serving statistics from every rank's (host-side gather)."""
    if dist is None:
        return dict(st, ranks=1)
    allst = [None] * dist.get_world_size()
    dist.all_gather_object(allst, dict(st, requests=st["requests"] if n_requests is None else n_requests))
    wall = max(s["wall_s"] for s in allst)
    ps = sum(s["particle_substeps"] for s in allst)
    return {"ranks": len(allst), "requests": sum(s["requests"] for s in allst), "wall_s": wall,
            "throughput": ps / wall if wall > 0 else 0.0, "particle_substeps": ps,
            "step_ms_p50": max(s["step_ms_p50"] for s in allst),
            "step_ms_p99": max(s["step_ms_p99"] for s in allst),
            "request_latency_s_p50": max(s["request_latency_s_p50"] for s in allst),
            "request_latency_s_p99": max(s["request_latency_s_p99"] for s in allst),
            "queue_latency_s_p50": max(s.get("queue_latency_s_p50", 0.0) for s in allst),
            "queue_latency_s_p99": max(s.get("queue_latency_s_p99", 0.0) for s in allst),
            "offered_load": (sum(s["offered_load"] for s in allst if s.get("offered_load")) or None)}
