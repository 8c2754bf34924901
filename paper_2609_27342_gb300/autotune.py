"""Launch-shape autotuner for a batch of scenes.

The batched substep has three launch parameters that do not change its
results (every sum is taken in a fixed order, and the kernel variants share
their arithmetic): the brick-kernel occupancy variant (resident CTAs per SM of
the per-brick P2G, G2P+MUSL and F-update kernels, i.e. registers per thread
against latency hiding), the node tile (threads per CTA of the per-node
kernels) and the number of substeps captured in one CUDA graph.  The tuner
times candidate shapes on the batch itself with CUDA events on the batch's
stream and keeps the fastest.

Every probe advances the simulation: tuning is a warm-up of the batch, not a
side computation.
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, Iterable, List, Optional

VARIANTS = (0, 1, 2)
NODE_TILES = (64, 128, 256, 512)
GRAPH_CHUNKS = (4, 8, 16, 32)

_cache: Dict[tuple, dict] = {}


def _time_shape(batch, stream, chunk: int, ntile: int, variant: int, substeps: int,
                rounds: int) -> tuple:
    """(ms per substep of one launch shape, best of ``rounds`` timed runs;
    substeps advanced)."""
    import torch
    batch.set_tiles(chunk, ntile, variant)
    n = max(chunk, int(math.ceil(substeps / chunk)) * chunk)
    batch.step(chunk)                       # captures this shape's graph, untimed
    best = math.inf
    for _ in range(rounds):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.step(n)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / n)
    return best, chunk + rounds * n


def autotune(batch, stream, key: Optional[tuple] = None, substeps: int = 16, rounds: int = 1,
             variants: Iterable[int] = VARIANTS, node_tiles: Iterable[int] = NODE_TILES,
             graph_chunks: Iterable[int] = GRAPH_CHUNKS, baseline=(16, 128, 0)) -> dict:
    """Pick (brick variant, node tile) on a full grid at a 16-substep graph,
    then the graph chunk for the winner; set it on ``batch`` and return
    ``{"best": {...}, "trials": [...], "substeps_advanced": n}``.

    The probes advance the scenes, and the cost of a substep drifts as cuts
    progress, so every candidate is timed between two timings of a fixed
    ``baseline`` shape (graph chunk, node tile, variant) and ranked by its
    time relative to their mean.  ``stream`` is the torch stream the batch
    launches on.  With ``key`` the result is cached for this process and a
    later call with the same key only applies it."""
    if key is not None and key in _cache:
        b = _cache[key]["best"]
        batch.set_tiles(b["graph_chunk"], b["node_tile"], b["brick_variant"])
        return dict(_cache[key], cached=True, substeps_advanced=0)
    trials: List[dict] = []
    advanced = 0
    seen = set()

    def probe(chunk, ntile, variant):
        nonlocal advanced, ref_ms
        if (chunk, ntile, variant) in seen:
            return
        seen.add((chunk, ntile, variant))
        ms, k = _time_shape(batch, stream, chunk, ntile, variant, substeps, rounds)
        ms_ref, k_ref = _time_shape(batch, stream, *baseline, substeps, rounds)
        advanced += k + k_ref
        trials.append({"brick_variant": variant, "node_tile": ntile, "graph_chunk": chunk,
                       "ms": ms, "relative": ms / (0.5 * (ref_ms + ms_ref))})
        ref_ms = ms_ref

    ref_ms, k0 = _time_shape(batch, stream, *baseline, substeps, rounds)
    advanced += k0
    trials.append({"brick_variant": baseline[2], "node_tile": baseline[1],
                   "graph_chunk": baseline[0], "ms": ref_ms, "relative": 1.0})
    seen.add(tuple(baseline))
    for v, t in itertools.product(variants, node_tiles):
        probe(16, t, v)
    best = min(trials, key=lambda r: r["relative"])
    for c in graph_chunks:
        probe(c, best["node_tile"], best["brick_variant"])
    best = min(trials, key=lambda r: r["relative"])
    batch.set_tiles(best["graph_chunk"], best["node_tile"], best["brick_variant"])
    out = {"best": {"brick_variant": best["brick_variant"], "node_tile": best["node_tile"],
                    "graph_chunk": best["graph_chunk"], "ms_per_substep": best["ms"],
                    "relative_to_baseline": best["relative"]},
           "baseline": {"graph_chunk": baseline[0], "node_tile": baseline[1],
                        "brick_variant": baseline[2]},
           "trials": trials, "substeps_advanced": advanced}
    if key is not None:
        _cache[key] = out
    return out
