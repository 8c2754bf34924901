"""Launch-shape autotuner for a batch of scenes.

The batched substep has launch parameters that do not change its results
(every sum is taken in a fixed order, and the kernel variants share their
arithmetic): the occupancy of each brick kernel (resident CTAs per SM of the
per-brick P2G, G2P+MUSL and F-update kernels, i.e. registers per thread
against latency hiding; one of three choices each, encoded in the brick
variant as p2g + 3 g2p + 9 fupd), the node tile (threads per CTA of the
per-node kernels) and the number of substeps captured in one CUDA graph.  The
tuner times candidate shapes on the batch itself with CUDA events on the
batch's stream and keeps the fastest: one brick kernel's occupancy at a time
(the kernels run one after the other, so their choices are independent),
then the node tile, then the graph chunk.

Every probe advances the simulation: tuning is a warm-up of the batch, not a
side computation.
"""
from __future__ import annotations

import math
from typing import Dict, Iterable, List, Optional

OCC_CHOICES = (0, 1, 2)   # per brick kernel
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


def pick(rows: List[dict], incumbent: Optional[dict], margin: float) -> dict:
    """The fastest of ``rows`` by relative time, unless it beats the
    ``incumbent`` (already timed) by less than ``margin``: short probes carry
    a timing noise of about a percent, and a shape that wins by less is not
    known to be faster."""
    best = min(rows, key=lambda r: r["relative"])
    if incumbent is not None and best is not incumbent and \
            best["relative"] > incumbent["relative"] * (1.0 - margin):
        return incumbent
    return best


def variant(p2g: int, g2p: int, fupd: int) -> int:
    """Brick variant of one occupancy choice per brick kernel."""
    return p2g + 3 * g2p + 9 * fupd


def autotune(batch, stream, key: Optional[tuple] = None, substeps: int = 16, rounds: int = 1,
             occ_choices: Iterable[int] = OCC_CHOICES, node_tiles: Iterable[int] = NODE_TILES,
             graph_chunks: Iterable[int] = GRAPH_CHUNKS, baseline=(16, 128, 0),
             margin: float = 0.01) -> dict:
    """Pick each brick kernel's occupancy in turn (the others held at their
    best so far) at a 16-substep graph, then the node tile, then the graph
    chunk; set the winner on ``batch`` and return
    ``{"best": {...}, "trials": [...], "substeps_advanced": n}``.

    The probes advance the scenes, and the cost of a substep drifts as cuts
    progress, so every candidate is timed between two timings of a fixed
    ``baseline`` shape (graph chunk, node tile, variant) and ranked by its
    time relative to their mean; a candidate replaces the shape it would
    change only when it is faster by more than ``margin`` (see ``pick``).
    ``stream`` is the torch stream the batch launches on.  With ``key`` the result is cached for this process and a
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
    def row(chunk, ntile, v):
        return next((r for r in trials if (r["graph_chunk"], r["node_tile"], r["brick_variant"]) ==
                     (chunk, ntile, v)), None)

    occ = [0, 0, 0]
    for k in range(3):          # P2G, G2P+MUSL, F update
        for c in occ_choices:
            o = list(occ)
            o[k] = c
            probe(16, baseline[1], variant(*o))
        rows = [r for r in trials if r["graph_chunk"] == 16 and r["node_tile"] == baseline[1]]
        best = pick(rows, row(16, baseline[1], variant(*occ)), margin)
        v = best["brick_variant"]
        occ = [v % 3, (v // 3) % 3, v // 9]
    for t in node_tiles:
        probe(16, t, variant(*occ))
    best = pick(trials, best, margin)
    for c in graph_chunks:
        probe(c, best["node_tile"], best["brick_variant"])
    best = pick(trials, best, margin)
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
