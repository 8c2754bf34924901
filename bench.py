#!/usr/bin/env python
"""Benchmark: batched TLMPM cutting substeps on GB300.

Workload: 256 uneven cuboid scenes (particle counts log-uniform in 4k-64k,
E log-uniform 1e4-1e6 Pa, nu uniform 0.25-0.45, seeded blade planes and
speeds 0.05-0.5 m/s, per-scene CFL substep), held in one packed batch and
advanced by CUDA-graph launches.  One "step" is one substep of every scene.
Metric: particle-substeps/s (whole job, all ranks).

Keys beyond the value: the plain one-scene-per-launch path on the same scenes
(``plain``), the end-to-end rate through the C ABI with per-step host I/O
(``e2e``), the dominant kernel's roofline (``roofline``, live CUDA events),
sampled SM clocks (``clocks``) and the FP64 oracle on the host cores
(``cpu_baseline``).  ``--impl reference`` times the oracle alone.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bm_inputs as bi  # noqa: E402

METRIC = "particle-substeps/s (batched, 256 uneven scenes)"
UNIT = "particle-substeps/s"
WORKLOAD = "batched 256 uneven neo-Hookean cuboids, 4k-64k particles, 1 cut each"
N_SCENES = 256
SEED = 2
SMS = 152
FP32_LANES = 128
FALLBACK_HBM_GBS = 6800.0

# Per-kernel compulsory traffic (bytes) and FP32 work (flop, FMA = 2) per
# particle, per node, per occupied slot and per 4x4x4-cell brick: the reads
# and writes of each kernel's own inputs and outputs, with brick-tile
# partials counted at 3.375 tiles per slot (6^3 tile nodes per 4^3 cells).
KERNEL_MODEL = {
    # contact, labels and stress are computed in the P2G brick kernel's
    # staging phase: it reads x, v, F, masks, the fractional offset and the
    # D/u_t flag (81 B) and writes the pending label; D and u_t (16 B) are
    # read only for flagged particles and written only where they change, so
    # they are not counted (the cell of a particle comes from the brick's
    # cell ranges, not from memory)
    "k_p2g_brick": {"bytes": (82, 0, 108, 2000), "flops": (1470, 0, 0, 0)},
    "k_p2g_node": {"bytes": (0, 12, 140, 0), "flops": (0, 0, 40, 0)},
    "k_g2p_musl": {"bytes": (68, 0, 162, 1080), "flops": (570, 0, 0, 0)},
    "k_musl_node": {"bytes": (0, 12, 86, 0), "flops": (0, 0, 20, 0)},
    "k_fupd": {"bytes": (97, 0, 54, 1080), "flops": (650, 0, 0, 0)},
}
# the substep's small kernels (bytes only): the tool step reads the bricks'
# wrench partials (48 B per brick); the slot rebuild reads each node's dirty
# flag and code count and writes its slot count (3 B per node), writes each
# brick's tile descriptors (4 B per tile node) and partial-sum range, and,
# per node, the slot offset and the first-slot entries of the <= 8 covering
# bricks (36 B) and each slot's code (8 B); the recount of the dirty nodes'
# codes (the particles of 27 cells each) comes on top
SMALL_KERNEL_BYTES = {
    "k_tool": (0, 0, 0, 48),
    "k_slot_count": (0, 3, 0, 0),
    "k_brick_tiles": (0, 0, 0, 4 * 216 + 8),
    "k_slot_scan": (0, 0, 0, 8),
    "k_slot_fill": (0, 37, 8, 0),
}
STEP_ALGORITHMIC_BYTES = 156  # per particle-substep: the state the method must move
LATE_FIRST = 900              # first substep of the late timing window (of the 1,000-substep rollout)
LAUNCHES_PER_SUBSTEP = 10     # kernels one batched substep launches (no pair contact)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.path = tempfile.mktemp(prefix="bm_clocks_", suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def code_hash(text: str) -> str:
    """Hash of a CUDA source's code: comments, trailing blanks and empty lines
    removed, so that an edit of the comments keeps a capture's key."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", l).rstrip() for l in text.splitlines()]
    return hashlib.sha256("\n".join(l for l in lines if l).encode()).hexdigest()[:16]


def kernel_source_hash() -> str:
    src = os.path.join(ROOT, "paper_2609_27342_gb300", "csrc", "bm_kernels.cu")
    return code_hash(open(src).read())


def ncu_traffic(kernel: str, units: dict):
    """Per-launch DRAM traffic from the committed ncu summary, scaled by units,
    or None when the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_code_sha256_16") != kernel_source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k:
        return None
    return k["bytes_per_particle"] * units["particles"]


# ---------------------------------------------------------------------------
# CPU oracle timing (host cores)
# ---------------------------------------------------------------------------

def oracle_rate(scenes, seconds: float = 12.0, min_rounds: int = 2, max_rounds: int = 10 ** 6,
                threads: int = 0):
    """Run oracle substeps of the given scenes in parallel threads until the
    time budget is spent.  Returns (particle-substeps/s, threads, rounds)."""
    from oracle import oracle as O
    O.build()
    threads = threads or os.cpu_count() or 1
    objs = [O.OracleScene(sc) for sc in scenes]
    pool = ThreadPoolExecutor(max_workers=threads)
    total, rounds = 0, 0
    t0 = time.perf_counter()
    while rounds < max_rounds and (rounds < min_rounds or time.perf_counter() - t0 < seconds):
        list(pool.map(lambda o: o.step(1), objs))
        total += sum(o.n for o in objs)
        rounds += 1
    wall = time.perf_counter() - t0
    pool.shutdown()
    return total / wall, min(threads, len(objs)), rounds, wall


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_scenes(rank: int, n_scenes: int = N_SCENES):
    """The batch of one rank: 256 uneven scenes seeded per rank (rank 0 uses
    the workload's seed), so ranks hold independent shards of the work.  A
    smaller n_scenes takes the first scenes of the same stream (a slice of
    the workload for profiling; the benchmark's value always uses all 256)."""
    return bi.batched_scenes(N_SCENES, seed=SEED + rank, n_substeps=100000)[:n_scenes]


def reduce_over_ranks(dist, ms: float, particles: int, device="cuda"):
    """(max of the timed milliseconds, sum of the particles) over all ranks;
    the job's throughput is the summed work over the slowest rank's time."""
    if dist is None:
        return ms, particles
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(particles)], device=device, dtype=torch.float64)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n.item()))


def run_native(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2609_27342_gb300 import build as B
    B.build()
    import paper_2609_27342_gb300 as pkg
    pkg.load()

    scenes = rank_scenes(rank, args.scenes)
    n_particles = sum(s.n for s in scenes)
    stream = torch.cuda.Stream()
    fps = [pkg.footprint(s) for s in scenes]
    nodes = [f[1] for f in fps]
    n_bricks = sum(f[2] for f in fps)

    # plain one-scene-per-launch path on the same scenes
    plain_objs = [pkg.Scene(s, stream=stream) for s in scenes]
    plain_steps = args.plain_steps
    plain_rate = None
    if plain_steps > 0:
        for o in plain_objs:
            o.step(1)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for o in plain_objs:
                o.step(plain_steps)
            e1.record(stream)
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1)
        plain_rate = n_particles * plain_steps / (plain_ms * 1e-3)
        log(f"plain path: {plain_rate:.3e} p-s/s ({plain_ms:.1f} ms for {plain_steps} substeps)")

    def make_batch(members):
        b = pkg.Batch(max_particles=n_particles, max_nodes=sum(nodes), max_scenes=len(scenes),
                      max_bricks=n_bricks, stream=stream)
        for o in members:
            b.add(o)
        return b

    # launch shape: autotuned (untimed) on a throwaway copy of the workload, so
    # that the timed substeps start from the scenes' initial state, unless
    # given on the command line
    if args.chunk and args.ntile and args.variant is not None:
        shape = {"graph_chunk": args.chunk, "node_tile": args.ntile,
                 "brick_variant": args.variant, "autotuned": False}
    else:
        from paper_2609_27342_gb300.autotune import autotune
        probe = [pkg.Scene(s, stream=stream) for s in scenes]
        tb = make_batch(probe)
        tuned = autotune(tb, stream)
        tb.close()
        for o in probe:
            o.close()
        del probe, tb
        shape = dict(tuned["best"], autotuned=True, candidates=len(tuned["trials"]))
        for t in tuned["trials"]:
            log(f"  autotune trial {t}")
        log(f"autotune: {tuned['best']}")
    batch = make_batch(plain_objs)
    batch.set_tiles(shape["graph_chunk"], shape["node_tile"], shape["brick_variant"])
    # warm-up (also captures the graphs)
    batch.step(args.warmup)
    torch.cuda.synchronize()
    infos = [o.info() for o in plain_objs]
    n_slots = sum(i.n_slots for i in infos)
    n_nodes = sum(i.n_nodes for i in infos)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms, job_particles = reduce_over_ranks(dist, e0.elapsed_time(e1), n_particles)
    value = job_particles * args.steps / (ms * 1e-3)
    err_bits = batch.errors()

    # per-kernel device times over the same number of substeps (live events)
    prof = batch.profile(max(3, min(args.steps, 20)))
    ktimes = {k: v[0] / max(v[1], 1) for k, v in prof.items()}
    units = {"particles": n_particles, "nodes": n_nodes, "slots": n_slots, "bricks": n_bricks}
    dom = max(KERNEL_MODEL, key=lambda k: ktimes.get(k, 0.0))
    mb, mf = KERNEL_MODEL[dom]["bytes"], KERNEL_MODEL[dom]["flops"]
    alg_bytes = mb[0] * n_particles + mb[1] * n_nodes + mb[2] * n_slots + mb[3] * n_bricks
    alg_flops = mf[0] * n_particles + mf[1] * n_nodes + mf[2] * n_slots + mf[3] * n_bricks
    t_dom = ktimes[dom] * 1e-3
    hbm_peak, hbm_src = measured_peaks()
    sm_mhz = clk.get("sm_mhz") or 1900.0
    alu_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    gbs = alg_bytes / t_dom / 1e9
    tfs = alg_flops / t_dom / 1e12
    hbm_frac, alu_frac = gbs / hbm_peak, tfs / alu_peak
    if hbm_frac >= alu_frac:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(hbm_frac, 4), "peak_source": hbm_src}
    else:
        roof = {"bound": "alu", "achieved": round(tfs, 3), "peak": round(alu_peak, 2),
                "unit": "TFLOP/s", "frac": round(alu_frac, 4),
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (sampled)"}
    # the FP32 FMA ceiling measured on this GPU (independent FMA chains on
    # every SM), beside the one derived from unit counts and the clock
    fma = ctypes.c_double(0.0)
    pkg._abi.check(pkg.load().bm_fp32_fma_peak(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(fma)))
    roof["alu_peak_measured_tflops"] = round(fma.value, 2)
    roof["alu_frac_of_measured"] = round(tfs / fma.value, 4) if fma.value > 0 else None
    traffic = ncu_traffic(dom, units)
    roof.update({"kernel": dom, "traffic": traffic, "algorithmic_bytes": alg_bytes,
                 "algorithmic_flops": alg_flops, "avg_launch_ms": round(ktimes[dom], 4),
                 "hbm_frac": round(hbm_frac, 4), "alu_frac": round(alu_frac, 4),
                 "kernel_ms": {k: round(v, 4) for k, v in ktimes.items()}})
    # every kernel of the substep: algorithmic bytes per launch over its
    # live CUDA-event time, against the measured HBM peak
    per = {}
    for k, mb in [(k, m["bytes"]) for k, m in KERNEL_MODEL.items()] + list(SMALL_KERNEL_BYTES.items()):
        t = ktimes.get(k, 0.0)
        if t <= 0.0:
            continue
        b = mb[0] * n_particles + mb[1] * n_nodes + mb[2] * n_slots + mb[3] * n_bricks
        per[k] = {"ms": round(t, 4), "bytes": int(b), "gbs": round(b / (t * 1e-3) / 1e9, 1),
                  "hbm_frac": round(b / (t * 1e-3) / 1e9 / hbm_peak, 4)}
    roof["kernels"] = per
    step_ms = ms / args.steps
    step_roof = STEP_ALGORITHMIC_BYTES * n_particles / (step_ms * 1e-3) / 1e9

    # late window: the same batch advanced (untimed) to substep LATE_FIRST of
    # its 1,000-substep rollout, where most bricks hold cut faces, then the
    # same number of substeps timed again (the early window above starts at
    # the rollout's beginning, where the cuts are still shallow)
    late = None
    done = args.warmup + args.steps + max(3, min(args.steps, 20))
    if args.late_window and done < LATE_FIRST:
        batch.step(LATE_FIRST - done)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0.record(stream)
        batch.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms_late, _ = reduce_over_ranks(dist, e0.elapsed_time(e1), n_particles)
        prof_late = batch.profile(max(3, min(args.steps, 20)))
        late = {"value": job_particles * args.steps / (ms_late * 1e-3), "unit": UNIT,
                "first_substep": LATE_FIRST, "substeps": args.steps,
                "ms_per_step": ms_late / args.steps,
                "step_hbm_frac": round(STEP_ALGORITHMIC_BYTES * n_particles /
                                       (ms_late / args.steps * 1e-3) / 1e9 / hbm_peak, 4),
                "kernel_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in prof_late.items()}}
        log(f"late window: {late}")

    # end to end through the C ABI on a fresh copy of the workload, over the
    # same substeps as the device-timed region: every substep the tool states
    # go in from pinned host memory and the reaction wrenches come back to it
    e2e_objs = [pkg.Scene(s, stream=stream) for s in scenes]
    eb = make_batch(e2e_objs)
    eb.set_tiles(shape["graph_chunk"], shape["node_tile"], shape["brick_variant"])
    n = len(e2e_objs)
    h_states = torch.empty((n, 18), dtype=torch.float64, pin_memory=True)
    h_wr = torch.empty((n, 6), dtype=torch.float64, pin_memory=True)
    pose = np.stack([o.tool_state() for o in e2e_objs])
    vel = pose[:, 12:15].copy()
    dts = np.array([s.dt for s in scenes])

    def e2e_substep():
        pose[:, 0:3] += vel * dts[:, None]
        h_states.numpy()[:] = pose
        eb.set_tool_states_ptr(h_states.data_ptr(), n, False)
        eb.step(1)
        eb.tool_wrenches_ptr(h_wr.data_ptr(), n, False)

    for _ in range(args.warmup):
        e2e_substep()
    e2e_steps = args.steps
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_substep()
    wall, _ = reduce_over_ranks(dist, (time.perf_counter() - t0) * 1e3, n_particles)
    e2e_value = job_particles * e2e_steps / (wall * 1e-3)
    eb.close()
    for o in e2e_objs:
        o.close()
    del e2e_objs, eb

    # adjoint calibration workload: 32,000 particles, 200 substeps, checkpoint
    # every 20, loss on the reaction-force trajectory against a target made at
    # E = 1.5e5 Pa; gradient vs central differences (relative step 1e-3)
    adjoint = None
    if args.adjoint and rank == 0:
        from paper_2609_27342_gb300.calibration import force_loss_and_grad, forces
        na = 200
        target = forces(bi.calibration_scene(E=1.5e5), na)
        spec = bi.calibration_scene()
        force_loss_and_grad(spec, target, na, every=20)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss, g = force_loss_and_grad(spec, target, na, every=20)
        torch.cuda.synchronize()
        t_fb = time.perf_counter() - t0
        t0 = time.perf_counter()
        forces(spec, na)
        torch.cuda.synchronize()
        t_f = time.perf_counter() - t0

        def lossf(**kw):
            return float(np.sum((forces(bi.calibration_scene(**kw), na) - target) ** 2))

        fd = {"E": (lossf(E=1.001e5) - lossf(E=0.999e5)) / 200.0,
              "nu": (lossf(nu=0.3003) - lossf(nu=0.2997)) / 6e-4,
              "speed": (lossf(speed=0.2002) - lossf(speed=0.1998)) / 4e-4}
        grad = {"E": g["E"], "nu": g["nu"], "speed": -float(g["v_seg"][0, 2])}
        adjoint = {"workload": "calibration cuboid, 32,000 particles, 200 substeps, "
                               "checkpoint every 20", "loss": loss, "grad": grad,
                   "fd_rel_step_1e-3": fd,
                   "rel_err_vs_fd": {k: abs(grad[k] - fd[k]) / abs(fd[k]) for k in fd},
                   "forward_s": t_f, "forward_backward_s": t_fb,
                   "particle_substeps_per_s_fwd_bwd": spec.n * na / t_fb}
        log(f"adjoint: {adjoint}")

    # single-cut cuboid (16,000 particles, plain path) and the cylinder with
    # two intersecting cuts, a push, a two-way tool and pair contact (about
    # 251k particles, plain path), timed once the blade is in the material
    configs = None
    if args.configs and rank == 0:
        configs = {}
        sc0 = bi.single_cut_cuboid()
        g0 = pkg.Scene(sc0, stream=stream)
        g0.step(10)
        torch.cuda.synchronize()
        e0.record(stream)
        g0.step(100)
        e1.record(stream)
        torch.cuda.synchronize()
        r0 = sc0.n * 100 / (e0.elapsed_time(e1) * 1e-3)
        g0.close()
        configs["single_cut"] = {"workload": "single-cut neo-Hookean cuboid, 16,000 particles",
                                 "path": "plain (one scene per launch)", "value": r0, "unit": UNIT,
                                 "substeps_timed": 100}
        sc1 = bi.cylinder_cuts_push()
        g1 = pkg.Scene(sc1, stream=stream)
        g1.step(100)  # the blade reaches the top of the cylinder
        torch.cuda.synchronize()
        e0.record(stream)
        g1.step(200)
        e1.record(stream)
        torch.cuda.synchronize()
        r1 = sc1.n * 200 / (e0.elapsed_time(e1) * 1e-3)
        # the same substeps through a one-scene batch (CUDA-graph launches)
        fp1 = pkg.footprint(sc1)
        b1 = pkg.Batch(max_particles=sc1.n, max_nodes=fp1[1], max_scenes=1, max_bricks=fp1[2],
                       pair_contact=True, stream=stream)
        g1b = pkg.Scene.in_batch(b1, sc1)
        b1.step(100)
        torch.cuda.synchronize()
        e0.record(stream)
        b1.step(200)
        e1.record(stream)
        torch.cuda.synchronize()
        r1b = sc1.n * 200 / (e0.elapsed_time(e1) * 1e-3)
        builds = int(g1b.info().contact_list_builds)
        g1b.close()
        b1.close()
        configs["cylinder"] = {"workload": "cylinder 0.2 m x r 0.02 m, dx 2 mm, two intersecting "
                                           "cuts and a push, 0.2 kg two-way tool, pair contact",
                               "particles": sc1.n, "path": "plain (one scene per launch)",
                               "value": r1, "unit": UNIT, "substeps_timed": 200,
                               "first_substep": 100, "error_bits": int(g1.info().error_bits),
                               "graph_path_value": r1b,
                               "graph_path": "one-scene batch (CUDA-graph launches), same substeps",
                               "contact_list_builds_in_300_substeps": builds}
        # reference-grid surface of the cylinder mid-stroke (visual only; not
        # part of the substep): full rebuild from the codes + embedding, and
        # the embedding alone, each call timed by the wall clock (it
        # synchronises to return the vertex and triangle counts)
        from paper_2609_27342_gb300.surface import Surface
        surf = Surface(g1, (2, 2, 2))
        nv, nt = surf.update()
        reps = 20
        t0 = time.perf_counter()
        for _ in range(reps):
            surf.update(rebuild=True)
        t_rebuild = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        for _ in range(reps):
            surf.update(rebuild=False)
        t_embed = (time.perf_counter() - t0) / reps
        lat = (2 * 100 + 1) * (2 * 20 + 1) * (2 * 20 + 1)
        configs["surface"] = {"workload": "cylinder surface at substep 300 (cut 0 mid-stroke), "
                                          "sub-cell lattice 2x2x2 per cell",
                              "vertices": nv, "triangles": nt, "lattice_cells": lat,
                              "rebuild_and_embed_ms": 1e3 * t_rebuild, "embed_ms": 1e3 * t_embed,
                              "lattice_cells_per_s": lat / t_rebuild, "calls_timed": reps}
        surf.close()
        g1.close()
        log(f"configs: {configs}")

    # parity of the batched path in the timed launch shape: the benchmark's
    # smallest scene in a one-scene batch, 400 substeps (the blade is well
    # into the material by then), against the FP64
    # oracle on the host (position error relative to the domain size)
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as O
        i0 = int(np.argmin([s.n for s in scenes]))
        sp = scenes[i0]
        pb = pkg.Batch(max_particles=sp.n, max_nodes=fps[i0][1], max_scenes=1, max_bricks=fps[i0][2],
                       stream=stream)
        gp = pkg.Scene(sp, stream=stream)
        pb.add(gp)
        pb.set_tiles(shape["graph_chunk"], shape["node_tile"], shape["brick_variant"])
        pb.step(400)
        r = gp.read("x", "mask1", "mask2")
        op = O.OracleScene(sp)
        op.step(400)
        dom = float(np.max(sp.X.max(0) - sp.X.min(0)))
        od = op.get("digits")[:, 0].astype(int)
        gdig = np.where(r["mask1"] & 1, 1, np.where(r["mask2"] & 1, 2, 0))
        parity = {"scene": i0, "particles": sp.n, "substeps": 400, "path": "batched, timed launch shape",
                  "pos_err_max_rel_domain": float(np.abs(r["x"] - op.get("x")).max() / dom),
                  "label_disagreement": int((od != gdig).sum()), "labelled": int((od > 0).sum())}
        pb.close()
        gp.close()
        log(f"parity: {parity}")

    # continuous-batching server on a Poisson request stream (rollouts of
    # 8k-500k particles, 200-2000 substeps, 1-3 cuts), admission by an HBM budget
    # (one server per GPU; requests routed to ranks by assigned work, the same
    # assignment computed on every rank; statistics combined on the host)
    serving = None
    if args.serve_requests > 0:
        from paper_2609_27342_gb300.serving import serve_sharded
        reqs = bi.serving_requests(n_requests=args.serve_requests, seed=3)
        budget = int(args.serve_budget_gb * (1 << 30))
        st = serve_sharded(reqs, rank, world, budget, dist=dist, max_chunk=16,
                           node_tile=shape["node_tile"], brick_variant=shape["brick_variant"])
        serving = {"requests": st["requests"], "ranks": st["ranks"], "rate_hz": 50,
                   "budget_gb": args.serve_budget_gb,
                   "throughput": st["throughput"], "unit": UNIT, "wall_s": st["wall_s"],
                   "offered_load": st.get("offered_load"),
                   "over_batched": st["throughput"] / value if value else None,
                   "step_ms_p50": st["step_ms_p50"], "step_ms_p99": st["step_ms_p99"],
                   "request_latency_s_p50": st["request_latency_s_p50"],
                   "request_latency_s_p99": st["request_latency_s_p99"],
                   "queue_latency_s_p50": st.get("queue_latency_s_p50"),
                   "queue_latency_s_p99": st.get("queue_latency_s_p99"),
                   "host_s": st.get("host_s")}
        log(f"serving: {serving}")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = scenes[:16]
        rate, thr, rounds, wall_c = oracle_rate(sample, seconds=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"first 16 of the 256 scenes ({sum(s.n for s in sample)} particles), "
                         f"{rounds} substeps each, FP64 C oracle, one scene per thread, "
                         f"{wall_c:.1f} s wall"}
        # the single-cut cuboid (16,000 particles) on one host core
        from oracle import oracle as O
        o0 = O.OracleScene(bi.single_cut_cuboid())
        t0 = time.perf_counter()
        o0.step(100)
        cpu["single_cut_1_core"] = {"value": o0.n * 100 / (time.perf_counter() - t0), "unit": UNIT,
                                    "sample": "substeps 0-99 of the 16,000-particle single-cut "
                                              "cuboid, FP64 oracle, one thread"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.scenes == N_SCENES else
                       f"first {args.scenes} of the 256 scenes of: {WORKLOAD} (profiling slice)",
                       "scenes": len(scenes), "particles": n_particles,
                       "job_particles": job_particles, "seeds": f"{SEED}..{SEED + world - 1} (one per rank)",
                       "nodes": n_nodes, "slots": n_slots, "seed": SEED,
                       "bricks": n_bricks, "substeps_timed": args.steps,
                       "windows": {"value": f"substeps {args.warmup}..{args.warmup + args.steps - 1} "
                                            "of the 1,000-substep rollout",
                                   "late_window": f"substeps {LATE_FIRST}..{LATE_FIRST + args.steps - 1}"
                                   if late else None},
                       "launch_shape": shape,
                       "parallelism": f"scene-sharded x{world} (each rank its own batch)",
                       "l2": "inputs larger than L2 (state ~1.2 GB vs 129 MB L2)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 18 * 8,
                    "d2h_bytes_per_step": n * 6 * 8, "steps": e2e_steps,
                    "api": "bm_batch_set_tool_states + bm_batch_step + bm_batch_tool_wrenches"},
            "gpu_launches": LAUNCHES_PER_SUBSTEP * args.steps,
            "roofline": roof,
            "step_hbm_roofline": {"bytes_per_particle_substep": STEP_ALGORITHMIC_BYTES,
                                  "achieved": round(step_roof, 1), "peak": hbm_peak,
                                  "unit": "GB/s", "frac": round(step_roof / hbm_peak, 4)},
            "late_window": late,
            "plain": {"value": plain_rate, "unit": UNIT, "substeps": plain_steps,
                      "launches_per_substep_per_scene": LAUNCHES_PER_SUBSTEP},
            "batched_over_plain": (value / world / plain_rate) if plain_rate else None,
            "clocks": clk,
            "serving": serving,
            "adjoint": adjoint,
            "parity": parity,
            "configs": configs,
            "cpu_baseline": cpu,
            "error_bits": err_bits,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    scenes = bi.batched_scenes(N_SCENES, seed=SEED, n_substeps=100000)[:16]
    from oracle import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    objs = [O.OracleScene(sc) for sc in scenes]
    pool = ThreadPoolExecutor(max_workers=threads)
    for _ in range(args.warmup):
        list(pool.map(lambda o: o.step(1), objs))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        list(pool.map(lambda o: o.step(1), objs))
    wall = time.perf_counter() - t0
    pool.shutdown()
    n = sum(o.n for o in objs)
    value = n * args.steps / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "scenes": N_SCENES, "seed": SEED,
                   "sample": f"first 16 scenes ({n} particles) per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(threads, len(objs)),
                         "kind": "oracle",
                         "sample": f"first 16 of the 256 scenes, {args.steps} substeps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_cylinder_profile(args):
    """Per-kernel CUDA-event times of the cylinder program (252,800 particles,
    two-way tool, pair contact) in a one-scene batch, at four points of the
    program; one JSON line."""
    import torch
    from paper_2609_27342_gb300 import build as B
    B.build()
    import paper_2609_27342_gb300 as pkg
    pkg.load()
    sc = bi.cylinder_cuts_push()
    fp = pkg.footprint(sc)
    stream = torch.cuda.Stream()
    b = pkg.Batch(max_particles=sc.n, max_nodes=fp[1], max_scenes=1, max_bricks=fp[2], pair_contact=True,
                  stream=stream)
    g = pkg.Scene.in_batch(b, sc)
    out = {"workload": "cylinder program (two intersecting cuts and a push, two-way tool, pair contact)",
           "particles": sc.n, "points": {}}
    done = 0
    for at in (300, 900, 2200, 2850):
        b.step(at - done)
        done = at
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(20)
        e1.record(stream)
        torch.cuda.synchronize()
        done += 20
        builds0 = int(g.info().contact_list_builds)
        prof = b.profile(10)
        done += 10
        out["points"][str(at)] = {
            "ms_per_substep": e0.elapsed_time(e1) / 20,
            "list_builds_in_10_profiled": int(g.info().contact_list_builds) - builds0,
            "kernel_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in prof.items() if v[1]}}
    out["error_bits"] = int(g.info().error_bits)
    b.close()
    print(json.dumps(out), flush=True)


def run_adjoint_only(args):
    """The calibration workload (32,000 particles, 200 substeps, checkpoint
    every 20): one forward + backward after a warm-up; one JSON line."""
    import torch
    from paper_2609_27342_gb300 import build as B
    B.build()
    import paper_2609_27342_gb300 as pkg
    pkg.load()
    from paper_2609_27342_gb300.calibration import force_loss_and_grad, forces
    na = 200
    target = forces(bi.calibration_scene(E=1.5e5), na)
    spec = bi.calibration_scene()
    force_loss_and_grad(spec, target, na, every=20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, g = force_loss_and_grad(spec, target, na, every=20)
    torch.cuda.synchronize()
    print(json.dumps({"workload": "calibration cuboid, 32,000 particles, 200 substeps, checkpoint every 20",
                      "forward_backward_s": time.perf_counter() - t0, "loss": loss,
                      "grad": {"E": g["E"], "nu": g["nu"], "speed": -float(g["v_seg"][0, 2])}}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--chunk", type=int, default=0, help="fix the graph chunk (with --ntile, "
                    "--variant; otherwise the launch shape is autotuned)")
    ap.add_argument("--ntile", type=int, default=0)
    ap.add_argument("--variant", type=int, default=None)
    ap.add_argument("--plain-steps", type=int, default=4)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false")
    ap.add_argument("--no-configs", dest="configs", action="store_false")
    ap.add_argument("--no-late-window", dest="late_window", action="store_false")
    ap.add_argument("--scenes", type=int, default=N_SCENES,
                    help="take the first scenes of the workload only (profiling slices)")
    ap.add_argument("--cylinder-profile", action="store_true",
                    help="only the per-kernel times of the cylinder program")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only one forward + backward of the calibration workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.cylinder_profile:
        run_cylinder_profile(args)
    elif args.adjoint_only:
        run_adjoint_only(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
