"""GPU parity of material-material contact (Eq. 10-13) and of the two-way
coupled tool (Eq. 14-16, Sec. III-G) against the FP64 oracle."""
import math

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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def colliding_blocks(speed=0.4):
    """Two blocks far apart in the reference grid (no shared stencil) whose
    current positions touch; they approach each other along x."""
    dx = 5e-3
    A = bi.lattice_cuboid((0.02, 0.02, 0.02), dx)
    B = bi.lattice_cuboid((0.02, 0.02, 0.02), dx, origin=(0.08, 0.0, 0.0))
    X = np.concatenate([A, B])
    sc = bi.Scene(X=X, dx=dx, V0=dx ** 3 / 8, gravity=(0, 0, 0), floor=False,
                  pair_contact=True, dt=1e-4)
    x = X.copy()
    nA = A.shape[0]
    x[nA:, 0] -= 0.06 - 0.0005   # gap of 2R - 0.5 mm: overlapping spheres soon
    v = np.zeros_like(X)
    v[:nA, 0] = speed
    v[nA:, 0] = -speed
    return sc, f32(x), f32(v), nA


def test_pair_contact_matches_oracle(pkg):
    sc, x, v, nA = colliding_blocks()
    o = O.OracleScene(sc)
    o.set("x", x)
    o.set("v", v)
    g = pkg.Scene(sc)
    g.write(x=x, v=v)
    for _ in range(3):
        o.step(10)
        g.step(10)
        r = g.read("x", "v")
        assert np.max(np.abs(r["x"] - o.get("x"))) <= 1e-5 * 0.1
        assert np.max(np.abs(r["v"] - o.get("v"))) <= 1e-3 * 0.4
    # contact really acted: the blocks slowed down
    assert np.mean(o.get("v")[:nA, 0]) < 0.9 * 0.4
    assert g.info().error_bits == 0


def test_pair_contact_conserves_momentum_on_gpu(pkg):
    """Eq. 13 impulses are exact negatives: total momentum is kept."""
    sc, x, v, nA = colliding_blocks(speed=0.8)
    g = pkg.Scene(sc)
    rng = np.random.default_rng(3)
    m1 = np.zeros(sc.n, np.uint32)
    m2 = np.zeros(sc.n, np.uint32)
    d = rng.integers(0, 3, sc.n)
    m1[d == 1] = 1
    m2[d == 2] = 1
    g.write(x=x, v=v, mask1=m1, mask2=m2)
    P0 = g.read("v")["v"].astype(np.float64).sum(0)
    for _ in range(40):
        g.step(1)
    P1 = g.read("v")["v"].astype(np.float64).sum(0)
    assert np.max(np.abs(P1 - P0)) < 1e-5 * 0.8 * sc.n


def test_cylinder_cuts_two_way_tool_and_contact(pkg):
    """A small cylinder cut by a dynamic (0.2 kg) blade on two intersecting
    strokes with pair contact on, then a lateral push with the blade inside
    the second cut (a non-cutting segment in contact): positions and the tool
    state follow the oracle over the whole program."""
    X = bi.lattice_cylinder(0.04, 0.01, 2e-3)
    mass = 0.2
    wz = -math.radians(30.0) / (20 * 5e-5)
    # blade normal after the -30 deg turn: rot_z(15 - 30) applied to +x
    c, sn = math.cos(math.radians(-15.0)), math.sin(math.radians(-15.0))
    # down 1.25 mm, withdraw clear of the top, rotate -30 deg in the air, cut
    # again, then push 0.6 mm along the blade normal without cutting
    segs = [bi.Segment(50, v=(0, 0, -0.5), cut_id=0), bi.Segment(60, v=(0, 0, 0.5), cut_id=0),
            bi.Segment(20, omega=(0, 0, wz), cut_id=-1), bi.Segment(70, v=(0, 0, -0.5), cut_id=1),
            bi.Segment(60, v=(0.2 * c, 0.2 * sn, 0.0), cut_id=-1)]
    blade = bi.Blade(pose_x=(0.02, 0.01, 0.0202), pose_R=bi.rot_z(15.0), mass=mass,
                     inertia=bi.plate_inertia(mass, 1e-3, 0.1, 0.1), segments=segs)
    sc = bi.Scene(X=X, E=5e4, nu=0.35, dx=2e-3, V0=(2e-3) ** 3 / 8, dt=5e-5, pair_contact=True,
                  blade=blade, G_c=5.0)
    o = O.OracleScene(sc)
    nst = 260
    g = pkg.Scene(sc, wrench_history=nst)
    o.step(nst)
    g.step(nst)
    L = float(np.max(sc.X.max(0) - sc.X.min(0)))
    err = np.max(np.abs(g.read("x")["x"] - o.get("x")))
    assert err <= 1e-5 * L, err
    to = o.tool()
    tg = g.tool_state()
    assert np.max(np.abs(tg[0:3] - to[0:3])) <= 1e-6 * L
    assert np.max(np.abs(tg[12:15] - to[12:15])) <= 1e-4 * max(1e-3, np.max(np.abs(to[12:15])))
    wo = o.wrench_history(0, nst)
    wg = g.wrench_history(0, nst)
    peak = np.max(np.abs(wo[:, :3]))
    assert peak > 0
    # the push is in contact: the reaction during it is a sizeable part of the peak
    assert np.max(np.abs(wo[200:, :3])) > 0.05 * peak
    ew = np.max(np.abs(wg[:, :3] - wo[:, :3])) / peak
    record("small_cylinder_push", pos_err=err / L, wrench_err=ew)
    assert ew <= 1e-4, ew
    codes_o, codes_g = o.get("code"), g.read("code")["code"]
    assert np.sum(codes_o != codes_g) <= max(1, 1e-4 * sc.n)
    assert len(np.unique(codes_g)) >= 3
    assert g.info().error_bits == 0


def test_pair_contact_checkpoint_and_batch_move_are_bitwise(pkg):
    """With material-material contact on, a checkpoint restore and a move into
    a batch mid-run both continue bit for bit: the candidate lists of the
    contact search travel with the particle state."""
    sc, x, v, nA = colliding_blocks(speed=0.8)
    fields = ("x", "v", "F", "pair_partner", "pair_u")
    g = pkg.Scene(sc)
    g.write(x=x, v=v)
    g.step(10)
    ck = g.checkpoint()
    g.step(15)
    ref = g.read(*fields)
    assert np.any(ref["pair_partner"] >= 0), "the blocks must be in contact"
    g.restore(ck)
    g.step(15)
    got = g.read(*fields)
    for k in fields:
        assert np.array_equal(got[k], ref[k]), k
    h = pkg.Scene(sc)
    h.write(x=x, v=v)
    h.step(10)
    fp = pkg.footprint(sc)
    b = pkg.Batch(max_particles=sc.n + 64, max_nodes=fp[1] + 64, max_scenes=2, pair_contact=True)
    b.add(h)
    b.step(15)
    got = h.read(*fields)
    for k in fields:
        assert np.array_equal(got[k], ref[k]), ("moved", k)
    b.close()
    g.close()
