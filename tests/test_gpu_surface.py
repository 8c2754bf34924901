"""GPU parity of the surface reconstruction (Sec. III-F) against the oracle.

Both sides get the same seeded state: the 16,000-particle single-cut cuboid
after one substep (so that cut 0's plane is recorded on each side by its own
run), with side codes and positions written by the test: cut 0 partial along
the blade's plane, cut 1 a full oblique cut without a recorded plane, and
each side of cut 1 displaced by its own translation plus a smooth field.

Bar: vertex and triangle counts, triangles and vertex codes bit-exact (they
are integer work); reference and current vertex positions within 1e-7 m
(float32 on coordinates of 0.1 m, about 2e-5 dx).  A batched scene's surface
equals the same scene's surface alone, bit for bit.
"""
import numpy as np
import pytest

import bm_inputs as bi
from oracle import oracle as O
from oracle import surface as S

pytestmark = pytest.mark.gpu

TOL = 1e-7


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2609_27342_gb300 as p
    from paper_2609_27342_gb300 import build
    build.build()
    p.load()
    return p


def synthetic_state(sc, seed=4):
    """Codes and positions written into both sides (not the method's output)."""
    X = np.asarray(sc.X, np.float64)
    rng = np.random.default_rng(seed)
    c = X.mean(0)
    # cut 0: the blade's plane x = 0.05, only the top 40 % labelled (a partial cut)
    top = X[:, 2] > X[:, 2].max() - 0.4 * (X[:, 2].max() - X[:, 2].min())
    s1 = np.where(top & (X[:, 0] < 0.05), 1, 0).astype(np.uint32)
    s2 = np.where(top & (X[:, 0] >= 0.05), 1, 0).astype(np.uint32)
    # cut 1: an oblique plane through the centre, full depth
    n1 = rng.normal(size=3)
    n1[0] = 0.3 * n1[0]
    n1 /= np.linalg.norm(n1)
    sd = (X - c) @ n1
    s1 |= np.where(sd < 0, 2, 0).astype(np.uint32)
    s2 |= np.where(sd >= 0, 2, 0).astype(np.uint32)
    u = 2e-4 * np.sin(40.0 * X[:, [1, 2, 0]]) + np.where((sd < 0)[:, None], -6e-4, 6e-4) * n1
    x = (X + u).astype(np.float32).astype(np.float64)
    return s1, s2, x


def oracle_surface(sc, s1, s2, x, planes, mask):
    r = S.reconstruct(sc.X, s1, s2, sc.dx, (2, 2, 2), planes, mask)
    r["cur"] = S.embed(r, sc.X, x, s1, s2, sc.dx, sc.origin)
    return r


def gpu_surface(pkg, g, s1, s2, x):
    from paper_2609_27342_gb300.surface import Surface

    g.write(x=x.astype(np.float32), mask1=s1, mask2=s2)
    f = Surface(g, (2, 2, 2))
    nv, nt = f.update()
    d = f.read()
    f.close()
    return nv, nt, d


def compare(d, nv, nt, r, s1, s2):
    assert nv == len(r["ref"]) and nt == len(r["tris"])
    assert np.array_equal(d["triangles"].astype(np.int64), r["tris"])
    assert np.array_equal(d["masks"][:, 0], s1[r["anchor"]])
    assert np.array_equal(d["masks"][:, 1], s2[r["anchor"]])
    assert np.abs(d["reference"] - r["ref"]).max() < TOL
    assert np.abs(d["vertices"] - r["cur"]).max() < TOL


def test_surface_parity_with_oracle(pkg):
    sc = bi.single_cut_cuboid()
    g = pkg.Scene(sc)
    g.step(1)
    o = O.OracleScene(sc)
    o.step(1)
    planes, mask = o.cut_planes()
    assert mask == 1
    s1, s2, x = synthetic_state(sc)
    nv, nt, d = gpu_surface(pkg, g, s1, s2, x)
    r = oracle_surface(sc, s1, s2, x, planes, mask)
    compare(d, nv, nt, r, s1, s2)
    # the surface is a closed chain; the pieces of cut 1 are separate
    T = d["triangles"].astype(np.int64)
    assert S.closed_chain(T)
    assert len(np.unique(S.components(nv, T))) == 2
    g.close()


def test_surface_uncut_box_and_rebuild(pkg):
    """No cut: the box closed form (counts and volume); an embed-only update
    keeps the topology; a rebuild after new codes changes it."""
    from paper_2609_27342_gb300.surface import Surface

    sc = bi.single_cut_cuboid()
    g = pkg.Scene(sc)
    f = Surface(g, (2, 2, 2))
    nv, nt = f.update()
    n = np.array([40, 20, 20])
    assert nv == np.prod(n + 1) - np.prod(n - 1)
    assert nt == 4 * (n[0] * n[1] + n[1] * n[2] + n[2] * n[0])
    d = f.read()
    vol = S.signed_volume(d["reference"].astype(np.float64), d["triangles"].astype(np.int64))
    assert vol == pytest.approx(0.1 * 0.05 * 0.05, rel=1e-5)
    assert np.abs(d["vertices"] - d["reference"]).max() == 0.0
    t = np.array([1e-3, -2e-3, 5e-4], np.float32)
    g.write(x=(np.asarray(sc.X, np.float32) + t))
    assert f.update(rebuild=False) == (nv, nt)
    d2 = f.read()
    assert np.array_equal(d2["triangles"], d["triangles"])
    assert np.abs(d2["vertices"] - (d["reference"] + t)).max() < TOL
    s1 = (np.asarray(sc.X)[:, 0] < 0.05).astype(np.uint32)
    g.write(mask1=s1, mask2=(1 - s1).astype(np.uint32))
    nv2, nt2 = f.update()
    assert nv2 > nv and nt2 > nt
    f.close()
    g.close()


def test_surface_of_batched_scene_matches_alone(pkg):
    """A scene inside a batch (its particles at a pool offset, its record not
    the first) gives the same surface as alone, bit for bit."""
    from paper_2609_27342_gb300.surface import Surface

    specs = bi.batched_scenes(3, seed=7)
    alone = pkg.Scene(specs[2])
    members = [pkg.Scene(s) for s in specs]
    fp = [pkg.footprint(s) for s in specs]
    b = pkg.Batch(max_particles=sum(s.n for s in specs), max_nodes=sum(f[1] for f in fp),
                  max_scenes=3, max_bricks=sum(f[2] for f in fp))
    for m in members:
        b.add(m)
    b.step(300)
    alone.step(300)
    outs = []
    for g in (alone, members[2]):
        f = Surface(g, (2, 2, 2))
        f.update()
        outs.append(f.read())
        f.close()
    for k in ("vertices", "reference", "triangles", "masks"):
        assert np.array_equal(outs[0][k], outs[1][k]), k
    assert (outs[0]["masks"] != 0).any()  # the cut has begun
    b.close()
    alone.close()


def test_surface_full_size_cylinder_properties(pkg):
    """The 252,800-particle cylinder after its first stroke has begun: the
    surface is a closed chain whose reference volume is the lattice voxels',
    and every vertex stays within a cell of its anchor particle."""
    from paper_2609_27342_gb300.surface import Surface

    sc = bi.cylinder_cuts_push()
    g = pkg.Scene(sc)
    g.step(700)
    f = Surface(g, (2, 2, 2))
    nv, nt = f.update()
    d = f.read()
    T = d["triangles"].astype(np.int64)
    assert S.closed_chain(T)
    vox = (sc.dx / 2) ** 3
    vol = S.signed_volume(d["reference"].astype(np.float64), T)
    assert vol == pytest.approx(sc.n * vox, rel=1e-4)
    m = g.read("x", "mask1", "mask2")
    assert ((m["mask1"] | m["mask2"]) != 0).sum() > 1000
    assert ((d["masks"][:, 0] | d["masks"][:, 1]) != 0).sum() > 100
    assert np.isfinite(d["vertices"]).all()
    f.close()
    g.close()


def test_surface_rejects_off_lattice_scene(pkg):
    from paper_2609_27342_gb300.surface import Surface

    sc = bi.single_cut_cuboid(jitter=0.2)
    g = pkg.Scene(sc)
    with pytest.raises(pkg.BMError):
        Surface(g, (2, 2, 2))
    g.close()


def test_surface_parity_anisotropic_lattice(pkg):
    """4 x 2 x 2 particles per cell (the 32,000-particle calibration cuboid):
    lattice spacing differs per axis; the same bit-exact topology and 1e-7 m
    positions against the oracle."""
    sc = bi.calibration_scene()
    g = pkg.Scene(sc)
    g.step(1)
    o = O.OracleScene(sc)
    o.step(1)
    planes, mask = o.cut_planes()
    assert mask == 1
    X = np.asarray(sc.X, np.float64)
    rng = np.random.default_rng(9)
    n1 = rng.normal(size=3)
    n1 /= np.linalg.norm(n1)
    sd = (X - X.mean(0)) @ n1
    s1 = np.where(sd < 0, 2, 0).astype(np.uint32)
    s2 = np.where(sd >= 0, 2, 0).astype(np.uint32)
    top = X[:, 2] > 0.03
    s1 |= np.where(top & (X[:, 0] < 0.05), 1, 0).astype(np.uint32)
    s2 |= np.where(top & (X[:, 0] >= 0.05), 1, 0).astype(np.uint32)
    x = (X + 3e-4 * np.cos(30.0 * X) + np.where((sd < 0)[:, None], 5e-4, -5e-4) * n1)
    x = x.astype(np.float32).astype(np.float64)
    from paper_2609_27342_gb300.surface import Surface

    g.write(x=x.astype(np.float32), mask1=s1, mask2=s2)
    f = Surface(g, (4, 2, 2))
    nv, nt = f.update()
    d = f.read()
    f.close()
    r = S.reconstruct(sc.X, s1, s2, sc.dx, (4, 2, 2), planes, mask)
    r["cur"] = S.embed(r, sc.X, x, s1, s2, sc.dx, sc.origin)
    compare(d, nv, nt, r, s1, s2)
    assert S.closed_chain(d["triangles"].astype(np.int64))
    g.close()
