"""Pins of the surface-reconstruction oracle (Sec. III-F) against closed forms.

Each case has a result fixed by geometry alone: the dual-contoured surface of
an axis-aligned box of lattice voxels is the box itself (vertex and triangle
counts, enclosed volume, Euler characteristic 2), a single voxel gives a cube
of 8 corners and 12 triangles, a cut along a lattice mid-plane gives two
closed boxes, a partial cut a closed surface with a zero-volume slit, and a
rigid motion of either side carries that side's surface with it.
"""
import numpy as np
import pytest

import bm_inputs as bi
from oracle import surface as S

DX = 0.002


def box(nx, ny, nz, per_axis=(2, 2, 2)):
    return bi.lattice_cuboid((nx * DX, ny * DX, nz * DX), DX, per_axis)


def uncoded(n):
    z = np.zeros(n, np.uint32)
    return z, z.copy()


def split_codes(X, axis, at, mask_rows=None):
    """Digit 1 below the plane X[axis] = at, digit 2 above (cut 0)."""
    lo = X[:, axis] < at
    s1 = lo.astype(np.uint32)
    s2 = (~lo).astype(np.uint32)
    if mask_rows is not None:
        s1 = s1 * mask_rows
        s2 = s2 * mask_rows
    return s1.astype(np.uint32), s2.astype(np.uint32)


def euler(nv, T):
    E = {(min(a, b), max(a, b)) for t in T for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    return nv - len(E) + len(T)


def test_single_voxel_is_a_cube():
    h = DX / 2
    X = np.array([[h / 2, h / 2, h / 2]])
    s1, s2 = uncoded(1)
    r = S.reconstruct(X, s1, s2, DX)
    V, T = r["ref"], r["tris"]
    assert len(V) == 8 and len(T) == 12
    # one representative at each corner of the voxel [0, h]^3
    corners = {tuple(np.round(v / h).astype(int)) for v in V}
    assert corners == {(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)}
    assert np.allclose(V, np.round(V / h) * h, atol=1e-15)
    assert S.signed_volume(V, T) == pytest.approx(h ** 3, rel=1e-12)
    assert S.directed_edges_paired(T)
    assert euler(len(V), T) == 2


@pytest.mark.parametrize("dims,per_axis", [((3, 2, 2), (2, 2, 2)), ((2, 3, 1), (2, 2, 2)),
                                           ((2, 2, 2), (4, 2, 2))])
def test_box_closed_form(dims, per_axis):
    X = box(*dims, per_axis=per_axis)
    s1, s2 = uncoded(len(X))
    r = S.reconstruct(X, s1, s2, DX, per_axis)
    V, T = r["ref"], r["tris"]
    n = np.array([dims[a] * per_axis[a] for a in range(3)])
    # cells touching the box but not inside it, one region each
    assert len(V) == np.prod(n + 1) - np.prod(n - 1)
    # one quad per boundary link, two triangles per quad
    assert len(T) == 2 * 2 * (n[0] * n[1] + n[1] * n[2] + n[2] * n[0])
    size = np.array(dims) * DX
    assert S.signed_volume(V, T) == pytest.approx(np.prod(size), rel=1e-9)
    assert S.directed_edges_paired(T)
    assert euler(len(V), T) == 2
    # every representative lies on the box's boundary
    L = r["lattice"]
    lo, hi = L.Xmin - L.h / 2, L.Xmin + (L.n - 0.5) * L.h
    dist = np.minimum(np.abs(V - lo), np.abs(V - hi)).min(axis=1)
    assert dist.max() < 1e-12


def test_qef_closed_forms():
    rng = np.random.default_rng(5)
    # three orthogonal planes meet at one point
    c = rng.normal(size=3)
    P = [c + [0, 1, 2], c + [3, 0, -1], c + [1, -2, 0]]
    N = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    assert np.allclose(S.qef_point(P, N), c, atol=1e-12)
    # one plane: the mass point (already on the plane)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    t1 = np.cross(n, [1, 0, 0])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    P = [c + a * t1 + b * t2 for a, b in rng.normal(size=(5, 2))]
    assert np.allclose(S.qef_point(P, [n] * 5), np.mean(P, axis=0), atol=1e-12)
    # two planes: the point of their line nearest the mass point
    P = [c + [0, 0.5, 0], c + [0.3, 0, 0], c + [0, -0.5, 0.2], c + [-0.1, 0, 0.7]]
    N = [[1, 0, 0], [0, 1, 0], [1, 0, 0], [0, 1, 0]]
    m = np.mean(P, axis=0)
    assert np.allclose(S.qef_point(P, N), [c[0], c[1], m[2]], atol=1e-12)


def test_hermite_of_a_cut_link():
    X = box(2, 1, 1)
    L = S.Lattice(X, DX)
    pl = np.zeros((32, 4))
    n = np.array([0.6, 0.8, 0.0])
    ja, jb = (1, 0, 0), (2, 0, 0)
    Xa, Xb = L.pos(ja), L.pos(jb)
    t = 0.3
    pl[3, :3] = n
    pl[3, 3] = n @ (Xa + t * (Xb - Xa))
    pa, pb = L.particle(*ja), L.particle(*jb)
    s1 = np.zeros(len(X), np.uint32)
    s2 = np.zeros(len(X), np.uint32)
    s1[pa] = 1 << 3
    s2[pb] = 1 << 3
    p, nout = S.link_hermite(L, s1, s2, pl, 1 << 3, ja, jb, pa, pb)
    assert np.allclose(p, Xa + t * (Xb - Xa), atol=1e-15)
    assert np.allclose(nout, n)  # digit 1 (s < 0) looks along +n
    p, nout = S.link_hermite(L, s1, s2, pl, 1 << 3, jb, ja, pb, pa)
    assert np.allclose(p, Xa + t * (Xb - Xa), atol=1e-15) and np.allclose(nout, -n)
    # a plane outside the link clamps to the nearer end; no plane: midpoint
    pl[3, 3] = n @ (Xa - 0.4 * (Xb - Xa))
    p, _ = S.link_hermite(L, s1, s2, pl, 1 << 3, ja, jb, pa, pb)
    assert np.allclose(p, Xa)
    p, nout = S.link_hermite(L, s1, s2, pl, 0, ja, jb, pa, pb)
    assert np.allclose(p, 0.5 * (Xa + Xb)) and np.allclose(nout, [1, 0, 0])
    # compatible codes: connected link, no Hermite data
    s2[pb] = 0
    assert S.link_hermite(L, s1, s2, pl, 1 << 3, ja, jb, pa, pb) is None


def test_regions_against_transitive_closure():
    """Union-find regions equal the components of the cell's link graph,
    computed by boolean matrix powers."""
    rng = np.random.default_rng(11)
    X = box(1, 1, 1)  # 2 x 2 x 2 lattice: the one interior cell holds all 8
    L = S.Lattice(X, DX)
    for _ in range(50):
        s1 = rng.integers(0, 4, len(X)).astype(np.uint32)
        s2 = (rng.integers(0, 4, len(X)).astype(np.uint32)) & ~s1
        parts, reg, nreg = S.cell_regions(L, s1, s2, (0, 0, 0))
        A = np.eye(8, dtype=bool)
        for q0, q1, _ in S.EDGES:
            p0, p1 = parts[q0], parts[q1]
            if S.conflict_bits(s1[p0], s2[p0], s1[p1], s2[p1]) == 0:
                A[q0, q1] = A[q1, q0] = True
        R = A.copy()
        for _ in range(8):
            R = (R.astype(int) @ A.astype(int)) > 0
        for a in range(8):
            for b in range(8):
                assert (reg[a] == reg[b]) == bool(R[a, b])
        assert nreg == len({tuple(R[q]) for q in range(8)})


@pytest.mark.parametrize("recorded", [False, True])
def test_full_cut_gives_two_closed_boxes(recorded):
    X = box(4, 2, 2)
    mid = 2 * DX
    s1, s2 = split_codes(X, 0, mid)
    pl = np.zeros((32, 4))
    pl[0] = [1, 0, 0, mid]
    r = S.reconstruct(X, s1, s2, DX, planes=pl, plane_mask=int(recorded))
    V, T = r["ref"], r["tris"]
    comp = S.components(len(V), T)
    assert len(np.unique(comp)) == 2
    half = 2 * DX * 2 * DX * 2 * DX
    for c in np.unique(comp):
        Tc = T[np.isin(T[:, 0], np.nonzero(comp == c)[0])]
        assert S.directed_edges_paired(Tc)
        assert S.signed_volume(V, Tc) == pytest.approx(half, rel=1e-6)
        assert euler(int((comp == c).sum()), Tc) == 2
    # the two cut faces coincide: the same point set on either side
    on = np.abs(V[:, 0] - mid) < 1e-9
    side = s1[r["anchor"]] == 1
    A = {tuple(np.round(v / 1e-7).astype(int)) for v in V[on & side]}
    B = {tuple(np.round(v / 1e-7).astype(int)) for v in V[on & ~side]}
    assert A == B and len(A) == 5 * 5


def test_partial_cut_is_a_closed_slit():
    X = box(4, 2, 2)
    mid = 2 * DX
    upper = (X[:, 2] > DX).astype(np.uint32)
    s1, s2 = split_codes(X, 0, mid, upper)
    pl = np.zeros((32, 4))
    pl[0] = [1, 0, 0, mid]
    r = S.reconstruct(X, s1, s2, DX, planes=pl, plane_mask=1)
    V, T = r["ref"], r["tris"]
    assert len(np.unique(S.components(len(V), T))) == 1
    assert S.directed_edges_paired(T)
    assert euler(len(V), T) == 2
    # the slit's two faces coincide: it encloses no volume
    assert S.signed_volume(V, T) == pytest.approx(4 * DX * 2 * DX * 2 * DX, rel=1e-9)


def test_oblique_cut_closed_pieces():
    X = box(4, 2, 2)
    n = np.array([1.0, 0.3, 0.2])
    n /= np.linalg.norm(n)
    off = n @ X.mean(0)
    sd = X @ n - off
    s1 = (sd < 0).astype(np.uint32)
    s2 = (sd >= 0).astype(np.uint32)
    pl = np.zeros((32, 4))
    pl[0, :3], pl[0, 3] = n, off
    r = S.reconstruct(X, s1, s2, DX, planes=pl, plane_mask=1)
    V, T = r["ref"], r["tris"]
    comp = S.components(len(V), T)
    assert len(np.unique(comp)) == 2
    vox = (DX / 2) ** 3
    for c in np.unique(comp):
        Tc = T[np.isin(T[:, 0], np.nonzero(comp == c)[0])]
        assert S.directed_edges_paired(Tc)
        side = s1[r["anchor"][comp == c][0]] == 1
        nvox = int((sd < 0).sum() if side else (sd >= 0).sum())
        # the cut face passes within half a lattice step of the voxel union's
        assert S.signed_volume(V, Tc) == pytest.approx(nvox * vox, rel=0.02)


def test_embedding_follows_each_side():
    X = box(4, 2, 2)
    origin = (-DX / 2,) * 3
    mid = 2 * DX
    s1, s2 = split_codes(X, 0, mid)
    r = S.reconstruct(X, s1, s2, DX)
    ref = r["ref"]
    # no motion: the surface stays at its reference position
    assert np.allclose(S.embed(r, X, X, s1, s2, DX, origin), ref, atol=1e-15)
    # rigid translation of everything
    t = np.array([1e-3, -2e-3, 5e-4])
    assert np.allclose(S.embed(r, X, X + t, s1, s2, DX, origin), ref + t, atol=1e-15)
    # each side moves with its own translation: the logical grids keep them apart
    t1, t2 = np.array([-3e-3, 0, 1e-3]), np.array([4e-3, 1e-3, 0])
    x = np.where((s1 == 1)[:, None], X + t1, X + t2)
    got = S.embed(r, X, x, s1, s2, DX, origin)
    side1 = s1[r["anchor"]] == 1
    assert np.allclose(got[side1], ref[side1] + t1, atol=1e-15)
    assert np.allclose(got[~side1], ref[~side1] + t2, atol=1e-15)


def test_embedding_single_field_reproduces_linear_motion_inside():
    """Without cuts, nodes whose B-spline support is full reproduce a linear
    displacement exactly (the quadratic B-spline reproduces linear functions),
    so representatives far enough from the boundary move with it; here every
    surface vertex is checked against a brute-force sum instead."""
    X = box(3, 2, 2)
    origin = (-DX / 2,) * 3
    s1, s2 = uncoded(len(X))
    r = S.reconstruct(X, s1, s2, DX)
    rng = np.random.default_rng(2)
    x = X + 1e-3 * rng.normal(size=X.shape)
    got = S.embed(r, X, x, s1, s2, DX, origin)
    for k in rng.choice(len(r["ref"]), 8, replace=False):
        c = r["ref"][k]
        f = (c - origin) / DX
        b = np.floor(f)
        num, den = np.zeros(3), 0.0
        for d in S.CORNERS:
            node = b + d
            wt = np.prod([f[a] - b[a] if d[a] else 1 - (f[a] - b[a]) for a in range(3)])
            Nw = np.array([np.prod([S.bspline((X[p, a] - origin[a]) / DX - node[a]) for a in range(3)])
                           for p in range(len(X))])
            if Nw.sum() > 0:
                num += wt * (Nw @ (x - X)) / Nw.sum()
                den += wt
        assert np.allclose(got[k], c + num / den, atol=1e-15)


def test_lattice_rejects_off_lattice_points():
    X = box(1, 1, 1).copy()
    X[0, 0] += 0.1 * DX
    with pytest.raises(ValueError):
        S.Lattice(X, DX)


def test_surface_of_a_simulated_cut():
    """The oracle's own single-cut run: the recorded plane is the blade's, the
    interior cut-face vertices lie on it, and the surface stays a closed
    chain with the cuboid's volume (the slit encloses none; along its ragged
    tip the two faces may share edges, so manifoldness is not asked)."""
    from oracle import oracle as O

    sc = bi.single_cut_cuboid(n_down=400)
    o = O.OracleScene(sc)
    o.step(400)
    planes, mask = o.cut_planes()
    assert mask == 1
    fr = o.frame()
    assert np.allclose(planes[0, :3], fr["n"]) and planes[0, 3] == pytest.approx(fr["n"] @ fr["xe"], abs=1e-12)
    s1, s2 = S.codes_from_digits(o.get("digits"))
    assert (s1 != 0).sum() > 50 and (s2 != 0).sum() > 50
    X = np.asarray(sc.X)
    r = S.reconstruct(X, s1, s2, sc.dx, planes=planes, plane_mask=mask)
    V, T = r["ref"], r["tris"]
    assert S.closed_chain(T)
    size = X.max(0) - X.min(0) + sc.dx / 2
    assert S.signed_volume(V, T) == pytest.approx(np.prod(size), rel=1e-6)
    # cells whose regions see only cut links place their vertex on the plane
    off = planes[0, :3] @ V.T - planes[0, 3]
    L = r["lattice"]
    interior = np.all((V > L.Xmin + L.h) & (V < L.Xmin + (L.n - 2) * L.h), axis=1)
    cutv = interior & (s1[r["anchor"]] | s2[r["anchor"]]).astype(bool)
    assert cutv.sum() > 20
    assert np.abs(off[cutv]).max() < 1e-9
    x = o.get("x")
    cur = S.embed(r, X, x, s1, s2, sc.dx, sc.origin)
    assert np.isfinite(cur).all() and np.abs(cur - V).max() < 5 * sc.dx


def test_two_intersecting_cuts_give_four_closed_boxes():
    """Two full axis cuts (x and y mid-planes, cuts 0 and 1) split the box into
    four closed quarter boxes; along the line where the cuts cross, each
    quarter keeps its own vertices."""
    X = box(4, 4, 2)
    s1x, s2x = split_codes(X, 0, 4 * DX / 2)
    s1y, s2y = split_codes(X, 1, 4 * DX / 2)
    s1 = (s1x | (s1y << 1)).astype(np.uint32)
    s2 = (s2x | (s2y << 1)).astype(np.uint32)
    pl = np.zeros((32, 4))
    pl[0] = [1, 0, 0, 2 * DX]
    pl[1] = [0, 1, 0, 2 * DX]
    r = S.reconstruct(X, s1, s2, DX, planes=pl, plane_mask=3)
    V, T = r["ref"], r["tris"]
    comp = S.components(len(V), T)
    assert len(np.unique(comp)) == 4
    quarter = 2 * DX * 2 * DX * 2 * DX
    for c in np.unique(comp):
        Tc = T[np.isin(T[:, 0], np.nonzero(comp == c)[0])]
        assert S.directed_edges_paired(Tc)
        assert euler(int((comp == c).sum()), Tc) == 2
        assert S.signed_volume(V, Tc) == pytest.approx(quarter, rel=1e-6)
        # every vertex of a quarter carries that quarter's code
        codes = {(int(s1[a]), int(s2[a])) for a in r["anchor"][comp == c]}
        assert len(codes) == 1
