"""FP64 oracle of the reference-grid surface reconstruction (Sec. III-F).

TEST INFRASTRUCTURE ONLY: imported by the test suite, never by the GPU
library.  Plain numpy and Python loops over the surface cells, written from
the method's description, in its order:

  1. Surface grid.  The uniform reference grid is the particles' own
     sub-cell lattice (spacing h_a = dx / k_a with k_a particles per cell
     along axis a); a lattice vertex is material when a particle sits on it.
     The original boundary is the boundary of the union of the material
     vertices' voxels (side h_a, centred on the vertex).
  2. Links and Hermite data.  Every pair of lattice neighbours is a link.
     Both ends material with compatible codes: connected.  Both ends
     material with conflicting codes: disconnected by the sweep; its Hermite
     data is the crossing of the lowest conflicting cut's plane (recorded
     when that cut began) with the link, clamped to the link, and the
     plane's normal oriented away from the end's side (the end with digit 1
     lies on the -n side); without a recorded plane, the link midpoint and
     the link direction.  One end material: a boundary link, with the voxel
     face midpoint and the outward axis direction.
  3. Local regions.  In each lattice cell (8 vertices, 12 links) the
     connected components of the material vertices over the connected links
     are the local material regions, ordered by their lowest corner; a region
     carries a surface representative when one of its vertices has a
     disconnected or boundary link among the cell's edges.
  4. Representatives (local dual contouring).  Each active region places one
     vertex at the minimiser of the quadratic error sum_i (n_i . (c - p_i))^2
     over its links' Hermite data, taken relative to the mass point (mean of
     the p_i) with the pseudo-inverse (eigenvalues below QEF_CUT dropped),
     then clamped to the cell.  A region on both sides of a cut gives two
     coincident faces because each side keeps its own representatives.
  5. Faces.  Every (Hermite link, material end) pair gives a quad over the
     representatives of that end's region in the four cells around the link,
     wound so that its normal points away from the end; each quad is split
     into (r0, r1, r2) and (r0, r2, r3), and triangles with a repeated vertex
     are dropped.
  6. Side-aware embedding.  A representative carries the code of its
     region's lowest corner particle (its anchor) and is embedded with fixed
     trilinear weights over the 8 reference-grid nodes around it, in the
     motion field of that code's logical grid: node displacement
     u_i = sum_p N_ip (x_p - X_p) / sum_p N_ip over particles with exactly
     that code (uniform particle mass cancels), current position
     X_r + sum_i t_i u_i / sum_i t_i over the nodes with such particles.

Ordering (so that the GPU output can be compared index by index): cells by
lower-corner lattice index (x fastest) over [-1, n_a - 1]; representatives
by cell, then region; links by their lower end's lattice index, then axis
x, y, z; quads by link, lower end first.
"""
from __future__ import annotations

import numpy as np

QEF_CUT = 0.1  # eigenvalues of sum n n^T below this are treated as zero (unit normals)

# cell corners q = qx + 2 qy + 4 qz and the 12 cell edges (q0, q1, axis)
CORNERS = [(q & 1, (q >> 1) & 1, (q >> 2) & 1) for q in range(8)]
EDGES = []
for _q in range(8):
    for _a in range(3):
        if not (_q >> _a) & 1:
            EDGES.append((_q, _q | (1 << _a), _a))


def bspline(t: float) -> float:
    """Quadratic B-spline N(t) (the TLMPM shape function of Eq. 1)."""
    t = abs(t)
    if t < 0.5:
        return 0.75 - t * t
    if t < 1.5:
        return 0.5 * (1.5 - t) ** 2
    return 0.0


class Lattice:
    """Sub-cell lattice of a scene's reference positions."""

    def __init__(self, X: np.ndarray, dx: float, per_axis=(2, 2, 2)):
        X = np.asarray(X, np.float64)
        self.h = np.array([dx / k for k in per_axis])
        self.Xmin = X.min(axis=0)
        j = np.rint((X - self.Xmin) / self.h).astype(np.int64)
        if np.abs(self.Xmin + j * self.h - X).max() > 1e-3 * self.h.min():
            raise ValueError("particles are not on the sub-cell lattice")
        self.n = j.max(axis=0) + 1
        self.j = j
        if len(np.unique(j[:, 0] + self.n[0] * (j[:, 1] + self.n[1] * j[:, 2]))) != len(X):
            raise ValueError("lattice point holds two particles")
        self.index = -np.ones(tuple(self.n[::-1]), np.int64)  # [z, y, x] -> particle
        self.index[j[:, 2], j[:, 1], j[:, 0]] = np.arange(len(X))

    def particle(self, jx: int, jy: int, jz: int) -> int:
        if 0 <= jx < self.n[0] and 0 <= jy < self.n[1] and 0 <= jz < self.n[2]:
            return int(self.index[jz, jy, jx])
        return -1

    def pos(self, j) -> np.ndarray:
        return self.Xmin + np.asarray(j, np.float64) * self.h


def conflict_bits(a1, a2, b1, b2) -> int:
    """Digits on which two codes (s1, s2 masks) disagree, both nonzero."""
    return (int(a1) & int(b2)) | (int(a2) & int(b1))


def link_hermite(L: Lattice, s1, s2, planes, plane_mask, ja, jb, pa: int, pb: int):
    """Hermite data of the link ja -> jb as seen from end a (material):
    (point, outward normal) or None when the link is connected or a is empty."""
    Xa, Xb = L.pos(ja), L.pos(jb)
    if pa < 0:
        return None
    if pb < 0:  # boundary link: voxel face midpoint, outward axis direction
        d = Xb - Xa
        return 0.5 * (Xa + Xb), d / np.linalg.norm(d)
    c = conflict_bits(s1[pa], s2[pa], s1[pb], s2[pb])
    if c == 0:
        return None
    k = (c & -c).bit_length() - 1  # lowest conflicting cut
    d = Xb - Xa
    if (plane_mask >> k) & 1:
        n = np.asarray(planes[k][:3], np.float64)
        off = float(planes[k][3])
        den = float(n @ d)
        t = 0.5
        if abs(den) > 1e-6 * np.linalg.norm(d):
            t = min(max((off - float(n @ Xa)) / den, 0.0), 1.0)
        nout = n if (int(s1[pa]) >> k) & 1 else -n  # digit 1 lies on the -n side
        return Xa + t * d, nout
    return 0.5 * (Xa + Xb), d / np.linalg.norm(d)


def qef_point(points, normals) -> np.ndarray:
    """Minimiser of sum (n_i . (c - p_i))^2 relative to the mass point, with the
    pseudo-inverse of sum n n^T (eigenvalues below QEF_CUT dropped)."""
    P = np.asarray(points, np.float64)
    N = np.asarray(normals, np.float64)
    m = P.mean(axis=0)
    A = N.T @ N
    r = N.T @ np.einsum("ij,ij->i", N, P - m)
    lam, V = np.linalg.eigh(A)
    delta = np.zeros(3)
    for i in range(3):
        if lam[i] >= QEF_CUT:
            delta += (V[:, i] @ r) / lam[i] * V[:, i]
    return m + delta


def cell_regions(L: Lattice, s1, s2, jl):
    """Corner particles, region id per corner (-1 empty) and region count of
    the cell with lower corner jl; regions numbered by lowest corner."""
    parts = [L.particle(jl[0] + c[0], jl[1] + c[1], jl[2] + c[2]) for c in CORNERS]
    parent = list(range(8))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a

    for q0, q1, _ in EDGES:
        p0, p1 = parts[q0], parts[q1]
        if p0 >= 0 and p1 >= 0 and conflict_bits(s1[p0], s2[p0], s1[p1], s2[p1]) == 0:
            r0, r1 = find(q0), find(q1)
            if r0 != r1:
                parent[max(r0, r1)] = min(r0, r1)
    reg = [-1] * 8
    roots = {}
    for q in range(8):
        if parts[q] >= 0:
            r = find(q)
            if r not in roots:
                roots[r] = len(roots)
            reg[q] = roots[r]
    return parts, reg, len(roots)


def reconstruct(X, s1, s2, dx: float, per_axis=(2, 2, 2), planes=None, plane_mask: int = 0,
                cells=None):
    """Topology and reference positions of the surface.

    Returns a dict: ``ref`` (V, 3) representative reference positions,
    ``anchor`` (V,) anchor particle, ``cell`` (V,) cell linear index,
    ``tris`` (T, 3) triangles, ``lattice`` the Lattice.  With ``cells`` (a
    set of cell linear indices) only those cells' representatives are
    computed (``ref`` rows of other cells are NaN, ``tris`` is empty)."""
    L = Lattice(X, dx, per_axis)
    s1 = np.asarray(s1, np.uint32)
    s2 = np.asarray(s2, np.uint32)
    if planes is None:
        planes = np.zeros((32, 4))
    nc = L.n + 1  # cells per axis, lower corners -1 .. n - 1

    # material count per cell, to skip cells that are fully empty or fully
    # material with no disconnected link (they carry no representative)
    occ = np.zeros(tuple(L.n[::-1] + 2), np.int8)
    occ[1:-1, 1:-1, 1:-1] = L.index >= 0
    tot = np.zeros(tuple(nc[::-1]), np.int64)
    for c in CORNERS:
        tot += occ[c[2]:c[2] + nc[2], c[1]:c[1] + nc[1], c[0]:c[0] + nc[0]]
    labelled = np.zeros(tuple(L.n[::-1] + 2), np.int8)
    lab = (s1 | s2) != 0
    labelled[L.j[:, 2] + 1, L.j[:, 1] + 1, L.j[:, 0] + 1] = lab
    anylab = np.zeros(tuple(nc[::-1]), np.int64)
    for c in CORNERS:
        anylab += labelled[c[2]:c[2] + nc[2], c[1]:c[1] + nc[1], c[0]:c[0] + nc[0]]
    cand = np.nonzero(((tot > 0) & (tot < 8)) | ((tot == 8) & (anylab > 0)))
    cand_lin = np.sort((cand[0] * nc[1] + cand[1]) * nc[0] + cand[2])

    rep_base = {}  # cell linear index -> (first rep, regions, reg list)
    ref, anchor, cell_of = [], [], []
    for lin in cand_lin:
        lin = int(lin)
        cx = lin % nc[0] - 1
        cy = (lin // nc[0]) % nc[1] - 1
        cz = lin // (nc[0] * nc[1]) - 1
        jl = (cx, cy, cz)
        parts, reg, nreg = cell_regions(L, s1, s2, jl)
        herm = [[] for _ in range(nreg)]
        for q0, q1, _ in EDGES:
            j0 = [jl[a] + CORNERS[q0][a] for a in range(3)]
            j1 = [jl[a] + CORNERS[q1][a] for a in range(3)]
            for qa, qb, ja, jb in ((q0, q1, j0, j1), (q1, q0, j1, j0)):
                hd = link_hermite(L, s1, s2, planes, plane_mask, ja, jb, parts[qa], parts[qb])
                if hd is not None:
                    herm[reg[qa]].append(hd)
        first = len(ref)
        ords = [-1] * nreg
        for r in range(nreg):
            if not herm[r]:
                continue
            ords[r] = len(ref) - first
            compute = cells is None or lin in cells
            if compute:
                c = qef_point([h[0] for h in herm[r]], [h[1] for h in herm[r]])
                lo = L.pos(jl)
                c = np.minimum(np.maximum(c, lo), lo + L.h)
            else:
                c = np.full(3, np.nan)
            q_anchor = min(q for q in range(8) if reg[q] == r)
            ref.append(c)
            anchor.append(parts[q_anchor])
            cell_of.append(lin)
        if len(ref) > first:
            rep_base[lin] = (first, [ords[r] if r >= 0 else -1 for r in reg])

    tris = []
    if cells is None:
        # a link with Hermite data is an edge of four cells that all carry a
        # representative, among them the cell whose lower corner is the link's
        # lower end: walking those cells in order walks the links in order
        for lin in sorted(rep_base):
            j = (lin % nc[0] - 1, (lin // nc[0]) % nc[1] - 1, lin // (nc[0] * nc[1]) - 1)
            for a in range(3):
                b, c = (a + 1) % 3, (a + 2) % 3
                if not (0 <= j[b] < L.n[b] and 0 <= j[c] < L.n[c]):
                    continue
                j1 = list(j)
                j1[a] += 1
                pa, pb = L.particle(*j), L.particle(*j1)
                for side, (pe, po, je, jo) in enumerate(((pa, pb, j, j1), (pb, pa, j1, j))):
                    if link_hermite(L, s1, s2, planes, plane_mask, je, jo, pe, po) is None:
                        continue
                    # cells around the link, counter-clockwise about +axis a
                    # (reversed for the upper end, whose outward side is -a)
                    order = [(0, 0), (1, 0), (1, 1), (0, 1)] if side == 0 else \
                        [(0, 0), (0, 1), (1, 1), (1, 0)]
                    rs = []
                    for sb, sc_ in order:
                        low = list(j)
                        low[b] -= sb
                        low[c] -= sc_
                        cl = ((low[2] + 1) * nc[1] + (low[1] + 1)) * nc[0] + (low[0] + 1)
                        q = sum((je[t] - low[t]) << t for t in range(3))
                        first, ordl = rep_base[cl]
                        rs.append(first + ordl[q])
                    for t in ((rs[0], rs[1], rs[2]), (rs[0], rs[2], rs[3])):
                        if len(set(t)) == 3:
                            tris.append(t)
    return {"ref": np.array(ref, np.float64).reshape(-1, 3), "anchor": np.array(anchor, np.int64),
            "cell": np.array(cell_of, np.int64), "tris": np.array(tris, np.int64).reshape(-1, 3),
            "lattice": L}


def node_fields(X, x, s1, s2, dx: float, origin):
    """Displacement field of every (node, code) logical grid: dict
    (ix, iy, iz, s1, s2) -> (sum N, sum N (x - X)) over particles with that code."""
    X = np.asarray(X, np.float64)
    u = np.asarray(x, np.float64) - X
    f = (X - np.asarray(origin, np.float64)) / dx
    base = np.floor(f - 0.5).astype(np.int64)
    acc = {}
    for p in range(len(X)):
        w = [[bspline(f[p, a] - (base[p, a] + o)) for o in range(3)] for a in range(3)]
        for oz in range(3):
            for oy in range(3):
                for ox in range(3):
                    N = w[0][ox] * w[1][oy] * w[2][oz]
                    key = (int(base[p, 0] + ox), int(base[p, 1] + oy), int(base[p, 2] + oz),
                           int(s1[p]), int(s2[p]))
                    e = acc.get(key)
                    if e is None:
                        acc[key] = [N, N * u[p]]
                    else:
                        e[0] += N
                        e[1] = e[1] + N * u[p]
    return acc


def embed(surf: dict, X, x, s1, s2, dx: float, origin, fields=None) -> np.ndarray:
    """Current positions of the representatives (side-aware trilinear embedding)."""
    if fields is None:
        fields = node_fields(X, x, s1, s2, dx, origin)
    X = np.asarray(X, np.float64)
    x = np.asarray(x, np.float64)
    origin = np.asarray(origin, np.float64)
    out = np.empty_like(surf["ref"])
    for r in range(len(surf["ref"])):
        c = surf["ref"][r]
        p0 = int(surf["anchor"][r])
        f = (c - origin) / dx
        b = np.floor(f).astype(np.int64)
        t = f - b
        num = np.zeros(3)
        den = 0.0
        for d in CORNERS:
            wt = 1.0
            for a in range(3):
                wt *= t[a] if d[a] else 1.0 - t[a]
            e = fields.get((int(b[0] + d[0]), int(b[1] + d[1]), int(b[2] + d[2]),
                            int(s1[p0]), int(s2[p0])))
            if e is None or e[0] <= 0.0:
                continue
            num += wt * e[1] / e[0]
            den += wt
        out[r] = c + (num / den if den > 0.0 else x[p0] - X[p0])
    return out


def codes_from_digits(digits: np.ndarray):
    """(s1, s2) masks from a particles x cuts array of ternary digits."""
    d = np.asarray(digits).astype(np.int64)
    s1 = np.zeros(len(d), np.uint64)
    s2 = np.zeros(len(d), np.uint64)
    for k in range(d.shape[1]):
        s1 |= (d[:, k] == 1).astype(np.uint64) << np.uint64(k)
        s2 |= (d[:, k] == 2).astype(np.uint64) << np.uint64(k)
    return s1.astype(np.uint32), s2.astype(np.uint32)


# -- mesh properties used by the pins ---------------------------------------

def signed_volume(V: np.ndarray, T: np.ndarray) -> float:
    """Enclosed volume of an oriented closed triangle mesh (divergence theorem)."""
    if len(T) == 0:
        return 0.0
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def directed_edges_paired(T: np.ndarray) -> bool:
    """Every directed edge (u, v) of the mesh appears once and (v, u) once."""
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    s = set(map(tuple, e.tolist()))
    if len(s) != len(e):
        return False
    return all((v, u) in s for u, v in s)


def closed_chain(T: np.ndarray) -> bool:
    """The triangles form a closed oriented chain: every directed edge (u, v)
    occurs as often as (v, u) (where two slit faces meet along a cut's tip
    an edge may carry four triangles)."""
    from collections import Counter

    c = Counter(map(tuple, np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]]).tolist()))
    return all(c[(v, u)] == n for (u, v), n in c.items())


def components(nv: int, T: np.ndarray) -> np.ndarray:
    """Connected component of every vertex through the triangles."""
    parent = np.arange(nv)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for t in T:
        r = [find(int(v)) for v in t]
        m = min(r)
        for q in r:
            parent[q] = m
    return np.array([find(i) for i in range(nv)])
