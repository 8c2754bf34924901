"""Pins of the oracle's building blocks against closed forms and textbook
results (CPU only).  Each test names the passage of the paper it pins."""
import itertools
import os
import math

import numpy as np
import pytest

from oracle import oracle as O


# --------------------------------------------------------------------------
# Eq. 1: quadratic B-spline on the reference grid
# --------------------------------------------------------------------------

def test_bspline_partition_and_completeness():
    rng = np.random.default_rng(0)
    for xl in rng.uniform(-3.0, 40.0, 500):
        b, w, dw = O.bspline(xl)
        nodes = b + np.arange(3)
        # partition of unity and zero-sum gradient
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs(dw.sum()) < 1e-14
        # linear completeness: sum_i N_i x_i = X and sum_i x_i dN_i = 1
        assert abs((w * nodes).sum() - xl) < 1e-12
        assert abs((dw * nodes).sum() - 1.0) < 1e-12
        # derivative consistent with the weights (central differences)
        h = 1e-6
        _, wp, _ = O.bspline(xl + h)
        _, wm, _ = O.bspline(xl - h)
        if O.bspline(xl + h)[0] == b and O.bspline(xl - h)[0] == b:
            assert np.allclose((wp - wm) / (2 * h), dw, atol=1e-8)
        # the base node is the one floor(X - 1/2): all weights positive inside
        assert b == math.floor(xl - 0.5)
        assert np.all(w >= 0)


def test_bspline_textbook_values():
    # particle exactly on a node: weights 1/8, 3/4, 1/8 (textbook quadratic B-spline)
    b, w, dw = O.bspline(5.0)
    assert b == 4
    assert np.allclose(w, [0.125, 0.75, 0.125], atol=0, rtol=0)
    assert np.allclose(dw, [-0.5, 0.0, 0.5])


# --------------------------------------------------------------------------
# stress (neo-Hookean, the workloads' constitutive model)
# --------------------------------------------------------------------------

def lame(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


def test_piola_zero_at_rest():
    P, clamped = O.piola(np.eye(3), *lame(1e5, 0.3))
    assert not clamped
    assert np.all(P == 0.0)


def test_piola_is_energy_gradient():
    mu, lam = lame(1e5, 0.3)
    rng = np.random.default_rng(1)
    for _ in range(20):
        F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        P, _ = O.piola(F, mu, lam)
        G = np.zeros((3, 3))
        h = 1e-6
        for i in range(3):
            for j in range(3):
                Fp = F.copy(); Fp[i, j] += h
                Fm = F.copy(); Fm[i, j] -= h
                G[i, j] = (O.psi(Fp, mu, lam) - O.psi(Fm, mu, lam)) / (2 * h)
        assert np.max(np.abs(G - P)) <= 1e-6 * max(1.0, np.max(np.abs(P)))


def test_piola_small_strain_is_linear_elasticity():
    mu, lam = lame(2e5, 0.35)
    rng = np.random.default_rng(2)
    H = 1e-7 * rng.standard_normal((3, 3))
    P, _ = O.piola(np.eye(3) + H, mu, lam)
    eps = 0.5 * (H + H.T)
    sigma = lam * np.trace(eps) * np.eye(3) + 2 * mu * eps
    assert np.max(np.abs(P - sigma)) < 1e-6 * np.max(np.abs(sigma))


def test_piola_frame_indifference():
    mu, lam = lame(1e5, 0.3)
    rng = np.random.default_rng(3)
    F = np.eye(3) + 0.1 * rng.standard_normal((3, 3))
    A = rng.standard_normal((3, 3))
    Q, _ = np.linalg.qr(A)
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    P1, _ = O.piola(Q @ F, mu, lam)
    P0, _ = O.piola(F, mu, lam)
    assert np.allclose(P1, Q @ P0, rtol=1e-10, atol=1e-8)


def test_piola_inverted_is_clamped_and_flagged():
    F = np.diag([1.0, 1.0, -0.5])
    P, clamped = O.piola(F, *lame(1e5, 0.3))
    assert clamped and np.all(np.isfinite(P))


# --------------------------------------------------------------------------
# Eq. 7 and the conflict predicate (Sec. III-D)
# --------------------------------------------------------------------------

def test_ternary_code_digits_bijection():
    for K in range(1, 5):
        seen = set()
        for digits in itertools.product(range(3), repeat=K):
            c = O.code(list(digits))
            assert c == sum(d * 3 ** k for k, d in enumerate(digits))
            assert [O.digit(c, k) for k in range(K)] == list(digits)
            seen.add(c)
        assert len(seen) == 3 ** K


def _masks(digits):
    s1 = sum(1 << k for k, d in enumerate(digits) if d == 1)
    s2 = sum(1 << k for k, d in enumerate(digits) if d == 2)
    return s1, s2


def test_conflict_matches_bitmask_form_exhaustively():
    """conflict(a,b) <=> (s1a & s2b) | (s2a & s1b) != 0 for every code pair, K <= 4."""
    for K in range(1, 5):
        allc = list(itertools.product(range(3), repeat=K))
        for da in allc:
            a = O.code(list(da))
            s1a, s2a = _masks(da)
            for db in allc:
                b = O.code(list(db))
                s1b, s2b = _masks(db)
                expect = ((s1a & s2b) | (s2a & s1b)) != 0
                assert O.conflict(a, b) == expect
    # unassigned (0) is compatible with both sides; 1 and 2 conflict
    assert not O.conflict(0, 1) and not O.conflict(0, 2) and O.conflict(1, 2)


def test_conflict_matches_hand_written_two_cut_table():
    """The oracle's conflict predicate against the 9 x 9 table of the
    two-cut codes written out by hand from Sec. III-D (tests/golden)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "eq7_conflict_k2.txt")
    rows = [l.strip() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 9 and all(len(r) == 9 for r in rows)
    for a in range(9):
        for b in range(9):
            assert O.conflict(a, b) == (rows[a][b] == "1"), (a, b)


# --------------------------------------------------------------------------
# Eq. 8: compatible coupling
# --------------------------------------------------------------------------

def test_coupling_all_compatible_is_single_field():
    rng = np.random.default_rng(4)
    codes = [0, 1, 3, 9 + 1]  # pairwise compatible: no digit pair (1,2)
    for a in codes:
        for b in codes:
            assert not O.conflict(a, b)
    m = rng.uniform(0.1, 2.0, 4)
    S = rng.standard_normal((4, 6))
    Sb = O.couple(codes, m, S)
    M = m.sum()
    expect = m[:, None] * S.sum(0)[None, :] / M
    assert np.allclose(Sb, expect, rtol=1e-13, atol=1e-15)


def test_coupling_all_conflicting_is_identity():
    codes = [1, 2]
    m = np.array([0.7, 1.3])
    S = np.array([[1.0, 2, 3, 4, 5, 6], [-1.0, 0.5, 2, -3, 1, 0]])
    assert np.array_equal(O.couple(codes, m, S), S)


def test_coupling_three_grids_hand_computed():
    # codes 0 (uncut), 1 and 2 (opposite sides): 0 couples to both, 1-2 do not
    codes = [0, 1, 2]
    m = np.array([1.0, 2.0, 3.0])
    S = np.array([[1.0], [4.0], [-2.0]])
    Sb = O.couple(codes, m, S)
    M = 6.0
    s0 = 1.0 + ((1.0 * 4.0 - 2.0 * 1.0) + (1.0 * -2.0 - 3.0 * 1.0)) / M
    s1 = 4.0 + (2.0 * 1.0 - 1.0 * 4.0) / M
    s2 = -2.0 + (3.0 * 1.0 - 1.0 * -2.0) / M
    assert np.allclose(Sb[:, 0], [s0, s1, s2], rtol=1e-15)


def test_coupling_conserves_sum_and_common_velocity():
    rng = np.random.default_rng(5)
    for _ in range(50):
        ns = rng.integers(1, 7)
        codes = [O.code(list(rng.integers(0, 3, 3))) for _ in range(ns)]
        codes = list(dict.fromkeys(codes))
        ns = len(codes)
        m = rng.uniform(0.01, 1.0, ns)
        S = rng.standard_normal((ns, 6))
        Sb = O.couple(codes, m, S)
        assert np.allclose(Sb.sum(0), S.sum(0), rtol=1e-12, atol=1e-12)
        # a common velocity u: S^a = m^a u is a fixed point
        u = rng.standard_normal(6)
        Su = m[:, None] * u[None, :]
        assert np.allclose(O.couple(codes, m, Su), Su, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------------------
# Eq. 12: friction with tangential spring history
# --------------------------------------------------------------------------

def test_friction_stick_and_slip_closed_form():
    n = np.array([0.0, 0.0, 1.0])
    dt, meff, gk, gc = 1e-4, 1e-3, 0.5, 0.5
    kt = gk * meff / dt ** 2
    ct = 2 * gc * math.sqrt(meff * kt)
    # stick: small tangential velocity, generous normal force
    vrel = np.array([1e-4, 0.0, -0.3])
    fn = 10.0
    ft, un = O.friction(np.zeros(3), n, vrel, fn, meff, dt, gk, gc, 0.5, 0.5)
    assert np.allclose(ft, [-ct * 1e-4, 0, 0])
    assert np.allclose(un, [dt * 1e-4, 0, 0])
    # slip: the force sits on the dynamic Coulomb bound, opposite to the trial
    vrel = np.array([3.0, 4.0, 0.0])
    fn = 1e-3
    ft, un = O.friction(np.zeros(3), n, vrel, fn, meff, dt, gk, gc, 0.2, 0.1)
    assert abs(np.linalg.norm(ft) - 0.1 * fn) < 1e-15
    assert np.allclose(ft / np.linalg.norm(ft), [-0.6, -0.8, 0.0])
    assert np.allclose(-kt * un - ct * np.array([3.0, 4.0, 0.0]), ft, rtol=1e-12)


def test_friction_history_transport_keeps_length():
    n = np.array([0.0, 0.0, 1.0])
    u = np.array([3e-6, 0.0, 4e-6])   # has a normal component: projected and rescaled
    ft, un = O.friction(u, n, np.zeros(3), 1e6, 1e-3, 1e-4, 0.5, 0.5, 0.5, 0.5)
    assert abs(np.linalg.norm(un) - 5e-6) < 1e-18
    assert abs(un[2]) == 0.0


# --------------------------------------------------------------------------
# blade box geometry (Eq. 14 closest point)
# --------------------------------------------------------------------------

def test_box_closest_point_cases():
    c = np.zeros(3)
    ax = np.eye(3)
    hext = np.array([0.5e-3, 0.05, 0.05])
    R = 1e-3
    # outside, straight over the +n face
    xc, nB, phi = O.box_closest(c, ax[0], ax[1], ax[2], hext, [0.01, 0.0, 0.0], R)
    assert np.allclose(xc, [0.5e-3, 0, 0]) and np.allclose(nB, [1, 0, 0])
    assert abs(phi - (0.01 - 0.5e-3 - R)) < 1e-15
    # outside, near the edge: closest point is on the edge line
    xc, nB, phi = O.box_closest(c, ax[0], ax[1], ax[2], hext, [0.5e-3 + 3e-3, 0.0, 0.05 + 4e-3], R)
    assert np.allclose(xc, [0.5e-3, 0, 0.05]) and np.allclose(nB, [0.6, 0, 0.8])
    assert abs(phi - (5e-3 - R)) < 1e-15
    # inside: nearest face is the thin side
    xc, nB, phi = O.box_closest(c, ax[0], ax[1], ax[2], hext, [-0.2e-3, 0.0, 0.0], R)
    assert np.allclose(nB, [-1, 0, 0]) and abs(phi - (-(0.3e-3) - R)) < 1e-15


# --------------------------------------------------------------------------
# Eq. 3, 4, 6: side labels (hand-computed tiny cases)
# --------------------------------------------------------------------------

def _lbl(x, v=(0, 0, 0), ve=(0, 0, -0.2), dt=1e-4):
    xe = (0.05, 0.025, 0.03)
    n, e, d = (1, 0, 0), (0, 1, 0), (0, 0, -1)
    return O.side_label(x, v, xe, n, e, d, ve, h=0.03, L=0.05, b_back=0.005, b_lead=0.005, dt=dt)


def test_side_label_hand_cases():
    # behind the edge (above it: f = -(z - z_e) <= 0), inside the band
    assert _lbl((0.049, 0.02, 0.032)) == 1          # s < 0 -> 1
    assert _lbl((0.051, 0.02, 0.032)) == 2          # s > 0 -> 2
    assert _lbl((0.05, 0.02, 0.032)) == 2           # s = 0 -> 2 (s >= 0)
    assert _lbl((0.05, 0.02, 0.030)) == 2           # f = 0 is behind (f <= 0)
    assert _lbl((0.049, 0.02, 0.029)) == 0          # in front: f > 0
    assert _lbl((0.05 + 0.031, 0.02, 0.032)) == 0   # |s| > h
    assert _lbl((0.05 + 0.030, 0.02, 0.032)) == 2   # |s| = h is inside (inclusive)
    assert _lbl((0.049, 0.025 + 0.051, 0.032)) == 0  # |l| > L
    assert _lbl((0.049, 0.02, 0.03 + 0.0051)) == 0  # f < -b_back (u_c dt = 2e-5)
    # the swept distance u_c dt widens the rear extent
    assert _lbl((0.049, 0.02, 0.03 + 0.005 + 1.5e-5)) == 1
    assert _lbl((0.049, 0.02, 0.03 + 0.005 + 1.5e-5), ve=(0, 0, 0)) == 0


# --------------------------------------------------------------------------
# Eq. 5: cutting progress
# --------------------------------------------------------------------------

def test_cut_progress_reaches_one_after_closed_form_count():
    rng = np.random.default_rng(6)
    for _ in range(50):
        Wth = rng.uniform(1e-6, 1e-4)
        Jc = rng.uniform(1e-7, 1e-5)
        uc = rng.uniform(0.01, 1.0)
        expect = math.ceil(Wth / (Jc * uc))
        D, k = 0.0, 0
        while D < 1.0:
            D = O.cut_progress(D, Jc, uc, Wth)
            k += 1
            assert k < 10 ** 6
        # rounding can move an exact multiple by one contact
        assert abs(k - expect) <= 1
        assert D == 1.0
