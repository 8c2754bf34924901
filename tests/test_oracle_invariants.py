"""Whole-substep invariants of the oracle (CPU only).

These pin the oracle's scene loop to what the paper and the mathematics fix:
rest, rigid translation, the momentum proposition of the appendix (Eq. 18),
the 1D bar wave speed, the label invariant after tool withdrawal (Sec. III-D,
Sec. IV-A), closed-form single-contact responses (Eq. 10-15), the reaction
identity (Eq. 16) and the interval-averaged wrench (Sec. III-G).
"""
import math

import numpy as np
import pytest

import bm_inputs as bi
from oracle import oracle as O


def small_block(cells=(4, 4, 4), dx=5e-3, **kw):
    X = bi.lattice_cuboid(tuple(c * dx for c in cells), dx)
    base = dict(X=X, dx=dx, V0=dx ** 3 / 8, gravity=(0.0, 0.0, 0.0), floor=False)
    base.update(kw)
    return bi.Scene(**base)


def test_rest_state_is_exactly_stationary():
    s = O.OracleScene(small_block())
    s.step(5)
    assert np.array_equal(s.get("x"), s.get("X"))
    assert np.all(s.get("v") == 0.0)
    F = s.get("F").reshape(-1, 3, 3)
    assert np.all(F == np.eye(3)[None])


def test_rigid_translation():
    sc = small_block(beta=0.99)
    s = O.OracleScene(sc)
    v0 = np.array([0.3, -0.2, 0.1])
    s.set("v", np.tile(v0, (sc.n, 1)))
    nsteps = 20
    s.step(nsteps)
    x = s.get("x")
    assert np.allclose(x, sc.X + v0[None, :] * sc.dt * nsteps, atol=1e-15, rtol=0)
    assert np.allclose(s.get("v"), v0[None, :], atol=1e-14)
    F = s.get("F").reshape(-1, 3, 3)
    assert np.max(np.abs(F - np.eye(3)[None])) < 1e-13


@pytest.mark.parametrize("beta", [0.0, 0.99, 1.0])
def test_momentum_conserved_random_codes_and_pair_contact(beta):
    """Appendix proposition: coupling + PIC/FLIP + MUSL keep sum m v."""
    sc = small_block(cells=(4, 3, 3), beta=beta, pair_contact=True)
    s = O.OracleScene(sc)
    rng = np.random.default_rng(7)
    digits = np.zeros((sc.n, O.MAX_CUTS))
    digits[:, :2] = rng.integers(0, 3, (sc.n, 2))
    s.set("digits", digits)
    s.set("v", 0.05 * rng.standard_normal((sc.n, 3)))
    F = np.tile(np.eye(3).ravel(), (sc.n, 1)) + 0.01 * rng.standard_normal((sc.n, 9))
    s.set("F", F)
    P0 = s.momentum()
    scale = sc.rho * sc.V0 * 0.05 * sc.n
    had_pairs = False
    for _ in range(10):
        s.step(1)
        had_pairs |= bool(np.any(s.get("J") != 0))
        assert np.max(np.abs(s.momentum() - P0)) < 1e-13 * scale
    assert had_pairs, "the test must exercise pair contact"


def test_momentum_balance_equals_applied_impulses():
    """Eq. 18: P^{n+1} = P^n + sum of gravity, floor and tool impulses."""
    sc = bi.single_cut_cuboid(size=(0.04, 0.02, 0.02), edge_z0=0.0205, speed=0.5, n_down=60)
    s = O.OracleScene(sc)
    m = sc.rho * sc.V0
    for _ in range(30):
        P0 = s.momentum()
        s.step(1)
        dP = s.momentum() - P0
        assert np.max(np.abs(dP - s.impulse_sum())) < 1e-12 * max(1e-9, np.max(np.abs(dP)))
    assert np.any(np.abs(s.wrench_history()) > 0), "blade must have touched the block"


def test_bar_wave_speed():
    """Free-free bar, nu = 0: fundamental period 2L/c with c = sqrt(E/rho)."""
    dx, ncell = 5e-3, 40
    L = ncell * dx
    X = bi.lattice_cuboid((L, dx, dx), dx)
    E, rho = 1e5, 1000.0
    sc = bi.Scene(X=X, E=E, nu=0.0, rho=rho, dx=dx, V0=dx ** 3 / 8, dt=1e-4, beta=0.99,
                  gravity=(0, 0, 0), floor=False)
    s = O.OracleScene(sc)
    v0 = 1e-4
    v = np.zeros((sc.n, 3))
    v[:, 0] = v0 * np.cos(np.pi * X[:, 0] / L)
    s.set("v", v)
    left = X[:, 0] < 0.25 * L
    m_left = []
    for _ in range(700):
        s.step(1)
        m_left.append(s.get("v")[left, 0].mean())
    m_left = np.array(m_left)
    t = (np.arange(len(m_left)) + 1) * sc.dt
    zc = []
    for i in range(len(m_left) - 1):
        if m_left[i] == 0 or (m_left[i] > 0) != (m_left[i + 1] > 0):
            a, b = m_left[i], m_left[i + 1]
            zc.append(t[i] + sc.dt * a / (a - b))
    assert len(zc) >= 3
    period = 2 * np.mean(np.diff(zc))
    expect = 2 * L / math.sqrt(E / rho)
    assert abs(period - expect) / expect < 0.02


def _withdrawal_scene(single_field=False, band=-1.0):
    dx = 5e-3
    X = bi.lattice_cuboid((0.04, 0.02, 0.02), dx)
    n_down = 270
    blade = bi.Blade(pose_x=(0.02, 0.01, 0.022),
                     segments=[bi.Segment(n_down, v=(0, 0, -1.0), cut_id=0),
                               bi.Segment(n_down, v=(0, 0, 1.0), cut_id=0),
                               bi.Segment(10 ** 6, v=(0, 10.0, 0.0), cut_id=-1)])
    sc = bi.Scene(X=X, dx=dx, V0=dx ** 3 / 8, gravity=(0, 0, 0), floor=False,
                  tool_contact=False, band_half_width=band, blade=blade)
    return sc, O.OracleScene(sc, single_field=single_field), 2 * n_down


def test_label_invariant_after_withdrawal():
    """After the blade has swept through and left, opposite sides exchange no
    momentum through any node (Sec. III-D); the single-field baseline does."""
    sc, s, n = _withdrawal_scene()
    s.step(n)
    digits = s.get("digits")[:, 0]
    assert np.all(digits > 0), "band of 6 dx must label the whole block"
    side1 = digits == 1
    assert np.array_equal(side1, sc.X[:, 0] < 0.02)
    v = np.zeros((sc.n, 3))
    v[side1, 0] = -0.1
    s.set("v", v)
    s.step(40)
    vv = s.get("v")
    assert np.all(vv[~side1] == 0.0)
    assert np.all(s.get("x")[~side1] == sc.X[~side1])
    assert np.all(np.abs(vv[side1, 0]) > 0)

    sc2, s2, n2 = _withdrawal_scene(single_field=True)
    s2.step(n2)
    s2.set("v", v)
    s2.step(40)
    assert np.max(np.abs(s2.get("v")[~side1])) > 1e-4, "single field must leak momentum"


def test_narrow_band_leaves_coupling_through_unassigned_material():
    sc, s, n = _withdrawal_scene(band=2.0e-3)
    s.step(n)
    digits = s.get("digits")[:, 0]
    assert np.any(digits == 0)
    side1 = digits == 1
    side2 = digits == 2
    v = np.zeros((sc.n, 3))
    v[side1, 0] = -0.1
    s.set("v", v)
    s.step(40)
    assert np.max(np.abs(s.get("v")[side2])) > 0


def test_digits_are_persistent_and_monotone():
    sc = bi.single_cut_cuboid(size=(0.04, 0.02, 0.02), edge_z0=0.021, speed=1.0, n_down=200)
    s = O.OracleScene(sc)
    prev = s.get("code")
    for _ in range(20):
        s.step(10)
        cur = s.get("code")
        changed = cur != prev
        assert np.all(prev[changed] == 0)
        assert np.all((cur == 0) | (cur == 1) | (cur == 2))
        prev = cur
    assert np.any(prev == 1) and np.any(prev == 2)


def _one_particle(x, v, X=(0.1, 0.1, 0.1), **kw):
    dx = 5e-3
    sc = bi.Scene(X=np.array([X], dtype=np.float64), dx=dx, V0=dx ** 3 / 8, **kw)
    s = O.OracleScene(sc)
    s.set("x", np.array([x]))
    s.set("v", np.array([v]))
    return sc, s


def test_floor_removes_predicted_penetration_in_one_step():
    """Eq. 15 with s_n = 1: the predicted gap is closed exactly in one step."""
    R = 5e-3 / 4
    sc, s = _one_particle((0.1, 0.1, R + 1e-5), (0.0, 0.0, -0.5), gravity=(0, 0, 0))
    s.step(1)
    z = s.get("x")[0, 2]
    assert abs((z - R) - 0.0) < 1e-15
    assert abs(s.get("v")[0, 2] - (-1e-5 / sc.dt)) < 1e-12


def test_two_spheres_head_on_stop_and_conserve_momentum():
    dx = 5e-3
    R = dx / 4
    X = np.array([[0.0125, 0.0125, 0.0125], [0.0125 + 20 * dx, 0.0125, 0.0125]])
    sc = bi.Scene(X=X, dx=dx, V0=dx ** 3 / 8, gravity=(0, 0, 0), floor=False, pair_contact=True)
    s = O.OracleScene(sc)
    u = 0.3
    xp = np.array([0.05, 0.05, 0.05])
    s.set("x", np.stack([xp, xp + np.array([2 * R, 0, 0])]))
    s.set("v", np.array([[u, 0, 0], [-u, 0, 0]]))
    s.step(1)
    v = s.get("v")
    assert np.allclose(v, 0.0, atol=1e-13 * u)
    J = s.get("J")
    m = sc.rho * sc.V0
    assert np.allclose(J[0], [-m * u, 0, 0], rtol=1e-13)
    assert np.array_equal(J[0], -J[1])


@pytest.mark.parametrize("theta_deg,mu,sticks", [(8.0, 0.2, True), (25.0, 0.2, False)])
def test_particle_on_incline(theta_deg, mu, sticks):
    """Coulomb law on a static tilted tool face: stick iff tan(theta) <= mu,
    otherwise slide with a = g (sin(theta) - mu cos(theta))."""
    th = math.radians(theta_deg)
    R = 5e-3 / 4
    nrm = np.array([-math.sin(th), 0.0, math.cos(th)])
    down = np.array([math.cos(th), 0.0, math.sin(th)])
    if down[2] > 0:
        down = -down
    t_e = np.array([0.0, 1.0, 0.0])
    dvec = np.cross(nrm, t_e)
    Rm = np.stack([nrm, t_e, dvec], axis=1)
    half_t = 0.05
    p0 = np.array([0.2, 0.2, 0.2])
    centre = p0 - nrm * (half_t + R)
    blade = bi.Blade(thickness=2 * half_t, half_length=1.0, height=2.0, mu_s=mu, mu_d=mu,
                     pose_x=tuple(centre - dvec * 1.0), pose_R=tuple(Rm.ravel()),
                     segments=[bi.Segment(10 ** 6, cut_id=-1)])
    dx = 5e-3
    sc = bi.Scene(X=np.array([[0.1, 0.1, 0.1]]), dx=dx, V0=dx ** 3 / 8, floor=False,
                  blade=blade, dt=1e-4)
    s = O.OracleScene(sc)
    s.set("x", p0[None, :])
    nsteps = 2000
    s.step(nsteps)
    T = nsteps * sc.dt
    # displacement along the downhill tangent of the face
    downhill = np.array([math.cos(th), 0.0, math.sin(th)])
    downhill = -downhill if downhill[2] > 0 else downhill
    disp = (s.get("x")[0] - p0) @ downhill
    g = 9.81
    if sticks:
        assert abs(disp) < 1e-5
    else:
        a = g * (math.sin(th) - mu * math.cos(th))
        assert abs(disp - 0.5 * a * T * T) / (0.5 * a * T * T) < 0.03


def test_wrench_is_minus_impulse_over_dt_and_interval_average():
    sc = bi.single_cut_cuboid(size=(0.04, 0.02, 0.02), edge_z0=0.0201, speed=0.5, n_down=100)
    sc = sc.replace(floor=False, gravity=(0, 0, 0))
    sc.blade.rigid_interval = 4
    s = O.OracleScene(sc)
    for _ in range(12):
        s.step(1)
        J = s.get("J").sum(0)
        W = s.wrench_history(s.step_count - 1, 1)[0]
        assert np.allclose(W[:3], -J / sc.dt, rtol=1e-12, atol=1e-15)
    hist = s.wrench_history(0, 12)
    assert np.any(hist != 0)
    # the rigid interval returns the mean of its 4 substeps (same net impulse)
    assert np.allclose(s.last_wrench(), hist[8:12].mean(0), rtol=1e-12, atol=1e-18)


def test_two_way_tool_conserves_total_momentum():
    """Eq. 16 + two-way coupling: with gravity, floor and servo off, the
    tool's momentum change is exactly minus the material's."""
    X = bi.lattice_cuboid((0.02, 0.02, 0.02), 5e-3)
    blade = bi.Blade(pose_x=(0.01, 0.01, 0.0205), mass=0.01, servo_gain=1e-12,
                     inertia=bi.plate_inertia(0.01, 1e-3, 0.1, 0.1), segments=[])
    sc = bi.Scene(X=X, gravity=(0, 0, 0), floor=False, blade=blade)
    s = O.OracleScene(sc)
    tool = s.tool()
    tool[12:15] = (0.0, 0.0, -0.5)
    s.set_tool(tool[0:3], tool[3:12], tool[12:15], tool[15:18])
    P0 = s.momentum() + blade.mass * s.tool()[12:15]
    for _ in range(40):
        s.step(1)
        P = s.momentum() + blade.mass * s.tool()[12:15]
        assert np.max(np.abs(P - P0)) < 1e-14
    assert np.any(np.abs(s.momentum()) > 1e-6), "tool must have pushed the block"
