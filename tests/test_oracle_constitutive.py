"""CPU pins of the oracle's fixed-corotated model (the paper's elastic model,
Sec. III-B): polar decomposition, stress as the energy derivative, frame
indifference, the small-strain limit, and the bar wave speed."""
import math

import numpy as np

import bm_inputs as bi
from oracle import oracle as O


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def test_polar_recovers_a_constructed_factorisation():
    """F = Q S0 with a rotation Q (unit quaternion) and an SPD S0: the polar
    decomposition returns Q and S0."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        Q = _rotation(rng)
        B = rng.normal(size=(3, 3))
        S0 = B @ B.T + 0.2 * np.eye(3)
        R, S = O.polar(Q @ S0)
        assert np.abs(R - Q).max() < 1e-10
        assert np.abs(S - S0).max() < 1e-10 * np.abs(S0).max()


def test_fixed_corotated_rest_and_rotation_are_stress_free():
    rng = np.random.default_rng(12)
    P, clamped = O.piola_fcr(np.eye(3), 3.0e4, 5.0e4)
    assert not clamped and np.abs(P).max() == 0.0
    for _ in range(5):
        P, _ = O.piola_fcr(_rotation(rng), 3.0e4, 5.0e4)
        assert np.abs(P).max() < 1e-9


def test_fixed_corotated_stress_is_the_energy_derivative():
    rng = np.random.default_rng(13)
    mu, lam = 3.0e4, 5.0e4
    for _ in range(5):
        F = np.eye(3) + 0.25 * rng.normal(size=(3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        P, _ = O.piola_fcr(F, mu, lam)
        h = 1e-6
        fd = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[i, j] += h
                Fm[i, j] -= h
                fd[i, j] = (O.psi_fcr(Fp, mu, lam) - O.psi_fcr(Fm, mu, lam)) / (2 * h)
        assert np.abs(fd - P).max() <= 1e-6 * np.abs(P).max()


def test_fixed_corotated_frame_indifference():
    rng = np.random.default_rng(14)
    for _ in range(5):
        F = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
        Q = _rotation(rng)
        P, _ = O.piola_fcr(F, 2.0e4, 1.0e4)
        PQ, _ = O.piola_fcr(Q @ F, 2.0e4, 1.0e4)
        assert np.abs(PQ - Q @ P).max() <= 1e-9 * np.abs(P).max()


def test_fixed_corotated_small_strain_limit_is_linear_elasticity():
    rng = np.random.default_rng(15)
    mu, lam = 2.5e4, 4.0e4
    H = rng.normal(size=(3, 3))
    eps = 1e-6
    P, _ = O.piola_fcr(np.eye(3) + eps * H, mu, lam)
    lin = mu * (H + H.T) + lam * np.trace(H) * np.eye(3)
    assert np.abs(P / eps - lin).max() <= 1e-4 * np.abs(lin).max()


def test_inverted_element_is_flagged():
    F = np.diag([1.0, 1.0, -0.5])
    assert O.piola_fcr(F, 1.0, 1.0)[1]


def test_fixed_corotated_bar_wave_speed():
    """Free-free bar, nu = 0: fundamental period 2L/c with c = sqrt(E/rho)."""
    dx, ncell = 5e-3, 40
    L = ncell * dx
    X = bi.lattice_cuboid((L, dx, dx), dx)
    E, rho = 1e5, 1000.0
    sc = bi.Scene(X=X, E=E, nu=0.0, rho=rho, dx=dx, V0=dx ** 3 / 8, dt=1e-4, beta=0.99,
                  gravity=(0, 0, 0), floor=False, model="fixed_corotated")
    s = O.OracleScene(sc)
    v = np.zeros((sc.n, 3))
    v[:, 0] = 1e-4 * np.cos(np.pi * X[:, 0] / L)
    s.set("v", v)
    left = X[:, 0] < 0.25 * L
    m_left = []
    for _ in range(700):
        s.step(1)
        m_left.append(s.get("v")[left, 0].mean())
    m_left = np.array(m_left)
    t = (np.arange(len(m_left)) + 1) * sc.dt
    zc = [t[i] + sc.dt * m_left[i] / (m_left[i] - m_left[i + 1]) for i in range(len(m_left) - 1)
          if (m_left[i] > 0) != (m_left[i + 1] > 0)]
    assert len(zc) >= 3
    period = 2 * np.mean(np.diff(zc))
    expect = 2 * L / math.sqrt(E / rho)
    assert abs(period - expect) / expect < 0.02


# ---------------------------------------------------------------------------
# von Mises plasticity projection (radial return in principal Hencky strains)
# ---------------------------------------------------------------------------

def _vm_equivalent(Fe, mu):
    """von Mises equivalent of the Hencky deviatoric Kirchhoff stress 2 mu e."""
    s = np.sqrt(np.linalg.eigvalsh(Fe.T @ Fe))
    eps = np.log(s)
    e = eps - eps.mean()
    return math.sqrt(1.5) * 2 * mu * np.linalg.norm(e), e


def test_vonmises_below_yield_is_identity():
    F = np.diag([1.01, 0.995, 1.0])
    out, acted = O.vonmises(F, 1e4, 1e6)
    assert not acted and np.array_equal(out, F)


def test_vonmises_projects_onto_the_yield_surface():
    rng = np.random.default_rng(21)
    mu, sy = 1.0e4, 2.0e3
    for _ in range(10):
        Q = _rotation(rng)
        F = Q @ np.diag(np.exp(rng.normal(scale=0.2, size=3))) @ _rotation(rng)
        q0, e0 = _vm_equivalent(F, mu)
        out, acted = O.vonmises(F, mu, sy)
        assert acted == (q0 > sy)
        if not acted:
            continue
        q1, e1 = _vm_equivalent(out, mu)
        assert abs(q1 - sy) <= 1e-9 * sy                          # on the surface
        assert abs(np.linalg.det(out) - np.linalg.det(F)) <= 1e-12  # isochoric
        assert np.allclose(np.sort(e1), np.sort(e0) * sy / q0, atol=1e-12)  # radial return
        again, _ = O.vonmises(out, mu, sy)
        assert np.abs(again - out).max() <= 1e-12                 # idempotent


def test_vonmises_is_rotation_equivariant():
    rng = np.random.default_rng(22)
    F = np.diag([1.3, 0.9, 0.85])
    Q, W = _rotation(rng), _rotation(rng)
    a, _ = O.vonmises(F, 1e4, 1e3)
    b, _ = O.vonmises(Q @ F @ W, 1e4, 1e3)
    assert np.abs(b - Q @ a @ W).max() <= 1e-12


def test_huge_yield_stress_leaves_the_run_elastic():
    import dataclasses
    sc = bi.single_cut_cuboid(size=(0.02, 0.01, 0.01), edge_z0=0.0102, speed=0.5, n_down=40,
                              dx=2.5e-3)
    a = O.OracleScene(sc)
    b = O.OracleScene(dataclasses.replace(sc, yield_stress=1e30))
    a.step(30)
    b.step(30)
    assert np.array_equal(a.get("x"), b.get("x"))


# ---------------------------------------------------------------------------
# Newtonian viscosity
# ---------------------------------------------------------------------------

def test_viscosity_vanishes_for_rigid_rotation_rates():
    rng = np.random.default_rng(23)
    F = _rotation(rng) @ np.diag([1.1, 0.95, 1.0])
    w = rng.normal(size=3)
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    P = O.viscous_piola(F, W @ F, 3.0)
    assert np.abs(P).max() <= 1e-12


def test_viscosity_simple_shear_closed_form():
    eta, g = 2.5, 0.7
    Fdot = np.zeros((3, 3))
    Fdot[0, 1] = g
    P = O.viscous_piola(np.eye(3), Fdot, eta)
    expect = np.zeros((3, 3))
    expect[0, 1] = expect[1, 0] = eta * g
    assert np.abs(P - expect).max() <= 1e-15


def _bar_decay_rate(eta):
    dx, ncell = 5e-3, 40
    L = ncell * dx
    X = bi.lattice_cuboid((L, dx, dx), dx)
    E, rho = 1e5, 1000.0
    sc = bi.Scene(X=X, E=E, nu=0.0, rho=rho, dx=dx, V0=dx ** 3 / 8, dt=1e-4, beta=1.0,
                  gravity=(0, 0, 0), floor=False, viscosity=eta)
    s = O.OracleScene(sc)
    v = np.zeros((sc.n, 3))
    v[:, 0] = 1e-4 * np.cos(np.pi * X[:, 0] / L)
    s.set("v", v)
    left = X[:, 0] < 0.25 * L
    peaks, prev, rising, t = [], 0.0, None, []
    hist = []
    for _ in range(1200):
        s.step(1)
        hist.append(s.get("v")[left, 0].mean())
    h = np.abs(np.array(hist))
    tt = (np.arange(len(h)) + 1) * sc.dt
    # peak magnitudes of the oscillation (local maxima of |v|)
    idx = [i for i in range(1, len(h) - 1) if h[i] >= h[i - 1] and h[i] > h[i + 1]]
    pk, pt = h[idx], tt[idx]
    slope = np.polyfit(pt, np.log(pk), 1)[0]
    return -slope, math.pi / L, rho


def test_viscous_bar_decays_at_the_kelvin_voigt_rate():
    """rho u_tt = E u_xx + 2 eta u_xxt: the fundamental mode decays as
    exp(-eta k^2 t / rho), k = pi / L (beyond the transfer's own damping)."""
    eta = 20.0
    r1, k, rho = _bar_decay_rate(eta)
    r0, _, _ = _bar_decay_rate(0.0)
    expect = eta * k * k / rho
    assert abs((r1 - r0) - expect) <= 0.15 * expect, (r1, r0, expect)
