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
