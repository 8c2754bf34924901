"""Cutting resistance inside the oracle's full substep (Sec. III-A, Eq. 5).

A single particle is held in front of the blade edge: before every substep
its position, velocity and deformation gradient and the blade pose are put
back to the same values, so each substep sees the same contact and only the
cutting progress D carries over.  The closed forms then fix the run:

* the blade's normal impulse is J_n = s_n m_p / dt * (R_p + dt u - delta)
  (Eq. 15 with w_B = 0, the particle delta in front of the edge face and the
  blade advancing at u); friction is zero (no tangential slip), so
  J_c = J_n and u_c = u;
* D grows by J_c u_c / W_th per substep, W_th = G_c (V^0)^(2/3) (1 - zeta) /
  zeta, and reaches 1 at substep ceil(W_th / (J_c u_c));
* until then the reaction on the blade along d is -J_c / dt (Eq. 16); on the
  substep after D = 1 the d component is released and the reaction is 0;
* a new cut id resets D to 0;
* contact behind the edge (f < 0) or with u_c <= u_min never accumulates.

None of these numbers is read from the oracle: they come from the scene
parameters and the paper's formulas, written out below.
"""
import math

import numpy as np

import bm_inputs as bi
from oracle import oracle as O

DX = 5e-3
V0 = DX ** 3 / 8
RHO = 1000.0
DT = 1e-4
X0 = np.array([0.0125, 0.0125, 0.0125])


def _scene(pose_x, segments, G_c=150.0):
    blade = bi.Blade(pose_x=tuple(pose_x), segments=segments)
    return bi.Scene(X=X0[None, :].copy(), dx=DX, V0=V0, rho=RHO, dt=DT, gravity=(0.0, 0.0, 0.0),
                    floor=False, G_c=G_c, blade=blade)


def _held_run(sc, n_steps):
    """Steps the scene n_steps times, restoring particle and blade pose before
    each substep; returns D and the blade reaction after every substep."""
    o = O.OracleScene(sc)
    tool0 = o.tool()
    Ds, W = [], []
    for _ in range(n_steps):
        o.set("x", sc.X)
        o.set("v", np.zeros((1, 3)))
        o.set("F", np.eye(3).reshape(1, 9))
        o.set("ut", np.zeros((1, 3)))
        o.set_tool(tool0[0:3], tool0[3:12], tool0[12:15], tool0[15:18])
        o.step(1)
        Ds.append(float(o.get("D")[0]))
        W.append(o.last_wrench().copy())
    return np.array(Ds), np.array(W)


def _closed_form(G_c, delta, speed):
    mp = RHO * V0
    Rp = V0 ** (1.0 / 3.0) / 2.0           # R_p = s_R (V^0)^(1/3) / 2, s_R = 1
    Jc = 1.0 * mp / DT * (Rp + DT * speed - delta)
    Wth = G_c * V0 ** (2.0 / 3.0) * (1.0 - 0.9) / 0.9
    return Jc, speed, Wth


def test_front_band_progress_count_and_release():
    delta, speed, G_c = 1.0e-3, 0.2, 150.0
    # particle at x_e + delta d with d = -z: the edge sits delta above it
    sc = _scene(X0 + np.array([0.0, 0.0, delta]),
                [bi.Segment(100, v=(0.0, 0.0, -speed), cut_id=0)], G_c=G_c)
    Jc, uc, Wth = _closed_form(G_c, delta, speed)
    K = math.ceil(Wth / (Jc * uc))
    assert 5 < K < 50 and Wth / (Jc * uc) % 1.0 > 0.05  # not near an integer
    D, W = _held_run(sc, K + 3)
    # D after k substeps: min(k J_c u_c / W_th, 1), reached at substep K exactly
    for k in range(1, K + 4):
        expect = min(k * Jc * uc / Wth, 1.0)
        assert abs(D[k - 1] - expect) <= 1e-12, (k, D[k - 1], expect)
    assert D[K - 2] < 1.0 and D[K - 1] == 1.0
    # reaction along d (= -z): -J_c/dt while D^n < 1 (substeps 1..K), 0 after
    Fd = -W[:, 2]
    for k in range(1, K + 1):
        assert abs(Fd[k - 1] - (-Jc / DT)) <= 1e-10 * Jc / DT, (k, Fd[k - 1])
    for k in range(K + 1, K + 4):
        assert abs(Fd[k - 1]) <= 1e-10 * Jc / DT, (k, Fd[k - 1])
    # the released component is along d only: no tangential reaction appears
    assert np.all(np.abs(W[:, :2]) <= 1e-10 * Jc / DT)


def test_new_cut_id_resets_progress():
    delta, speed, G_c = 1.0e-3, 0.2, 150.0
    n1 = 4
    sc = _scene(X0 + np.array([0.0, 0.0, delta]),
                [bi.Segment(n1, v=(0.0, 0.0, -speed), cut_id=0),
                 bi.Segment(10, v=(0.0, 0.0, -speed), cut_id=1)], G_c=G_c)
    Jc, uc, Wth = _closed_form(G_c, delta, speed)
    D, W = _held_run(sc, n1 + 3)
    inc = Jc * uc / Wth
    assert abs(D[n1 - 1] - n1 * inc) <= 1e-12
    # first substep of cut 1: D was reset to 0, then one increment
    for j in range(3):
        assert abs(D[n1 + j] - (j + 1) * inc) <= 1e-12, (j, D[n1 + j])
        assert abs(-W[n1 + j, 2] - (-Jc / DT)) <= 1e-10 * Jc / DT


def test_same_cut_id_continues_progress():
    # a second segment with the same cut id is the same cut: no reset
    delta, speed, G_c = 1.0e-3, 0.2, 150.0
    sc = _scene(X0 + np.array([0.0, 0.0, delta]),
                [bi.Segment(3, v=(0.0, 0.0, -speed), cut_id=0),
                 bi.Segment(10, v=(0.0, 0.0, -speed), cut_id=0)], G_c=G_c)
    Jc, uc, Wth = _closed_form(G_c, delta, speed)
    D, _ = _held_run(sc, 6)
    for k in range(1, 7):
        assert abs(D[k - 1] - k * Jc * uc / Wth) <= 1e-12


def test_contact_behind_the_edge_never_accumulates():
    # particle pressed against the blade's side face, 2 mm behind the edge
    # (f = -2 mm < 0): tool contact is active but outside the front band
    half_thick = 0.5e-3
    Rp = V0 ** (1.0 / 3.0) / 2.0
    a = half_thick + Rp - 1e-4
    b = 2e-3
    # x = x_e + a n - b d with n = +x, d = -z  =>  x_e = x - a n + b d
    xe = X0 - np.array([a, 0.0, 0.0]) + np.array([0.0, 0.0, -b])
    sc = _scene(xe, [bi.Segment(100, v=(0.0, 0.0, -0.2), cut_id=0)])
    D, W = _held_run(sc, 20)
    assert np.all(D == 0.0)
    assert np.all(W[:, 0] < 0.0)  # the side face pushes the particle along +n


def test_slow_advance_never_accumulates():
    # u_c = u_min exactly (strict inequality) and u_c below it, contact active
    delta = 1.0e-3
    for speed in (1e-3, 5e-4):
        sc = _scene(X0 + np.array([0.0, 0.0, delta]),
                    [bi.Segment(100, v=(0.0, 0.0, -speed), cut_id=0)])
        Jc, _, _ = _closed_form(50.0, delta, speed)
        D, W = _held_run(sc, 20)
        assert np.all(D == 0.0), speed
        # full normal reaction every substep (nothing is ever released)
        assert np.allclose(-W[:, 2], -Jc / DT, rtol=1e-10, atol=0.0)


def test_lead_band_edge_is_inclusive():
    # f = b_lead (= dx) exactly in front of the edge is still the front band,
    # f just beyond it is not; both overlap the blade through a larger
    # particle radius (s_R = 5 so R_p > b_lead)
    # (the particle sits at z = 0 so that f = z_e is computed without rounding)
    speed = 0.2
    x1 = np.array([X0[0], X0[1], 0.0])
    for f, accumulates in ((DX, True), (DX * (1 + 1e-9), False)):
        blade = bi.Blade(pose_x=tuple(x1 + np.array([0.0, 0.0, f])),
                         segments=[bi.Segment(100, v=(0.0, 0.0, -speed), cut_id=0)])
        sc = bi.Scene(X=x1[None, :].copy(), dx=DX, V0=V0, rho=RHO, dt=DT,
                      gravity=(0.0, 0.0, 0.0), floor=False, s_R=5.0, blade=blade)
        D, W = _held_run(sc, 1)
        assert W[0, 2] > 0.0  # contact active in both cases
        assert (D[0] > 0.0) == accumulates, (f, D)
