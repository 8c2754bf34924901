"""CPU pins of the FP64 oracle adjoint (reverse mode of one substep, with the
discrete decisions held fixed) used for calibration of E, nu and the blade
velocity from reaction-force trajectories (Eq. 16).

Pinned against things other than the adjoint itself: the transpose identity
of the Eq. 8 coupling map, central finite differences of the stress, a
dot-product test of a whole substep against central differences of the
forward oracle, and the gradient of a multi-substep loss against central
differences of the forward oracle."""
import dataclasses

import numpy as np
import pytest

import bm_inputs as bi
from oracle import oracle as O


def test_couple_transpose_identity():
    """<C S, T> = <S, C^T T> for the Eq. 8 map with conflicting codes."""
    rng = np.random.default_rng(1)
    # codes: 0 (unassigned), 1 / 2 (sides of cut 0), 4 / 5 (cut 1 digit 1 with
    # cut 0 sides 1 / 2), 7 (cut 0 side 1, cut 1 side 2)
    codes = [0, 1, 2, 4, 5, 7]
    for _ in range(5):
        m = rng.uniform(0.05, 1.0, len(codes))
        S = rng.normal(size=(len(codes), 6))
        T = rng.normal(size=(len(codes), 6))
        lhs = np.sum(O.couple(codes, m, S) * T)
        rhs = np.sum(S * O.couple_T(codes, m, T))
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


def test_piola_vjp_matches_finite_differences():
    rng = np.random.default_rng(2)
    mu, lam = 3.8e4, 5.7e4
    for _ in range(5):
        F = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
        Pb = rng.normal(size=(3, 3))
        dF = rng.normal(size=(3, 3))
        Fb, mub, lamb = O.piola_vjp(F, mu, lam, Pb)
        eps = 1e-6
        fd = (O.piola(F + eps * dF, mu, lam)[0] - O.piola(F - eps * dF, mu, lam)[0]) / (2 * eps)
        assert abs(np.sum(Pb * fd) - np.sum(Fb * dF)) <= 1e-6 * np.abs(Fb).sum() * np.abs(dF).max()
        fd_mu = (O.piola(F, mu * (1 + 1e-6), lam)[0] - O.piola(F, mu * (1 - 1e-6), lam)[0]) / (2e-6 * mu)
        fd_lam = (O.piola(F, mu, lam * (1 + 1e-6))[0] - O.piola(F, mu, lam * (1 - 1e-6))[0]) / (2e-6 * lam)
        assert abs(np.sum(Pb * fd_mu) - mub) <= 1e-6 * (abs(mub) + 1)
        assert abs(np.sum(Pb * fd_lam) - lamb) <= 1e-6 * (abs(lamb) + 1)


def _contact_scene(E=8e4, nu=0.32, v_seg=(0.0, 0.0, -0.3)):
    """A small block with the blade already 1.5 mm inside its top, moving
    down: blade contact (stick and slip), the front band, floor contact."""
    dx = 2.5e-3
    sc = bi.single_cut_cuboid(size=(0.02, 0.01, 0.01), dx=dx, edge_z0=0.0085, speed=0.3,
                              E=E, nu=nu, G_c=5.0)
    b = dataclasses.replace(sc.blade, segments=[bi.Segment(100, v=tuple(v_seg), cut_id=0)])
    return dataclasses.replace(sc, blade=b, gravity=(0.0, 0.0, -9.81))


def _random_state(sc, rng):
    n = sc.n
    x = sc.X + 1e-4 * rng.normal(size=(n, 3))
    x[:, 2] -= sc.X[:, 2].min() - 0.0002  # bottom layer presses into the floor
    v = 0.05 * rng.normal(size=(n, 3))
    F = np.tile(np.eye(3).ravel(), (n, 1)) + 0.02 * rng.normal(size=(n, 9))
    ut = 2e-5 * rng.normal(size=(n, 3))
    D = np.where(rng.uniform(size=n) < 0.5, 1.0, 0.3)
    digits = np.zeros((n, O.MAX_CUTS))
    digits[:, 1] = np.where(sc.X[:, 0] < 0.01, 1, 2)  # an earlier cut splits the block
    digits[rng.uniform(size=n) < 0.2, 1] = 0
    return {"x": x, "v": v, "F": F, "ut": ut, "D": D, "digits": digits}


def _one_substep(sc, st, xB=None):
    """The scene at its second substep (the cut has started, so D is not
    reset) with the given state and tool position."""
    o = O.OracleScene(sc, wrench_capacity=4)
    t = o.tool()
    o.step(1)
    for k in ("x", "v", "F", "ut", "D", "digits"):
        o.set(k, st[k])
    o.set_tool(t[0:3] if xB is None else xB, t[3:12], t[12:15], t[15:18])
    return o


def _outputs(sc, st, xB=None):
    o = _one_substep(sc, st, xB)
    o.step(1)
    return {"x": o.get("x"), "v": o.get("v"), "F": o.get("F"), "ut": o.get("ut"),
            "force": o.wrench_history(1, 1)[0, :3], "xB": o.tool()[0:3]}


def test_substep_adjoint_dot_product():
    """<adjoint out, delta in> = d/de <adjoint in, outputs(in + e delta)> for
    state, tool position, E, nu and the blade velocity (central differences
    of the forward oracle, no decision flips at this step size)."""
    rng = np.random.default_rng(5)
    sc = _contact_scene()
    st = _random_state(sc, rng)
    out0 = _outputs(sc, st)
    assert np.linalg.norm(out0["force"]) > 0  # the blade is in contact
    w = {k: rng.normal(size=np.shape(v)) for k, v in out0.items()}

    def L(scn, state, xB=None):
        o = _outputs(scn, state, xB)
        return sum(float(np.sum(w[k] * o[k])) for k in w)

    o = _one_substep(sc, st)
    adj = O.OracleAdjoint(sc.n)
    for k in ("x", "v", "F", "ut"):
        adj.field(k)[:] = w[k].reshape(sc.n, -1)
    adj.field("xB")[:] = w["xB"]
    adj.substep(o, w["force"])
    th = adj.theta(o)

    # state directions
    for name, scale in (("x", 1e-9), ("v", 1e-7), ("F", 1e-7), ("ut", 1e-10)):
        d = rng.normal(size=st[name].shape)
        sp = dict(st, **{name: st[name] + scale * d})
        sm = dict(st, **{name: st[name] - scale * d})
        fd = (L(sc, sp) - L(sc, sm)) / (2 * scale)
        ad = float(np.sum(adj.field(name) * d.reshape(sc.n, -1)))
        assert abs(fd - ad) <= 1e-5 * max(abs(ad), 1e-8 * np.abs(adj.field(name)).sum()), (name, fd, ad)
    # tool position
    xB0 = o.tool()[0:3]
    d = rng.normal(size=3)
    fd = (L(sc, st, xB0 + 1e-9 * d) - L(sc, st, xB0 - 1e-9 * d)) / 2e-9
    ad = float(np.dot(adj.field("xB")[0], d))
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    # material parameters
    for name, val in (("E", sc.E), ("nu", sc.nu)):
        h = 1e-7 * val
        fd = (L(dataclasses.replace(sc, **{name: val + h}), st) -
              L(dataclasses.replace(sc, **{name: val - h}), st)) / (2 * h)
        assert abs(fd - th[name]) <= 1e-5 * abs(th[name]), (name, fd, th[name])
    # blade velocity of the active segment
    for i in range(3):
        vp = np.array(sc.blade.segments[0].v)
        vm = vp.copy()
        vp[i] += 1e-8
        vm[i] -= 1e-8
        fd = (L(_contact_scene(v_seg=vp), st) - L(_contact_scene(v_seg=vm), st)) / 2e-8
        ad = th["v_seg"][0, i]
        assert abs(fd - ad) <= 1e-5 * max(abs(ad), 1e-3 * np.abs(th["v_seg"][0]).max()), (i, fd, ad)


def _calib(E=1e5, nu=0.3, speed=0.2, n_steps=40):
    """Config-4 geometry scaled down: a 20 x 10 x 10 mm block at 16
    particles per cell, the edge 0.5 mm above the top."""
    sc = bi.single_cut_cuboid(ppc_axes=(4, 2, 2), size=(0.02, 0.01, 0.01), dx=2.5e-3,
                              n_down=n_steps, edge_z0=0.0102, speed=speed, E=E, nu=nu,
                              G_c=0.5)
    return sc


@pytest.mark.parametrize("every", [7, 60])
def test_loss_gradient_matches_central_differences(every):
    """dL/dE, dL/dnu, dL/dspeed of L = sum_n |F_B^n - F_target^n|^2 over 60
    substeps (target generated at E = 1.5 E) against central differences of
    the forward oracle; the checkpoint interval does not change the result."""
    n = 60
    target = O.forces(_calib(E=1.5e5, n_steps=n), n)
    g = O.gradient(_calib(n_steps=n), target, n, every=every)
    assert g["loss"] > 0
    dspeed = -g["dv_seg"][0, 2]  # v_seg = (0, 0, -speed)
    for name, base, kw, ad in (("E", 1e5, "E", g["dE"]), ("nu", 0.3, "nu", g["dnu"]),
                               ("speed", 0.2, "speed", dspeed)):
        h = 1e-6 * base
        lp = O.force_loss(O.forces(_calib(n_steps=n, **{kw: base + h}), n), target)
        lm = O.force_loss(O.forces(_calib(n_steps=n, **{kw: base - h}), n), target)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - ad) <= 1e-3 * abs(fd), (name, fd, ad)
