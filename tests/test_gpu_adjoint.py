"""GPU checkpoints and the GPU adjoint of the substep (calibration of E, nu
and the blade velocity from reaction-force trajectories, Eq. 16) against the
FP64 oracle adjoint and against central finite differences."""
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


def _calib(E=1e5, nu=0.3, speed=0.2, n_steps=60):
    """Calibration geometry scaled down: 20 x 10 x 10 mm block, 16 particles
    per cell, the edge 0.5 mm above the top, D release within the run."""
    return bi.single_cut_cuboid(ppc_axes=(4, 2, 2), size=(0.02, 0.01, 0.01), dx=2.5e-3,
                                n_down=n_steps, edge_z0=0.0102, speed=speed, E=E, nu=nu,
                                G_c=0.5)


def test_checkpoint_restore_is_bitwise(pkg):
    sc = bi.single_cut_cuboid(size=(0.04, 0.02, 0.02), edge_z0=0.0205, speed=0.5, n_down=200)
    s = pkg.Scene(sc, wrench_history=60)
    s.step(15)
    ck_dev = s.checkpoint()
    ck_host = s.checkpoint(device=False)
    s.step(20)
    ref = s.read("x", "v", "F", "D", "ut", "mask1", "mask2")
    ref_w = s.wrench_history(15, 20)
    assert np.abs(ref_w[:, :3]).max() > 0
    for ck in (ck_dev, ck_host):
        s.restore(ck)
        assert s.info().step == 15
        s.step(20)
        got = s.read("x", "v", "F", "D", "ut", "mask1", "mask2")
        for k in ref:
            assert np.array_equal(got[k], ref[k]), k
        assert np.array_equal(s.wrench_history(15, 20), ref_w)
    # a checkpoint stays valid after the scene moves into a batch (scenes
    # that keep a wrench history stay on the plain path, so use another)
    s2 = pkg.Scene(sc)
    s2.step(15)
    ck2 = s2.checkpoint()
    b = pkg.Batch(max_particles=sc.n + 100, max_nodes=50000, max_scenes=2)
    b.add(s2)
    b.step(7)
    s2.restore(ck2)
    b.step(20)
    got = s2.read("x", "v", "F", "D", "ut", "mask1", "mask2")
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    b.close()


def test_checkpoint_rejects_foreign_buffer(pkg):
    a = pkg.Scene(_calib())
    b = pkg.Scene(bi.single_cut_cuboid(size=(0.02, 0.01, 0.02), edge_z0=0.021))
    with pytest.raises(pkg.BMError):
        b.restore(a.checkpoint())


def test_adjoint_matches_oracle_adjoint(pkg):
    """dL/dE, dL/dnu, dL/dspeed of L = sum_n |F_B^n - F_target^n|^2 over 60
    substeps (checkpoint every 7): float32 GPU adjoint vs FP64 oracle adjoint
    on the same scene and target."""
    from paper_2609_27342_gb300.calibration import force_loss_and_grad
    n = 60
    target = O.forces(_calib(E=1.5e5, n_steps=n), n)
    sc = _calib(n_steps=n)
    ref = O.gradient(sc, target, n, every=7)
    loss, g = force_loss_and_grad(sc, target, n, every=7)
    # measured on GB300: loss 2.3e-5, dE 9e-6, dnu 9e-6, dv 4.8e-5 (relative)
    assert abs(loss - ref["loss"]) <= 2e-4 * ref["loss"]
    assert abs(g["E"] - ref["dE"]) <= 1e-4 * abs(ref["dE"]), (g["E"], ref["dE"])
    assert abs(g["nu"] - ref["dnu"]) <= 1e-4 * abs(ref["dnu"]), (g["nu"], ref["dnu"])
    assert abs(g["v_seg"][0, 2] - ref["dv_seg"][0, 2]) <= 5e-4 * abs(ref["dv_seg"][0, 2])


def test_adjoint_full_size_matches_oracle_adjoint_and_differences(pkg):
    """The calibration workload itself (32,000 particles, 200 substeps,
    checkpoint every 20; target at E = 1.5e5 Pa): float32 GPU adjoint vs the
    FP64 oracle adjoint, the error stated per result; and the oracle adjoint
    vs central differences of the FP64 forward at relative step 1e-7.

    The force trajectory has jumps (a cutting-progress release or a label
    moving by one substep when a parameter moves), so differences at a large
    step mix the smooth derivative with the density of those events; at a
    step of 1e-7 no event moves (an event inside the bracket would show as
    a difference many orders of magnitude off) and the differences measure
    the derivative with the decisions held, which is what the adjoint
    computes."""
    from paper_2609_27342_gb300.calibration import force_loss_and_grad
    n, every = 200, 20
    target = O.forces(bi.calibration_scene(E=1.5e5), n)
    sc = bi.calibration_scene()
    ref = O.gradient(sc, target, n, every=every)
    loss, g = force_loss_and_grad(sc, target, n, every=every)
    err = {"loss": abs(loss - ref["loss"]) / ref["loss"],
           "E": abs(g["E"] - ref["dE"]) / abs(ref["dE"]),
           "nu": abs(g["nu"] - ref["dnu"]) / abs(ref["dnu"]),
           "speed": abs(g["v_seg"][0, 2] - ref["dv_seg"][0, 2]) / abs(ref["dv_seg"][0, 2])}

    def L(**kw):
        return O.force_loss(O.forces(bi.calibration_scene(**kw), n), target)

    h = 1e-7
    jobs = {"E": ({"E": 1e5 * (1 + h)}, {"E": 1e5 * (1 - h)}, 2 * h * 1e5),
            "nu": ({"nu": 0.3 * (1 + h)}, {"nu": 0.3 * (1 - h)}, 2 * h * 0.3),
            "speed": ({"speed": 0.2 * (1 + h)}, {"speed": 0.2 * (1 - h)}, 2 * h * 0.2)}
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(6) as ex:
        fut = {k: (ex.submit(L, **a), ex.submit(L, **b), d) for k, (a, b, d) in jobs.items()}
        fd = {k: (p.result() - m.result()) / d for k, (p, m, d) in fut.items()}
    # d/d(speed) of a downward segment velocity v_z = -speed is -dL/dv_z
    ad_o = {"E": ref["dE"], "nu": ref["dnu"], "speed": -ref["dv_seg"][0, 2]}
    fd_err = {k: abs(ad_o[k] - fd[k]) / abs(fd[k]) for k in fd}
    record("adjoint_full_size", **{"gpu_vs_oracle_" + k: v for k, v in err.items()},
           **{"oracle_vs_fd_" + k: v for k, v in fd_err.items()})
    assert err["loss"] <= 1e-3, err
    assert err["E"] <= 1e-3 and err["nu"] <= 1e-3 and err["speed"] <= 1e-3, err
    assert all(v <= 1e-4 for v in fd_err.values()), fd_err


def test_adjoint_autograd_matches_central_differences(pkg):
    """The autograd.Function on the calibration workload (32,000 particles,
    200 substeps, checkpoint every 20; target at E = 1.5e5 Pa) against
    central differences of the GPU forward with relative step 1e-3."""
    import torch
    from paper_2609_27342_gb300.calibration import ForceTrajectory, forces
    n = 200
    target = torch.as_tensor(forces(bi.calibration_scene(E=1.5e5), n))
    spec = bi.calibration_scene()
    E = torch.tensor(1e5, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    v = torch.tensor([[0.0, 0.0, -0.2]], dtype=torch.float64, requires_grad=True)
    F = ForceTrajectory.apply(E, nu, v, spec, n, 20)
    loss = ((F - target) ** 2).sum()
    loss.backward()

    def L(**kw):
        f = forces(bi.calibration_scene(**kw), n)
        return float(np.sum((f - target.numpy()) ** 2))

    fd = {"E": (L(E=1e5 * 1.001) - L(E=1e5 * 0.999)) / (2e-3 * 1e5),
          "nu": (L(nu=0.3 * 1.001) - L(nu=0.3 * 0.999)) / (2e-3 * 0.3),
          "speed": (L(speed=0.2 * 1.001) - L(speed=0.2 * 0.999)) / (2e-3 * 0.2)}
    ad = {"E": E.grad.item(), "nu": nu.grad.item(), "speed": -v.grad[0, 2].item()}
    rel = {k: abs(ad[k] - fd[k]) / abs(fd[k]) for k in fd}
    record("adjoint_autograd_fd_1e-3", **rel)
    # E and the blade speed: the float32 differences at relative step 1e-3
    # agree with the adjoint.  For nu a step of 1e-3 moves cutting-progress
    # releases and labels by a substep (the loss jumps there), so those
    # differences include the event density that the adjoint -- the
    # derivative with the decisions held -- leaves out by construction; nu is
    # checked against the FP64 adjoint and FP64 differences at a step that
    # moves no event (test above) and only loosely here.
    tol = {"E": 1e-3, "nu": 0.1, "speed": 1e-2}
    for k in fd:
        assert rel[k] <= tol[k], (k, ad[k], fd[k])
