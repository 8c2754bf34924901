"""Material calibration: gradients of reaction-force trajectories.

``ForceTrajectory`` is a ``torch.autograd.Function`` that runs a scene for
``n_steps`` substeps and returns its per-substep reaction force F_B^n
(Eq. 16) as a float64 tensor; its backward pass applies the library's
hand-written adjoint of the substep (bm_adjoint_*) in reverse order, with a
checkpoint of the complete state every ``every`` substeps: each checkpoint
interval is recomputed forward once, its per-substep states kept as
checkpoints too, then the adjoint runs back through them.  The discrete
decisions of the forward run (codes, contact active sets, stick or slip, D
release) are held fixed.  Gradients flow to E, nu and the linear velocities
of the blade's trajectory segments.  All simulation work runs in the CUDA
kernels; this module only orders the calls.
"""
from __future__ import annotations

import copy
from typing import Optional, Tuple

import numpy as np

from .sim import Adjoint, Scene


def with_params(spec, E: float, nu: float, v_seg) -> object:
    """Copy of a scene description with material and segment velocities
    replaced (the description is not modified)."""
    sc = copy.copy(spec)
    sc.E, sc.nu = float(E), float(nu)
    if spec.blade is not None:
        b = copy.copy(spec.blade)
        segs = []
        for s, v in zip(spec.blade.segments, np.asarray(v_seg, np.float64).reshape(-1, 3)):
            t = copy.copy(s)
            t.v = tuple(float(c) for c in v)
            segs.append(t)
        b.segments = segs
        sc.blade = b
    return sc


def _run_forward(spec, n_steps: int, every: int, stream=None):
    scene = Scene(spec, stream=stream, wrench_history=n_steps)
    ck = []
    k = 0
    while k < n_steps:
        ck.append((k, scene.checkpoint()))
        m = min(every, n_steps - k)
        scene.step(m)
        k += m
    forces = scene.wrench_history(0, n_steps)[:, :3].copy()
    return scene, ck, forces


def _run_backward(scene: Scene, ck, fbar: np.ndarray, every: int, n_steps: int) -> dict:
    adj = Adjoint(scene)
    for k0, buf in reversed(ck):
        k1 = min(k0 + every, n_steps)
        scene.restore(buf)
        tape = []
        for j in range(k0, k1):
            tape.append(scene.checkpoint())
            if j + 1 < k1:
                scene.step(1)
        for j in range(k1 - 1, k0 - 1, -1):
            scene.restore(tape[j - k0])
            adj.substep(fbar[j])
        del tape
    out = adj.params()
    adj.close()
    return out


try:
    import torch

    class ForceTrajectory(torch.autograd.Function):
        """forces = ForceTrajectory.apply(E, nu, v_seg, spec, n_steps, every)

        E, nu: 0-d float64 tensors; v_seg: (segments, 3) float64 tensor of
        the blade's segment linear velocities; returns (n_steps, 3) float64
        reaction forces.  Backward gives dL/dE, dL/dnu, dL/dv_seg."""

        @staticmethod
        def forward(ctx, E, nu, v_seg, spec, n_steps: int, every: int = 20):
            sc = with_params(spec, E.item(), nu.item(), v_seg.detach().cpu().numpy())
            scene, ck, forces = _run_forward(sc, n_steps, every)
            ctx.scene, ctx.ck, ctx.n_steps, ctx.every = scene, ck, n_steps, every
            ctx.n_seg = v_seg.shape[0]
            return torch.as_tensor(forces, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_forces):
            fbar = grad_forces.detach().cpu().numpy().astype(np.float64)
            g = _run_backward(ctx.scene, ctx.ck, fbar, ctx.every, ctx.n_steps)
            ctx.scene.close()
            ctx.ck = None
            dE = torch.tensor(g["E"], dtype=torch.float64)
            dnu = torch.tensor(g["nu"], dtype=torch.float64)
            dv = torch.as_tensor(g["v_seg"][:ctx.n_seg], dtype=torch.float64)
            return dE, dnu, dv, None, None, None

except ImportError:  # torch is the package's plumbing; without it only the helpers below work
    ForceTrajectory = None


def force_loss_and_grad(spec, target: np.ndarray, n_steps: int, every: int = 20) -> Tuple[float, dict]:
    """L = sum_n |F_B^n - F_target^n|^2 and its gradient w.r.t. E, nu and the
    segment velocities (adjoint with checkpoints), without autograd."""
    scene, ck, forces = _run_forward(spec, n_steps, every)
    fbar = 2.0 * (forces - np.asarray(target, np.float64))
    g = _run_backward(scene, ck, fbar, every, n_steps)
    scene.close()
    loss = float(np.sum((forces - target) ** 2))
    n_seg = len(spec.blade.segments) if spec.blade is not None else 0
    return loss, {"E": g["E"], "nu": g["nu"], "v_seg": g["v_seg"][:n_seg], "forces": forces}


def forces(spec, n_steps: int) -> np.ndarray:
    """Reaction-force trajectory of a scene (n_steps x 3, float64)."""
    scene = Scene(spec, wrench_history=n_steps)
    scene.step(n_steps)
    f = scene.wrench_history(0, n_steps)[:, :3].copy()
    scene.close()
    return f
