"""Seeded synthetic workloads shared by the oracle and the CUDA path.

This module only *describes* inputs: particle reference positions sampled on
a lattice, material and contact parameters, blade geometry and prescribed
blade trajectories, and request streams.  It holds none of the method's
arithmetic (no shape functions, stresses, contact laws or grid transfers), so
the FP64 oracle and the GPU library can both consume it without sharing code.

Every position is rounded to the nearest float32 so that both sides start from
bit-identical reference positions.

Workload recipes (paper scene parameters where the paper prints them):
  * cuboid / cylinder sampling with 2x2x2 particles per reference cell at
    offsets 1/4 and 3/4 of a cell (16 per cell for the 2x2x4 lattice);
  * a 1 mm planar blade, half-length 50 mm, height 100 mm;
  * contact constants s_R = s_n = 1, gamma_k = gamma_c = 0.5, blade mu = 0.2
    (the knife friction used in the paper's banana experiment, Sec. IV-C);
  * zeta = 0.9 (Sec. IV-C), G_c a scene parameter (default 50 J/m^2).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


def _f32(a: np.ndarray) -> np.ndarray:
    """Round to float32 and return as float64 (exactly representable)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


# ----------------------------------------------------------------------------
# particle sampling
# ----------------------------------------------------------------------------

def lattice_cuboid(size: Sequence[float], dx: float, per_axis=(2, 2, 2),
                   origin=(0.0, 0.0, 0.0), jitter: float = 0.0,
                   seed: int = 0) -> np.ndarray:
    """Regular lattice of ``per_axis`` particles per cell filling a box.

    Cell c along an axis holds particles at (c + (j + 1/2)/k) * dx for
    j = 0..k-1 (k = 2 gives offsets 1/4 and 3/4).  ``jitter`` is a fraction
    of the sub-cell spacing (uniform, seeded); it is kept below 1/2 so a
    particle never leaves its sub-cell.
    """
    n = [int(round(s / dx)) for s in size]
    axes = []
    for a in range(3):
        k = per_axis[a]
        c = np.arange(n[a])[:, None]
        j = np.arange(k)[None, :]
        axes.append(((c + (j + 0.5) / k) * dx).reshape(-1) + origin[a])
    gx, gy, gz = np.meshgrid(axes[0], axes[1], axes[2], indexing="ij")
    X = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        sub = np.array([dx / k for k in per_axis])
        X = X + rng.uniform(-jitter, jitter, X.shape) * sub[None, :]
    return _f32(X)


def lattice_cylinder(length: float, radius: float, dx: float,
                     per_axis=(2, 2, 2), origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Lattice points of a cylinder with axis along x.

    The cylinder spans x in [0, length] and rests on z = 0: its axis is at
    (y, z) = (radius, radius) relative to ``origin``.
    """
    box = lattice_cuboid((length, 2 * radius, 2 * radius), dx, per_axis, (0.0, 0.0, 0.0))
    r2 = (box[:, 1] - radius) ** 2 + (box[:, 2] - radius) ** 2
    X = box[r2 <= radius * radius] + np.asarray(origin)[None, :]
    return _f32(X)


# ----------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------

@dataclass
class Segment:
    """Piecewise-constant tool twist held for ``n_steps`` substeps.

    For a kinematic tool this is the prescribed twist; for a dynamic tool it
    is the servo target.  ``cut_id`` >= 0 names the cut (ternary digit)
    this stroke creates; -1 marks a non-cutting move (push).
    """
    n_steps: int
    v: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    omega: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    cut_id: int = -1


@dataclass
class Blade:
    """Planar blade: an oriented box behind a straight edge (tool frame).

    The tool frame origin is the pose position x_B; the edge midpoint sits at
    ``edge_point`` in tool coordinates.  normal/edge_dir/front_dir are the
    tool-frame n, e, d of the paper's blade coordinates (Sec. III-C).
    """
    edge_point: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    normal: Tuple[float, float, float] = (1.0, 0.0, 0.0)
    edge_dir: Tuple[float, float, float] = (0.0, 1.0, 0.0)
    front_dir: Tuple[float, float, float] = (0.0, 0.0, -1.0)
    half_length: float = 0.05
    thickness: float = 1e-3
    height: float = 0.1
    mu_s: float = 0.2
    mu_d: float = 0.2
    mass: float = 0.0                      # 0 => kinematic (w_B = 0)
    inertia: Tuple[float, ...] = (0.0,) * 9  # body frame, row-major
    pose_x: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    pose_R: Tuple[float, ...] = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    servo_gain: float = 0.0                # <= 0 => 1/(10 dt)
    rigid_interval: int = 1
    segments: List[Segment] = field(default_factory=list)


@dataclass
class Scene:
    """Everything one simulation needs besides the solver itself."""
    X: np.ndarray                          # (N, 3) reference positions
    E: float = 1e5
    nu: float = 0.3
    rho: float = 1000.0
    dx: float = 5e-3
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    V0: float = (5e-3) ** 3 / 8
    dt: float = 1e-4
    beta: float = 0.99
    gravity: Tuple[float, float, float] = (0.0, 0.0, -9.81)
    floor: bool = True
    floor_z: float = 0.0
    s_R: float = 1.0
    s_n: float = 1.0
    gamma_k: float = 0.5
    gamma_c: float = 0.5
    pair_contact: bool = False
    pair_mu_s: float = 0.2
    pair_mu_d: float = 0.2
    G_c: float = 50.0
    zeta: float = 0.9
    u_min: float = 1e-3
    b_back: float = -1.0                   # <= 0 => dx
    b_lead: float = -1.0                   # <= 0 => dx
    band_half_width: float = -1.0          # <= 0 => 6 dx  (h_k, Sec. III-D)
    tool_contact: bool = True
    blade: Optional[Blade] = None
    name: str = ""
    model: str = "neo_hookean"   # or "fixed_corotated" (the paper's elastic model)
    yield_stress: float = 0.0    # > 0: von Mises plasticity projection (Pa)
    viscosity: float = 0.0       # > 0: Newtonian viscosity (Pa s)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    def replace(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)


def plate_inertia(mass: float, thickness: float, length: float, height: float):
    """Box inertia about its centre in the blade frame (n, e, d axes)."""
    a, b, c = thickness, length, height
    return (mass * (b * b + c * c) / 12.0, 0.0, 0.0,
            0.0, mass * (a * a + c * c) / 12.0, 0.0,
            0.0, 0.0, mass * (a * a + b * b) / 12.0)


def rot_z(deg: float):
    c, s = math.cos(math.radians(deg)), math.sin(math.radians(deg))
    return (c, -s, 0.0, s, c, 0.0, 0.0, 0.0, 1.0)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def single_cut_cuboid(ppc_axes=(2, 2, 2), n_down: int = 500, edge_z0: float = 0.052,
                      speed: float = 0.2, size=(0.10, 0.05, 0.05), dx: float = 5e-3,
                      dt: float = 1e-4, E: float = 1e5, nu: float = 0.3,
                      G_c: float = 50.0, jitter: float = 0.0, seed: int = 0) -> Scene:
    """Single cut, plain method: neo-Hookean cuboid 0.10 x 0.05 x 0.05 m.

    E = 1e5 Pa, nu = 0.3, rho = 1000, dx = 5 mm (20 x 10 x 10 cells),
    2^3 particles per cell (16,000), gravity and a frictionless floor; a 1 mm
    planar blade in the plane x = 0.05 moves down at ``speed`` with
    prescribed kinematics; dt = 1e-4 s.
    """
    X = lattice_cuboid(size, dx, ppc_axes, jitter=jitter, seed=seed)
    ppc = ppc_axes[0] * ppc_axes[1] * ppc_axes[2]
    blade = Blade(pose_x=(size[0] / 2, size[1] / 2, edge_z0),
                  segments=[Segment(n_down, v=(0.0, 0.0, -speed), cut_id=0)])
    return Scene(X=X, E=E, nu=nu, dx=dx, V0=dx ** 3 / ppc, dt=dt, G_c=G_c,
                 blade=blade, name="single_cut_cuboid")


def cylinder_cuts_push(dx: float = 2e-3, length: float = 0.2, radius: float = 0.02,
                       dt: float = 5e-5, scale_steps: float = 1.0) -> Scene:
    """Progressive + intersecting cuts with a push, two-way coupled tool.

    Neo-Hookean cylinder 0.2 m long, r = 0.02 m (axis along x, resting on
    the floor), E = 5e4 Pa, nu = 0.35, dx = 2 mm, 2^3 particles per cell
    (about 251k particles); tool mass 0.2 kg with plate inertia, servo
    tracking of the segment twists; material-material contact on;
    dt = 5e-5 s, 4,000 substeps in total (``scale_steps`` shrinks every
    segment for short runs).  Program (world-frame twists about the edge
    midpoint):
      1. cut 0: plane rotated +15 deg about z through x = 0.1 m, down 45 mm
         in 800 substeps, up again in 800;
      2. rotate -30 deg about z in 100 substeps (no cut);
      3. cut 1: down 45 mm in 800 substeps (planes 30 deg apart, meeting at
         the cylinder axis), back up to z = 10 mm in 200;
      4. push: 10 mm along the blade normal at 0.5 m/s in 400 substeps (no
         cut), then lift clear in the remaining 900.
    """
    X = lattice_cylinder(length, radius, dx)
    z0 = 2 * radius + 0.005
    s = scale_steps
    n_down = max(1, int(round(800 * s)))
    n_rot = max(1, int(round(100 * s)))
    n_up2 = max(1, int(round(200 * s)))
    n_push = max(1, int(round(400 * s)))
    n_lift = max(1, int(round(900 * s)))
    vz = 0.045 / (n_down * dt)
    wz = -math.radians(30.0) / (n_rot * dt)
    vz2 = (0.010 - (z0 - 0.045)) / (n_up2 * dt)
    # blade normal after the rotation: rot_z(-15) applied to +x
    c, sn = math.cos(math.radians(-15.0)), math.sin(math.radians(-15.0))
    vpush = 0.010 / (n_push * dt)
    segs = [Segment(n_down, v=(0, 0, -vz), cut_id=0),
            Segment(n_down, v=(0, 0, vz), cut_id=0),
            Segment(n_rot, omega=(0, 0, wz), cut_id=-1),
            Segment(n_down, v=(0, 0, -vz), cut_id=1),
            Segment(n_up2, v=(0, 0, vz2), cut_id=1),
            Segment(n_push, v=(vpush * c, vpush * sn, 0.0), cut_id=-1),
            Segment(n_lift, v=(0, 0, 0.05 / (n_lift * dt)), cut_id=-1)]
    mass = 0.2
    thick, half_len, height = 1e-3, 0.05, 0.1
    blade = Blade(pose_x=(length / 2, radius, z0), pose_R=rot_z(15.0),
                  mass=mass, inertia=plate_inertia(mass, thick, 2 * half_len, height),
                  thickness=thick, half_length=half_len, height=height, segments=segs)
    return Scene(X=X, E=5e4, nu=0.35, dx=dx, V0=dx ** 3 / 8, dt=dt,
                 pair_contact=True, blade=blade, name="cylinder_cuts_push")


def p_wave_speed(E: float, nu: float, rho: float) -> float:
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    return math.sqrt((lam + 2 * mu) / rho)


def batched_scenes(n_scenes: int = 256, seed: int = 2, n_min: int = 4096,
                   n_max: int = 65536, dx: float = 5e-3, n_substeps: int = 1000,
                   rho: float = 1000.0) -> List[Scene]:
    """Uneven batch: cuboids with particle counts log-uniform in [4k, 64k].

    Sizes 2:1:1 with n_y = n_z = round((N/16)^(1/3)) cells and n_x = 2 n_y
    (8 particles per cell), E log-uniform in [1e4, 1e6] Pa, nu uniform in
    [0.25, 0.45], a blade plane through the centre with a seeded random
    normal, front direction -z projected into the plane, speed uniform in
    [0.05, 0.5] m/s, per-scene dt = min(1e-4, 0.3 dx / c_p).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_scenes):
        N = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        ny = max(2, int(round((N / 16.0) ** (1.0 / 3.0))))
        nx = 2 * ny
        size = (nx * dx, ny * dx, ny * dx)
        E = math.exp(rng.uniform(math.log(1e4), math.log(1e6)))
        nu = rng.uniform(0.25, 0.45)
        speed = rng.uniform(0.05, 0.5)
        # random unit normal, made orthogonal to z where possible so that the
        # blade can sweep downward through the body
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        d = np.array([0.0, 0.0, -1.0])
        d = d - d.dot(nrm) * nrm
        if np.linalg.norm(d) < 0.3:   # nearly horizontal plane: tilt the normal
            nrm = np.array([nrm[0], nrm[1], 0.3 * np.sign(nrm[2] or 1.0)])
            nrm /= np.linalg.norm(nrm)
            d = np.array([0.0, 0.0, -1.0]) - (-nrm[2]) * nrm
        d /= np.linalg.norm(d)
        e = np.cross(d, nrm)
        e /= np.linalg.norm(e)
        R = np.stack([nrm, e, d], axis=1)  # columns: tool axes in world
        X = lattice_cuboid(size, dx)
        cp = p_wave_speed(E, nu, rho)
        dt = min(1e-4, 0.3 * dx / cp)
        centre = np.array(size) / 2
        edge0 = centre - d * (size[2] / 2 + 0.002)
        blade = Blade(normal=(1.0, 0.0, 0.0), edge_dir=(0.0, 1.0, 0.0), front_dir=(0.0, 0.0, 1.0),
                      half_length=float(max(size)),
                      pose_x=tuple(float(t) for t in edge0), pose_R=tuple(float(t) for t in R.ravel()),
                      segments=[Segment(n_substeps, v=tuple(float(t) for t in speed * d), cut_id=0)])
        # reference grid offset by half a cell: each base cell (Eq. 1 stencil
        # origin) then holds exactly one lattice cell's 2 x 2 x 2 particles
        out.append(Scene(X=X, E=E, nu=nu, rho=rho, dx=dx, origin=(-dx / 2,) * 3,
                         V0=dx ** 3 / 8, dt=dt, blade=blade, name=f"batch{i}"))
    return out


@dataclass
class Request:
    arrival_s: float
    scene: Scene
    n_substeps: int


def serving_requests(n_requests: int = 64, rate_hz: float = 50.0, seed: int = 3,
                     n_min: int = 8000, n_max: int = 500000, dx: float = 5e-3,
                     steps_min: int = 200, steps_max: int = 2000,
                     rho: float = 1000.0) -> List[Request]:
    """Poisson request stream of cutting rollouts.

    Particle counts log-uniform in [8k, 500k], substeps uniform in
    {200..2000}, 1-3 sequential cuts per rollout, each a downward stroke
    with a random plane as in the uneven batch.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        N = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        ny = max(2, int(round((N / 16.0) ** (1.0 / 3.0))))
        nx = 2 * ny
        size = (nx * dx, ny * dx, ny * dx)
        E = math.exp(rng.uniform(math.log(1e4), math.log(1e6)))
        nu = rng.uniform(0.25, 0.45)
        n_steps = int(rng.integers(steps_min, steps_max + 1))
        n_cuts = int(rng.integers(1, 4))
        cp = p_wave_speed(E, nu, rho)
        dt = min(1e-4, 0.3 * dx / cp)
        X = lattice_cuboid(size, dx)
        # one vertical plane per cut, spaced along x; strokes share the step budget
        per = max(1, n_steps // n_cuts)
        speed = rng.uniform(0.05, 0.5)
        segs = [Segment(per if k < n_cuts - 1 else n_steps - per * (n_cuts - 1),
                        v=(0.0, 0.0, -speed), cut_id=k) for k in range(n_cuts)]
        blade = Blade(pose_x=(size[0] / 2, size[1] / 2, size[2] + 0.002),
                      half_length=float(max(size)), segments=segs)
        out.append(Request(arrival_s=t, scene=Scene(X=X, E=E, nu=nu, rho=rho, dx=dx,
                                                     origin=(-dx / 2,) * 3, V0=dx ** 3 / 8,
                                                     dt=dt, blade=blade, name=f"req{i}"),
                           n_substeps=n_steps))
    return out


def calibration_scene(E: float = 1e5, nu: float = 0.3, speed: float = 0.2,
                      n_steps: int = 200) -> Scene:
    """Adjoint calibration workload: the single-cut cuboid at 16 particles per
    cell (2 x 2 x 4 lattice, doubled along the blade normal -> 32,000
    particles), edge starting 0.5 mm above the top, 200 substeps."""
    return single_cut_cuboid(ppc_axes=(4, 2, 2), n_down=n_steps, edge_z0=0.0505,
                             speed=speed, E=E, nu=nu)


def scene_fields(sc: Scene) -> dict:
    """Flat parameter dictionary (no derived quantities)."""
    d = {f.name: getattr(sc, f.name) for f in dataclasses.fields(sc)}
    d.pop("X")
    d.pop("blade")
    d.pop("name")
    return d
