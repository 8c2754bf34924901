"""ctypes shim over the FP64 C oracle (bm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the package smoke check
and the CPU-baseline leg of the benchmark, never by the GPU library.  The shim
only marshals arguments; every step of the method is in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_CUTS = 32
MAX_SEG = 16
HIST = 16   # pair-contact history entries per particle

E_INVERTED = 1
E_NONFINITE = 2
E_HIST_OVERFLOW = 4


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double), ("dx", C.c_double),
                ("origin", C.c_double * 3), ("V0", C.c_double), ("dt", C.c_double),
                ("beta", C.c_double), ("g", C.c_double * 3), ("floor_on", C.c_int),
                ("floor_z", C.c_double), ("s_R", C.c_double), ("s_n", C.c_double),
                ("gamma_k", C.c_double), ("gamma_c", C.c_double), ("pair_on", C.c_int),
                ("pair_mu_s", C.c_double), ("pair_mu_d", C.c_double), ("Gc", C.c_double),
                ("zeta", C.c_double), ("u_min", C.c_double), ("b_back", C.c_double),
                ("b_lead", C.c_double), ("h", C.c_double), ("tool_contact_on", C.c_int),
                ("single_field", C.c_int), ("model", C.c_int), ("yield_stress", C.c_double),
                ("viscosity", C.c_double)]


class Seg(C.Structure):
    _fields_ = [("n_steps", C.c_int), ("cut_id", C.c_int), ("v", C.c_double * 3),
                ("w", C.c_double * 3)]


class BladeC(C.Structure):
    _fields_ = [("edge", C.c_double * 3), ("n", C.c_double * 3), ("e", C.c_double * 3),
                ("d", C.c_double * 3), ("half_len", C.c_double), ("thick", C.c_double),
                ("height", C.c_double), ("mu_s", C.c_double), ("mu_d", C.c_double),
                ("mass", C.c_double), ("inertia", C.c_double * 9), ("x0", C.c_double * 3),
                ("R0", C.c_double * 9), ("kv", C.c_double), ("rigid_interval", C.c_int),
                ("nseg", C.c_int), ("seg", Seg * MAX_SEG)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_create.restype = C.c_void_p
            L.or_create.argtypes = [C.POINTER(Params), C.POINTER(BladeC), C.c_int64, dp, C.c_int64]
            L.or_destroy.argtypes = [C.c_void_p]
            L.or_step.argtypes = [C.c_void_p, C.c_int]
            L.or_step.restype = C.c_int
            L.or_get.argtypes = [C.c_void_p, C.c_int, dp]
            L.or_set.argtypes = [C.c_void_p, C.c_int, dp]
            L.or_get_tool.argtypes = [C.c_void_p, dp]
            L.or_set_tool.argtypes = [C.c_void_p, dp]
            L.or_get_frame.argtypes = [C.c_void_p, dp]
            L.or_set_step.argtypes = [C.c_void_p, C.c_int64, C.c_int]
            L.or_step_count.argtypes = [C.c_void_p]
            L.or_step_count.restype = C.c_int64
            L.or_errors.argtypes = [C.c_void_p]
            L.or_errors.restype = C.c_uint
            L.or_cut_planes.argtypes = [C.c_void_p, dp]
            L.or_cut_planes.restype = C.c_uint
            L.or_impulse_sum.argtypes = [C.c_void_p, dp]
            L.or_last_wrench.argtypes = [C.c_void_p, dp]
            L.or_wrench_history.argtypes = [C.c_void_p, C.c_int64, C.c_int64, dp]
            L.or_grid_dims.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.or_slot_count.argtypes = [C.c_void_p]
            L.or_slot_count.restype = C.c_int64
            L.or_momentum.argtypes = [C.c_void_p, dp]
            L.or_bspline.argtypes = [C.c_double, dp, dp]
            L.or_bspline.restype = C.c_int
            L.or_psi.argtypes = [dp, C.c_double, C.c_double]
            L.or_psi.restype = C.c_double
            L.or_piola.argtypes = [dp, C.c_double, C.c_double, dp]
            L.or_piola.restype = C.c_int
            L.or_code.argtypes = [C.POINTER(C.c_ubyte), C.c_int]
            L.or_code.restype = C.c_int64
            L.or_digit.argtypes = [C.c_int64, C.c_int]
            L.or_digit.restype = C.c_int
            L.or_conflict.argtypes = [C.c_int64, C.c_int64]
            L.or_conflict.restype = C.c_int
            L.or_couple.argtypes = [C.c_int, C.POINTER(C.c_int64), dp, C.c_int, dp]
            L.or_friction.argtypes = [dp, dp, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, dp, dp]
            L.or_box_closest.argtypes = [dp, dp, dp, dp, dp, dp, C.c_double, dp, dp, dp]
            L.or_side_label.argtypes = [dp, dp, dp, dp, dp, dp, dp, C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_double]
            L.or_side_label.restype = C.c_int
            L.or_cut_progress.argtypes = [C.c_double] * 4
            L.or_cut_progress.restype = C.c_double
            L.or_clone.argtypes = [C.c_void_p]
            L.or_clone.restype = C.c_void_p
            L.or_adj_create.argtypes = [C.c_int64]
            L.or_adj_create.restype = C.c_void_p
            L.or_adj_destroy.argtypes = [C.c_void_p]
            L.or_adj_field.argtypes = [C.c_void_p, C.c_int]
            L.or_adj_field.restype = dp
            L.or_adj_theta.argtypes = [C.c_void_p, C.c_void_p, dp]
            L.or_adj_substep.argtypes = [C.c_void_p, C.c_void_p, dp]
            L.or_adj_substep.restype = C.c_int
            L.or_piola_vjp.argtypes = [dp, C.c_double, C.c_double, dp, dp, dp, dp]
            L.or_couple_T.argtypes = [C.c_int, C.POINTER(C.c_int64), dp, C.c_int, dp]
            L.or_polar.argtypes = [dp, dp, dp]
            L.or_piola_fcr.argtypes = [dp, C.c_double, C.c_double, dp]
            L.or_piola_fcr.restype = C.c_int
            L.or_psi_fcr.argtypes = [dp, C.c_double, C.c_double]
            L.or_psi_fcr.restype = C.c_double
            L.or_vonmises.argtypes = [dp, C.c_double, C.c_double]
            L.or_vonmises.restype = C.c_int
            L.or_viscous_piola.argtypes = [dp, dp, C.c_double, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    if n is not None:
        assert a.size == n
    return a


# ---------------------------------------------------------------------------
# unit-level functions
# ---------------------------------------------------------------------------

def bspline(xl: float):
    w = np.zeros(3)
    dw = np.zeros(3)
    b = lib().or_bspline(float(xl), _dp(w), _dp(dw))
    return b, w, dw


def piola(F, mu, lam):
    F = _arr(F, 9)
    P = np.zeros(9)
    clamped = lib().or_piola(_dp(F), mu, lam, _dp(P))
    return P.reshape(3, 3), bool(clamped)


def polar(F):
    """Polar decomposition F = R S (FP64, Jacobi eigen-decomposition of F^T F)."""
    F = _arr(F, 9)
    R = np.zeros(9)
    S = np.zeros(9)
    lib().or_polar(_dp(F), _dp(R), _dp(S))
    return R.reshape(3, 3), S.reshape(3, 3)


def piola_fcr(F, mu, lam):
    """Fixed-corotated first Piola-Kirchhoff stress and the inverted flag."""
    F = _arr(F, 9)
    P = np.zeros(9)
    clamped = lib().or_piola_fcr(_dp(F), mu, lam, _dp(P))
    return P.reshape(3, 3), bool(clamped)


def vonmises(Fe, mu, sigma_y):
    """von Mises projection of an elastic deformation gradient; returns the
    projected matrix and whether the projection acted."""
    a = _arr(Fe, 9).copy()
    acted = lib().or_vonmises(_dp(a), mu, sigma_y)
    return a.reshape(3, 3), bool(acted)


def viscous_piola(F, Fdot, eta):
    """First Piola-Kirchhoff form of the Newtonian viscous stress."""
    P = np.zeros(9)
    lib().or_viscous_piola(_dp(_arr(F, 9)), _dp(_arr(Fdot, 9)), eta, _dp(P))
    return P.reshape(3, 3)


def psi_fcr(F, mu, lam) -> float:
    return lib().or_psi_fcr(_dp(_arr(F, 9)), mu, lam)


def psi(F, mu, lam) -> float:
    F = _arr(F, 9)
    return lib().or_psi(_dp(F), mu, lam)


def code(digits) -> int:
    d = np.zeros(MAX_CUTS, dtype=np.uint8)
    d[:len(digits)] = digits
    return lib().or_code(d.ctypes.data_as(C.POINTER(C.c_ubyte)), MAX_CUTS)


def digit(c: int, k: int) -> int:
    return lib().or_digit(int(c), int(k))


def conflict(a: int, b: int) -> bool:
    return bool(lib().or_conflict(int(a), int(b)))


def couple(codes, m, S):
    codes = np.ascontiguousarray(np.asarray(codes, dtype=np.int64))
    m = _arr(m)
    S = np.ascontiguousarray(np.asarray(S, dtype=np.float64)).copy()
    ns, nc = S.shape
    lib().or_couple(ns, codes.ctypes.data_as(C.POINTER(C.c_int64)), _dp(m), nc, _dp(S))
    return S


def couple_T(codes, m, S):
    """Transpose of the Eq. 8 coupling map (masses and codes fixed)."""
    codes = np.ascontiguousarray(np.asarray(codes, dtype=np.int64))
    m = _arr(m)
    S = np.ascontiguousarray(np.asarray(S, dtype=np.float64)).copy()
    ns, nc = S.shape
    lib().or_couple_T(ns, codes.ctypes.data_as(C.POINTER(C.c_int64)), _dp(m), nc, _dp(S))
    return S


def piola_vjp(F, mu, lam, Pb):
    """(dP/dF)^T Pb, dP/dmu : Pb, dP/dlambda : Pb of the neo-Hookean stress."""
    F = _arr(F, 9)
    Pb = _arr(Pb, 9)
    Fb = np.zeros(9)
    mub = np.zeros(1)
    lamb = np.zeros(1)
    lib().or_piola_vjp(_dp(F), mu, lam, _dp(Pb), _dp(Fb), _dp(mub), _dp(lamb))
    return Fb.reshape(3, 3), float(mub[0]), float(lamb[0])


def friction(u_hist, n, vrel, fn, meff, dt, gk, gc, mus, mud):
    ft = np.zeros(3)
    un = np.zeros(3)
    lib().or_friction(_dp(_arr(u_hist, 3)), _dp(_arr(n, 3)), _dp(_arr(vrel, 3)), fn, meff, dt,
                      gk, gc, mus, mud, _dp(ft), _dp(un))
    return ft, un


def box_closest(c, ax_n, ax_e, ax_d, hext, x, R):
    xc = np.zeros(3)
    nB = np.zeros(3)
    phi = np.zeros(1)
    lib().or_box_closest(_dp(_arr(c, 3)), _dp(_arr(ax_n, 3)), _dp(_arr(ax_e, 3)),
                         _dp(_arr(ax_d, 3)), _dp(_arr(hext, 3)), _dp(_arr(x, 3)), R,
                         _dp(xc), _dp(nB), _dp(phi))
    return xc, nB, float(phi[0])


def side_label(x, v, xe, n, e, d, ve, h, L, b_back, b_lead, dt) -> int:
    return lib().or_side_label(_dp(_arr(x, 3)), _dp(_arr(v, 3)), _dp(_arr(xe, 3)),
                               _dp(_arr(n, 3)), _dp(_arr(e, 3)), _dp(_arr(d, 3)),
                               _dp(_arr(ve, 3)), h, L, b_back, b_lead, dt)


def cut_progress(D, Jc, uc, Wth) -> float:
    return lib().or_cut_progress(D, Jc, uc, Wth)


# ---------------------------------------------------------------------------
# scene
# ---------------------------------------------------------------------------

def _params(sc, single_field=False) -> Params:
    p = Params()
    p.E, p.nu, p.rho, p.dx = sc.E, sc.nu, sc.rho, sc.dx
    p.origin = (C.c_double * 3)(*sc.origin)
    p.V0, p.dt, p.beta = sc.V0, sc.dt, sc.beta
    p.g = (C.c_double * 3)(*sc.gravity)
    p.floor_on, p.floor_z = int(sc.floor), sc.floor_z
    p.s_R, p.s_n, p.gamma_k, p.gamma_c = sc.s_R, sc.s_n, sc.gamma_k, sc.gamma_c
    p.pair_on, p.pair_mu_s, p.pair_mu_d = int(sc.pair_contact), sc.pair_mu_s, sc.pair_mu_d
    p.Gc, p.zeta, p.u_min = sc.G_c, sc.zeta, sc.u_min
    p.b_back, p.b_lead, p.h = sc.b_back, sc.b_lead, sc.band_half_width
    p.tool_contact_on = int(sc.tool_contact)
    p.single_field = int(single_field)
    p.model = {"neo_hookean": 0, "fixed_corotated": 1}[getattr(sc, "model", "neo_hookean")]
    p.yield_stress = float(getattr(sc, "yield_stress", 0.0))
    p.viscosity = float(getattr(sc, "viscosity", 0.0))
    return p


def _blade(b) -> BladeC:
    B = BladeC()
    B.edge = (C.c_double * 3)(*b.edge_point)
    B.n = (C.c_double * 3)(*b.normal)
    B.e = (C.c_double * 3)(*b.edge_dir)
    B.d = (C.c_double * 3)(*b.front_dir)
    B.half_len, B.thick, B.height = b.half_length, b.thickness, b.height
    B.mu_s, B.mu_d, B.mass = b.mu_s, b.mu_d, b.mass
    B.inertia = (C.c_double * 9)(*b.inertia)
    B.x0 = (C.c_double * 3)(*b.pose_x)
    B.R0 = (C.c_double * 9)(*b.pose_R)
    B.kv = b.servo_gain
    B.rigid_interval = b.rigid_interval
    assert len(b.segments) <= MAX_SEG
    B.nseg = len(b.segments)
    for i, s in enumerate(b.segments):
        B.seg[i].n_steps = s.n_steps
        B.seg[i].cut_id = s.cut_id
        B.seg[i].v = (C.c_double * 3)(*s.v)
        B.seg[i].w = (C.c_double * 3)(*s.omega)
    return B


class OracleScene:
    """One FP64 scene built from a ``bm_inputs.Scene``."""

    FIELDS = {"X": (0, 3), "x": (1, 3), "v": (2, 3), "F": (3, 9), "D": (4, 1),
              "ut": (5, 3), "code": (6, 1), "J": (7, 3), "digits": (8, MAX_CUTS),
              "hist": (9, 4 * HIST)}

    def __init__(self, sc, single_field: bool = False, wrench_capacity: int = 0,
                 _handle=None):
        self._L = lib()
        if _handle is not None:  # a clone of another scene (see clone())
            self.n = sc.n
            self.params, self._blade = sc.params, sc._blade
            self.wrench_capacity = sc.wrench_capacity
            self._h = _handle
            return
        X = _arr(sc.X)
        self.n = sc.n
        self.params = _params(sc, single_field)
        self._blade = _blade(sc.blade) if sc.blade is not None else None
        cap = wrench_capacity if wrench_capacity > 0 else (
            sum(s.n_steps for s in sc.blade.segments) + 16 if sc.blade is not None else 0)
        self.wrench_capacity = cap
        self._h = self._L.or_create(C.byref(self.params),
                                    C.byref(self._blade) if self._blade is not None else None,
                                    self.n, _dp(X), cap)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_destroy(h)
            self._h = None

    def step(self, n: int = 1) -> int:
        return self._L.or_step(self._h, int(n))

    def clone(self) -> "OracleScene":
        """Deep copy of the whole state (a checkpoint)."""
        return OracleScene(self, _handle=self._L.or_clone(self._h))

    def get(self, name: str) -> np.ndarray:
        fid, w = self.FIELDS[name]
        out = np.zeros(self.n * w)
        self._L.or_get(self._h, fid, _dp(out))
        if name == "code":
            return out.astype(np.int64)
        return out.reshape(self.n, w) if w > 1 else out

    def set(self, name: str, value) -> None:
        fid, w = self.FIELDS[name]
        a = _arr(value, self.n * w)
        if self._L.or_set(self._h, fid, _dp(a)) != 0:
            raise ValueError(f"field {name} is read-only")

    def tool(self) -> np.ndarray:
        out = np.zeros(18)
        self._L.or_get_tool(self._h, _dp(out))
        return out

    def set_tool(self, xB, R, vB, wB) -> None:
        a = np.concatenate([_arr(xB, 3), _arr(R, 9), _arr(vB, 3), _arr(wB, 3)])
        self._L.or_set_tool(self._h, _dp(a))

    def frame(self) -> dict:
        out = np.zeros(15)
        self._L.or_get_frame(self._h, _dp(out))
        return {"xe": out[0:3], "n": out[3:6], "e": out[6:9], "d": out[9:12], "ve": out[12:15]}

    def set_step(self, step: int, current_cut: int) -> None:
        """Substep counter and cut in progress, for continuing from a copied state."""
        self._L.or_set_step(self._h, int(step), int(current_cut))

    @property
    def step_count(self) -> int:
        return self._L.or_step_count(self._h)

    @property
    def errors(self) -> int:
        return self._L.or_errors(self._h)

    def cut_planes(self):
        """(planes, mask): planes[k] = (n, n . x_e) of cut k in the world frame
        at the substep the cut began; bit k of mask marks cut k as recorded."""
        out = np.zeros(MAX_CUTS * 4)
        mask = self._L.or_cut_planes(self._h, _dp(out))
        return out.reshape(MAX_CUTS, 4), int(mask)

    def impulse_sum(self) -> np.ndarray:
        out = np.zeros(3)
        self._L.or_impulse_sum(self._h, _dp(out))
        return out

    def last_wrench(self) -> np.ndarray:
        out = np.zeros(6)
        self._L.or_last_wrench(self._h, _dp(out))
        return out

    def wrench_history(self, first: int = 0, count: int | None = None) -> np.ndarray:
        if count is None:
            count = self.step_count - first
        out = np.zeros(6 * count)
        if self._L.or_wrench_history(self._h, first, count, _dp(out)) != 0:
            raise IndexError("wrench history out of range")
        return out.reshape(count, 6)

    def grid_dims(self):
        lo = (C.c_int * 3)()
        dim = (C.c_int * 3)()
        self._L.or_grid_dims(self._h, lo, dim)
        return tuple(lo), tuple(dim)

    def slot_count(self) -> int:
        return self._L.or_slot_count(self._h)

    def momentum(self) -> np.ndarray:
        out = np.zeros(3)
        self._L.or_momentum(self._h, _dp(out))
        return out


# ---------------------------------------------------------------------------
# adjoint (reverse mode) with checkpoints
# ---------------------------------------------------------------------------

class OracleAdjoint:
    """Adjoint state of one scene: x, v, F, u_t adjoints plus the parameter
    accumulators (dL/dmu, dL/dlambda, tool position, segment velocities)."""

    def __init__(self, n: int):
        self._L = lib()
        self.n = n
        self._h = self._L.or_adj_create(n)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_adj_destroy(h)
            self._h = None

    def field(self, name: str) -> np.ndarray:
        which, w = {"x": (0, 3), "v": (1, 3), "F": (2, 9), "ut": (3, 3), "xB": (4, 3)}[name]
        ptr = self._L.or_adj_field(self._h, which)
        return np.ctypeslib.as_array(ptr, shape=(1 if name == "xB" else self.n, w))

    def substep(self, scene: "OracleScene", force_bar) -> None:
        fb = _arr(force_bar, 3)
        if self._L.or_adj_substep(scene._h, self._h, _dp(fb)) != 0:
            raise ValueError("adjoint needs a kinematic translating blade, rigid interval 1 "
                             "and no pair contact")

    def theta(self, scene: "OracleScene") -> dict:
        out = np.zeros(7 + 3 * MAX_SEG)
        self._L.or_adj_theta(self._h, scene._h, _dp(out))
        return {"E": out[0], "nu": out[1], "mu": out[2], "lam": out[3], "xB": out[4:7],
                "v_seg": out[7:].reshape(MAX_SEG, 3)}


def force_loss(forces: np.ndarray, target: np.ndarray) -> float:
    """L = sum_n |F_B^n - F_target^n|^2 over the reaction-force trajectory."""
    return float(np.sum((np.asarray(forces) - np.asarray(target)) ** 2))


def forces(sc, n_steps: int) -> np.ndarray:
    """Reaction-force trajectory F_B^n (Eq. 16), n_steps x 3."""
    o = OracleScene(sc, wrench_capacity=n_steps)
    o.step(n_steps)
    return o.wrench_history(0, n_steps)[:, :3].copy()


def gradient(sc, target: np.ndarray, n_steps: int, every: int = 20) -> dict:
    """Loss and its gradient w.r.t. E, nu and the blade's segment
    velocities, by the FP64 adjoint with a checkpoint every ``every``
    substeps (each checkpoint interval is recomputed forward once)."""
    o = OracleScene(sc, wrench_capacity=n_steps)
    ck = {}
    for k in range(n_steps):
        if k % every == 0:
            ck[k] = o.clone()
        o.step(1)
    F = o.wrench_history(0, n_steps)[:, :3].copy()
    fbar = 2.0 * (F - np.asarray(target))
    adj = OracleAdjoint(sc.n)
    for k0 in sorted(ck, reverse=True):
        k1 = min(k0 + every, n_steps)
        states = []
        t = ck[k0].clone()
        for _ in range(k0, k1):
            states.append(t.clone())
            t.step(1)
        for k in range(k1 - 1, k0 - 1, -1):
            adj.substep(states[k - k0], fbar[k])
        del states, t
    th = adj.theta(o)
    return {"loss": force_loss(F, target), "forces": F, "dE": th["E"], "dnu": th["nu"],
            "dv_seg": th["v_seg"][:len(sc.blade.segments)] if sc.blade else None,
            "dxB0": th["xB"], "adjoint": adj}
