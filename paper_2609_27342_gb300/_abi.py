"""ctypes declarations of the C ABI in include/blademaster.h.

Argument marshalling only.  Loading fails loudly when the shared library has
not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

MAX_CUTS = 32
MAX_SEGMENTS = 16

OK = 0
E_INVALID, E_OOM, E_CUDA, E_SLOT_OVERFLOW = -1, -2, -3, -4
E_INVERTED, E_NONFINITE, E_CONTACT_OVERFLOW, E_TIMEOUT = -5, -6, -7, -8
E_TOO_MANY_CUTS, E_CAPACITY = -9, -10

ERRBIT_SLOT_OVERFLOW = 1
ERRBIT_INVERTED = 2
ERRBIT_NONFINITE = 4
ERRBIT_CONTACT_OVERFLOW = 8
ERRBIT_TOO_MANY_CUTS = 16

MODEL_NEO_HOOKEAN, MODEL_FIXED_COROTATED = 0, 1

FIELD_X, FIELD_x, FIELD_v, FIELD_F, FIELD_D = 1, 2, 4, 8, 16
FIELD_UT, FIELD_CODE, FIELD_MASK1, FIELD_MASK2 = 32, 64, 128, 256
FIELD_PAIR_PARTNER, FIELD_PAIR_U = 512, 1024
PAIR_HIST = 16

# name -> (bit, components, numpy dtype)
FIELDS = {
    "X": (FIELD_X, 3, "float32"), "x": (FIELD_x, 3, "float32"), "v": (FIELD_v, 3, "float32"),
    "F": (FIELD_F, 9, "float32"), "D": (FIELD_D, 1, "float32"), "ut": (FIELD_UT, 3, "float32"),
    "code": (FIELD_CODE, 1, "int64"), "mask1": (FIELD_MASK1, 1, "uint32"),
    "mask2": (FIELD_MASK2, 1, "uint32"),
    "pair_partner": (FIELD_PAIR_PARTNER, PAIR_HIST, "int32"),
    "pair_u": (FIELD_PAIR_U, 3 * PAIR_HIST, "float32"),
}

D3 = C.c_double * 3
D9 = C.c_double * 9


class SceneDesc(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double), ("dx", C.c_double),
                ("origin", D3), ("V0", C.c_double), ("dt", C.c_double), ("beta", C.c_double),
                ("gravity", D3), ("floor_enabled", C.c_int), ("floor_z", C.c_double),
                ("s_R", C.c_double), ("s_n", C.c_double), ("gamma_k", C.c_double),
                ("gamma_c", C.c_double), ("pair_contact", C.c_int), ("pair_mu_s", C.c_double),
                ("pair_mu_d", C.c_double), ("G_c", C.c_double), ("zeta", C.c_double),
                ("u_min", C.c_double), ("b_back", C.c_double), ("b_lead", C.c_double),
                ("band_half_width", C.c_double), ("tool_contact", C.c_int),
                ("wrench_history", C.c_int), ("model", C.c_int), ("yield_stress", C.c_double),
                ("viscosity", C.c_double)]


class Segment(C.Structure):
    _fields_ = [("n_steps", C.c_int), ("cut_id", C.c_int), ("v", D3), ("omega", D3)]


class BladeDesc(C.Structure):
    _fields_ = [("edge_point", D3), ("normal", D3), ("edge_dir", D3), ("front_dir", D3),
                ("half_length", C.c_double), ("thickness", C.c_double), ("height", C.c_double),
                ("mu_s", C.c_double), ("mu_d", C.c_double), ("mass", C.c_double),
                ("inertia", D9), ("pose_x", D3), ("pose_R", D9), ("servo_gain", C.c_double),
                ("rigid_interval", C.c_int), ("n_segments", C.c_int),
                ("segments", Segment * MAX_SEGMENTS)]


class SceneInfo(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("n_nodes", C.c_int64), ("n_slots", C.c_int64),
                ("slot_capacity", C.c_int64), ("step", C.c_int64), ("error_bits", C.c_uint32),
                ("grid_lo", C.c_int * 3), ("grid_dim", C.c_int * 3), ("current_cut", C.c_int32),
                ("contact_list_builds", C.c_int64)]


class BatchDesc(C.Structure):
    _fields_ = [("max_particles", C.c_int64), ("max_nodes", C.c_int64), ("max_slots", C.c_int64),
                ("max_bricks", C.c_int64), ("max_scenes", C.c_int), ("graph_chunk", C.c_int),
                ("node_tile", C.c_int), ("pair_contact", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Alloc(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


# every entry point the header declares, with its signature
VP = C.c_void_p
PVP = C.POINTER(C.c_void_p)
PD = C.POINTER(C.c_double)
SIGNATURES = {
    "bm_scene_create": (C.c_int, [C.POINTER(SceneDesc), C.POINTER(C.c_float), C.c_int64,
                                  C.POINTER(Alloc), VP, PVP]),
    "bm_add_blade": (C.c_int, [VP, C.POINTER(BladeDesc), C.POINTER(C.c_int)]),
    "bm_set_tool_state": (C.c_int, [VP, C.c_int, PD, PD]),
    "bm_get_tool_state": (C.c_int, [VP, C.c_int, PD, PD]),
    "bm_step": (C.c_int, [VP, C.c_int]),
    "bm_scene_set_stop": (C.c_int, [VP, C.c_int64]),
    "bm_read_state": (C.c_int, [VP, C.c_uint32, PVP, C.c_int]),
    "bm_write_state": (C.c_int, [VP, C.c_uint32, PVP, C.c_int]),
    "bm_read_state_noalloc": (C.c_int, [VP, C.c_uint32, PVP]),
    "bm_tool_wrench": (C.c_int, [VP, C.c_int, PD]),
    "bm_wrench_history": (C.c_int, [VP, C.c_int, C.c_int64, C.c_int64, PD]),
    "bm_scene_info_get": (C.c_int, [VP, C.POINTER(SceneInfo)]),
    "bm_checkpoint_size": (C.c_int, [VP, C.POINTER(C.c_int64)]),
    "bm_checkpoint_save": (C.c_int, [VP, VP, C.c_int]),
    "bm_checkpoint_restore": (C.c_int, [VP, VP, C.c_int]),
    "bm_adjoint_create": (C.c_int, [VP, PVP]),
    "bm_adjoint_reset": (C.c_int, [VP]),
    "bm_adjoint_substep": (C.c_int, [VP, PD]),
    "bm_adjoint_state": (C.c_int, [VP, C.c_uint32, PVP, C.c_int, C.c_int]),
    "bm_adjoint_params": (C.c_int, [VP, PD, C.c_int]),
    "bm_adjoint_destroy": (C.c_int, [VP]),
    "bm_surface_create": (C.c_int, [VP, C.POINTER(C.c_int), PVP]),
    "bm_surface_update": (C.c_int, [VP, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "bm_surface_read": (C.c_int, [VP, VP, VP, VP, VP, C.c_int]),
    "bm_surface_destroy": (C.c_int, [VP]),
    "bm_fp32_fma_peak": (C.c_int, [VP, PD]),
    "bm_scene_destroy": (C.c_int, [VP]),
    "bm_batch_create": (C.c_int, [C.POINTER(BatchDesc), C.POINTER(Alloc), VP, PVP]),
    "bm_batch_scene_create": (C.c_int, [VP, C.POINTER(SceneDesc), C.POINTER(BladeDesc),
                                        C.POINTER(C.c_float), C.c_int64, PVP]),
    "bm_batch_add": (C.c_int, [VP, VP]),
    "bm_batch_remove": (C.c_int, [VP, VP]),
    "bm_batch_step": (C.c_int, [VP, C.c_int]),
    "bm_scene_footprint": (C.c_int, [C.POINTER(SceneDesc), C.POINTER(C.c_float), C.c_int64,
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "bm_batch_set_tool_states": (C.c_int, [VP, PD, C.c_int, C.c_int]),
    "bm_batch_tool_wrenches": (C.c_int, [VP, PD, C.c_int, C.c_int]),
    "bm_batch_members": (C.c_int, [VP, PVP, C.c_int]),
    "bm_batch_errors": (C.c_int, [VP, C.POINTER(C.c_uint32)]),
    "bm_batch_set_tiles": (C.c_int, [VP, C.c_int, C.c_int, C.c_int]),
    "bm_batch_destroy": (C.c_int, [VP]),
    "bm_batch_profile": (C.c_int, [VP, C.c_int, PD, C.POINTER(C.c_int), C.c_int]),
    "bm_kernel_name": (C.c_char_p, [C.c_int]),
    "bm_last_error": (C.c_char_p, []),
    "bm_version": (C.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


class BMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"blademaster error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the shared library (raises if it is missing and not built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise ImportError(
                        f"libblademaster.so not built ({path}); run "
                        "`python -c 'import __graft_entry__ as g; g.build()'`")
                _build.build()
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(rc: int) -> int:
    if rc < 0:
        msg = load().bm_last_error()
        raise BMError(rc, msg.decode() if msg else "")
    return rc
