"""Reference-grid surface of a scene (Sec. III-F), reconstructed by the
library's CUDA kernels (bm_surface_*): links of the sub-cell particle lattice
disconnected where the side codes conflict, one dual-contouring vertex per
local region, quads around every link with Hermite data, and the side-aware
trilinear embedding that moves each vertex with its own side's logical grid.
Output goes to a headless device or host buffer (optionally an OBJ file);
the reconstruction never feeds back into the simulation.
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, Tuple

import numpy as np

from . import _abi as A
from .sim import Scene


class Surface:
    """Surface of one scene (plain or batched).  ``lattice`` is the number of
    particles per reference cell along each axis (2, 2, 2 for 8 per cell)."""

    def __init__(self, scene: Scene, lattice=(2, 2, 2)):
        self._L = A.load()
        self.scene = scene
        k = (C.c_int * 3)(*[int(t) for t in lattice])
        h = C.c_void_p()
        A.check(self._L.bm_surface_create(scene.handle, k, C.byref(h)))
        self._h = h
        self.n_vertices = 0
        self.n_triangles = 0

    def update(self, rebuild: bool = True) -> Tuple[int, int]:
        """Rebuild the topology from the current codes (``rebuild``) and
        re-embed the vertices in the current motion field."""
        nv, nt = C.c_int64(), C.c_int64()
        A.check(self._L.bm_surface_update(self._h, int(bool(rebuild)), C.byref(nv), C.byref(nt)))
        self.n_vertices, self.n_triangles = nv.value, nt.value
        return self.n_vertices, self.n_triangles

    def read(self) -> Dict[str, np.ndarray]:
        """Host copies of the last update: vertices (current positions),
        reference (reference positions), triangles, masks (s1, s2 per vertex)."""
        nv, nt = self.n_vertices, self.n_triangles
        out = {"vertices": np.zeros((nv, 3), np.float32), "reference": np.zeros((nv, 3), np.float32),
               "triangles": np.zeros((nt, 3), np.int32), "masks": np.zeros((nv, 2), np.uint32)}
        A.check(self._L.bm_surface_read(self._h, out["vertices"].ctypes.data, out["reference"].ctypes.data,
                                        out["triangles"].ctypes.data, out["masks"].ctypes.data, 0))
        return out

    def read_into(self, vertices=None, triangles=None) -> None:
        """Device-to-device copy into caller buffers (e.g. CUDA tensors of
        shape (n_vertices, 3) float32 and (n_triangles, 3) int32)."""
        A.check(self._L.bm_surface_read(self._h, _ptr(vertices), None, _ptr(triangles), None, 1))

    def write_obj(self, path: str) -> None:
        d = self.read()
        with open(path, "w") as fh:
            for v in d["vertices"]:
                fh.write(f"v {v[0]:.7g} {v[1]:.7g} {v[2]:.7g}\n")
            for t in d["triangles"]:
                fh.write(f"f {t[0] + 1} {t[1] + 1} {t[2] + 1}\n")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.bm_surface_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    if t is None:
        return None
    return t.data_ptr() if hasattr(t, "data_ptr") else t.ctypes.data
