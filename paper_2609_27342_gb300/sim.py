"""Thin Python binding over the C ABI: scenes and batches.

Only argument marshalling lives here; every step of the substep runs in the
library's CUDA kernels.  PyTorch supplies device memory (optionally, through
its caching allocator) and streams.
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

from . import _abi as A


def _d3(v):
    return A.D3(*[float(t) for t in v])


def scene_desc(sc, wrench_history: int = 0) -> A.SceneDesc:
    """C descriptor from a ``bm_inputs.Scene``-like object."""
    d = A.SceneDesc()
    d.E, d.nu, d.rho, d.dx = sc.E, sc.nu, sc.rho, sc.dx
    d.origin = _d3(sc.origin)
    d.V0, d.dt, d.beta = sc.V0, sc.dt, sc.beta
    d.gravity = _d3(sc.gravity)
    d.floor_enabled, d.floor_z = int(sc.floor), sc.floor_z
    d.s_R, d.s_n, d.gamma_k, d.gamma_c = sc.s_R, sc.s_n, sc.gamma_k, sc.gamma_c
    d.pair_contact, d.pair_mu_s, d.pair_mu_d = int(sc.pair_contact), sc.pair_mu_s, sc.pair_mu_d
    d.G_c, d.zeta, d.u_min = sc.G_c, sc.zeta, sc.u_min
    d.b_back, d.b_lead, d.band_half_width = sc.b_back, sc.b_lead, sc.band_half_width
    d.tool_contact = int(sc.tool_contact)
    d.wrench_history = int(wrench_history)
    d.model = {"neo_hookean": A.MODEL_NEO_HOOKEAN, "fixed_corotated": A.MODEL_FIXED_COROTATED}[
        getattr(sc, "model", "neo_hookean")]
    d.yield_stress = float(getattr(sc, "yield_stress", 0.0))
    d.viscosity = float(getattr(sc, "viscosity", 0.0))
    return d


def blade_desc(b) -> A.BladeDesc:
    B = A.BladeDesc()
    B.edge_point, B.normal = _d3(b.edge_point), _d3(b.normal)
    B.edge_dir, B.front_dir = _d3(b.edge_dir), _d3(b.front_dir)
    B.half_length, B.thickness, B.height = b.half_length, b.thickness, b.height
    B.mu_s, B.mu_d, B.mass = b.mu_s, b.mu_d, b.mass
    B.inertia = A.D9(*b.inertia)
    B.pose_x = _d3(b.pose_x)
    B.pose_R = A.D9(*b.pose_R)
    B.servo_gain = b.servo_gain
    B.rigid_interval = b.rigid_interval
    if len(b.segments) > A.MAX_SEGMENTS:
        raise ValueError("too many trajectory segments")
    B.n_segments = len(b.segments)
    for i, s in enumerate(b.segments):
        B.segments[i].n_steps = int(s.n_steps)
        B.segments[i].cut_id = int(s.cut_id)
        B.segments[i].v = _d3(s.v)
        B.segments[i].omega = _d3(s.omega)
    return B


class TorchAllocator:
    """bm_alloc callbacks backed by PyTorch's caching allocator."""

    def __init__(self, device: int = 0):
        import torch
        self._torch = torch
        self.device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              stream or 0))
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._a = A.ALLOC_FN(_alloc)
        self._f = A.FREE_FN(_free)
        self.struct = A.Alloc(self._a, self._f, None)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    h = getattr(stream, "cuda_stream", stream)
    return int(h) if h else None


def _buffer_ptr(buf, nbytes: int):
    """(address, on_device) of a contiguous torch tensor or numpy array of at
    least nbytes bytes."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"] or buf.nbytes < nbytes:
            raise ValueError("buffer must be contiguous and hold the checkpoint")
        return buf.ctypes.data, 0
    if not buf.is_contiguous() or buf.numel() * buf.element_size() < nbytes:
        raise ValueError("buffer must be contiguous and hold the checkpoint")
    return buf.data_ptr(), int(buf.is_cuda)


class Scene:
    """One simulation scene on the GPU (C handle ``bm_scene_t``)."""

    def __init__(self, sc, stream=None, allocator: Optional[TorchAllocator] = None,
                 wrench_history: int = 0):
        self._L = A.load()
        X = np.ascontiguousarray(np.asarray(sc.X, dtype=np.float32))
        self.n = int(X.shape[0])
        self.spec = sc
        self._alloc = allocator
        self._desc = scene_desc(sc, wrench_history)
        h = C.c_void_p()
        A.check(self._L.bm_scene_create(
            C.byref(self._desc), X.ctypes.data_as(C.POINTER(C.c_float)), self.n,
            C.byref(allocator.struct) if allocator is not None else None,
            _stream_handle(stream), C.byref(h)))
        self._h = h
        self.batch = None
        if sc.blade is not None:
            self._blade = blade_desc(sc.blade)
            bid = C.c_int()
            A.check(self._L.bm_add_blade(self._h, C.byref(self._blade), C.byref(bid)))

    @classmethod
    def in_batch(cls, batch: "Batch", sc) -> "Scene":
        """Create the scene directly inside ``batch``'s pools (no device
        allocation of its own); raises BMError(E_CAPACITY) when it does not fit."""
        self = cls.__new__(cls)
        self._L = A.load()
        X = np.ascontiguousarray(np.asarray(sc.X, dtype=np.float32))
        self.n = int(X.shape[0])
        self.spec = sc
        self._alloc = None
        self._desc = scene_desc(sc, 0)
        self._blade = blade_desc(sc.blade) if sc.blade is not None else None
        h = C.c_void_p()
        A.check(self._L.bm_batch_scene_create(
            batch._h, C.byref(self._desc),
            C.byref(self._blade) if self._blade is not None else None,
            X.ctypes.data_as(C.POINTER(C.c_float)), self.n, C.byref(h)))
        self._h = h
        self.batch = batch
        batch.scenes.append(self)
        return self

    @property
    def handle(self):
        return self._h

    # -- checkpoints -------------------------------------------------------
    def checkpoint_size(self) -> int:
        n = C.c_int64()
        A.check(self._L.bm_checkpoint_size(self._h, C.byref(n)))
        return int(n.value)

    def checkpoint(self, out=None, device: bool = True):
        """Complete simulation state in one buffer (bm_checkpoint_save): a
        uint8 torch tensor on the current device, or a host numpy array with
        ``device=False``; ``out`` reuses a buffer of checkpoint_size bytes."""
        nbytes = self.checkpoint_size()
        if out is None:
            if device:
                import torch
                out = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            else:
                out = np.empty(nbytes, dtype=np.uint8)
        ptr, on_dev = _buffer_ptr(out, nbytes)
        A.check(self._L.bm_checkpoint_save(self._h, C.c_void_p(ptr), on_dev))
        return out

    def restore(self, buf) -> None:
        """Restore a checkpoint of this scene (bm_checkpoint_restore)."""
        ptr, on_dev = _buffer_ptr(buf, self.checkpoint_size())
        A.check(self._L.bm_checkpoint_restore(self._h, C.c_void_p(ptr), on_dev))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.bm_scene_destroy(self._h)
            self._h = None
        b = getattr(self, "batch", None)
        if b is not None and self in b.scenes:
            b.scenes.remove(self)
        self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        A.check(self._L.bm_step(self._h, int(n)))

    def set_stop(self, substep: int) -> None:
        """Stop advancing once `substep` substeps are taken (-1: never); the
        scene is then left untouched by later steps, alone or in a batch."""
        A.check(self._L.bm_scene_set_stop(self._h, int(substep)))

    def read(self, *names: str) -> Dict[str, np.ndarray]:
        names = names or ("x", "v")
        order = sorted(names, key=lambda k: A.FIELDS[k][0])
        mask, outs, ptrs = 0, {}, []
        for k in order:
            bit, w, dt = A.FIELDS[k]
            mask |= bit
            a = np.zeros((self.n, w) if w > 1 else (self.n,), dtype=dt)
            outs[k] = a
            ptrs.append(a.ctypes.data)
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        A.check(self._L.bm_read_state(self._h, mask, arr, 0))
        return outs

    def read_noalloc(self, *names: str) -> Dict[str, np.ndarray]:
        """``read`` through the entry point that allocates no device memory
        (fields up to 16 MiB each; see bm_read_state_noalloc)."""
        names = names or ("x", "v")
        order = sorted(names, key=lambda k: A.FIELDS[k][0])
        mask, outs, ptrs = 0, {}, []
        for k in order:
            bit, w, dt = A.FIELDS[k]
            mask |= bit
            a = np.zeros((self.n, w) if w > 1 else (self.n,), dtype=dt)
            outs[k] = a
            ptrs.append(a.ctypes.data)
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        A.check(self._L.bm_read_state_noalloc(self._h, mask, arr))
        return outs

    def read_device(self, fields: Dict[str, "object"]) -> None:
        """Read into device tensors (dict name -> contiguous torch tensor)."""
        order = sorted(fields, key=lambda k: A.FIELDS[k][0])
        mask = 0
        ptrs = []
        for k in order:
            mask |= A.FIELDS[k][0]
            ptrs.append(fields[k].data_ptr())
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        A.check(self._L.bm_read_state(self._h, mask, arr, 1))

    def write(self, **fields) -> None:
        order = sorted(fields, key=lambda k: A.FIELDS[k][0])
        mask, keep, ptrs = 0, [], []
        for k in order:
            bit, w, dt = A.FIELDS[k]
            a = np.ascontiguousarray(np.asarray(fields[k], dtype=dt).reshape(self.n, w) if w > 1
                                     else np.asarray(fields[k], dtype=dt).reshape(self.n))
            mask |= bit
            keep.append(a)
            ptrs.append(a.ctypes.data)
        arr = (C.c_void_p * len(ptrs))(*ptrs)
        A.check(self._L.bm_write_state(self._h, mask, arr, 0))

    def info(self) -> A.SceneInfo:
        out = A.SceneInfo()
        A.check(self._L.bm_scene_info_get(self._h, C.byref(out)))
        return out

    def tool_wrench(self) -> np.ndarray:
        out = np.zeros(6)
        A.check(self._L.bm_tool_wrench(self._h, 0, out.ctypes.data_as(A.PD)))
        return out

    def wrench_history(self, first: int, count: int) -> np.ndarray:
        out = np.zeros((count, 6))
        A.check(self._L.bm_wrench_history(self._h, 0, first, count, out.ctypes.data_as(A.PD)))
        return out

    def set_tool_state(self, xB, R, vB, wB) -> None:
        pose = np.ascontiguousarray(np.concatenate([np.ravel(xB), np.ravel(R)]).astype(np.float64))
        tw = np.ascontiguousarray(np.concatenate([np.ravel(vB), np.ravel(wB)]).astype(np.float64))
        A.check(self._L.bm_set_tool_state(self._h, 0, pose.ctypes.data_as(A.PD),
                                          tw.ctypes.data_as(A.PD)))

    def tool_state(self) -> np.ndarray:
        pose = np.zeros(12)
        tw = np.zeros(6)
        A.check(self._L.bm_get_tool_state(self._h, 0, pose.ctypes.data_as(A.PD),
                                          tw.ctypes.data_as(A.PD)))
        return np.concatenate([pose, tw])


def footprint(sc) -> tuple:
    """(particles, nodes, bricks, bytes) a scene takes in a batch."""
    L = A.load()
    X = np.ascontiguousarray(np.asarray(sc.X, dtype=np.float32))
    d = scene_desc(sc)
    p, nd, br, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    A.check(L.bm_scene_footprint(C.byref(d), X.ctypes.data_as(C.POINTER(C.c_float)), X.shape[0],
                                 C.byref(p), C.byref(nd), C.byref(br), C.byref(b)))
    return p.value, nd.value, br.value, b.value


class Adjoint:
    """Adjoint of the substep for one scene (bm_adjoint_*): state adjoints
    plus accumulated parameter gradients."""

    FIELDS = {"x": (A.FIELD_x, 3), "v": (A.FIELD_v, 3), "F": (A.FIELD_F, 9), "ut": (A.FIELD_UT, 3)}

    def __init__(self, scene: "Scene"):
        self._L = A.load()
        self.scene = scene
        h = C.c_void_p()
        A.check(self._L.bm_adjoint_create(scene.handle, C.byref(h)))
        self._h = h

    def reset(self) -> None:
        A.check(self._L.bm_adjoint_reset(self._h))

    def substep(self, force_bar) -> None:
        """Adjoint of the substep the scene is about to take; force_bar =
        dL/dF_B of that substep's reaction force."""
        fb = (C.c_double * 3)(*[float(t) for t in force_bar])
        A.check(self._L.bm_adjoint_substep(self._h, fb))

    def state(self, *names: str) -> Dict[str, np.ndarray]:
        names = sorted(names, key=lambda k: self.FIELDS[k][0])
        mask, bufs, out = 0, [], {}
        n = self.scene.n
        for k in names:
            bit, w = self.FIELDS[k]
            mask |= bit
            out[k] = np.zeros((n, w), np.float32)
            bufs.append(out[k].ctypes.data)
        arr = (C.c_void_p * len(bufs))(*bufs)
        A.check(self._L.bm_adjoint_state(self._h, mask, arr, 0, 0))
        return out

    def set_state(self, **fields) -> None:
        names = sorted(fields, key=lambda k: self.FIELDS[k][0])
        mask, bufs, keep = 0, [], []
        for k in names:
            bit, w = self.FIELDS[k]
            a = np.ascontiguousarray(np.asarray(fields[k], np.float32).reshape(self.scene.n, w))
            keep.append(a)
            mask |= bit
            bufs.append(a.ctypes.data)
        arr = (C.c_void_p * len(bufs))(*bufs)
        A.check(self._L.bm_adjoint_state(self._h, mask, arr, 0, 1))

    def params(self) -> dict:
        out = (C.c_double * (7 + 3 * A.MAX_SEGMENTS))()
        A.check(self._L.bm_adjoint_params(self._h, out, len(out)))
        a = np.array(out[:])
        return {"E": a[0], "nu": a[1], "mu": a[2], "lam": a[3], "xB": a[4:7],
                "v_seg": a[7:].reshape(A.MAX_SEGMENTS, 3)}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.bm_adjoint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Packed pools holding many scenes, stepped by CUDA-graph launches."""

    def __init__(self, max_particles: int, max_nodes: int, max_scenes: int,
                 max_slots: int = 0, max_bricks: int = 0, graph_chunk: int = 16,
                 node_tile: int = 128, pair_contact: bool = False, stream=None,
                 allocator: Optional[TorchAllocator] = None):
        self._L = A.load()
        d = A.BatchDesc(int(max_particles), int(max_nodes), int(max_slots), int(max_bricks),
                        int(max_scenes), int(graph_chunk), int(node_tile), int(pair_contact))
        h = C.c_void_p()
        self._alloc = allocator
        A.check(self._L.bm_batch_create(C.byref(d),
                                        C.byref(allocator.struct) if allocator else None,
                                        _stream_handle(stream), C.byref(h)))
        self._h = h
        self.scenes: List[Scene] = []

    def add(self, s: Scene) -> None:
        A.check(self._L.bm_batch_add(self._h, s.handle))
        s.batch = self
        self.scenes.append(s)

    def remove(self, s: Scene) -> None:
        A.check(self._L.bm_batch_remove(self._h, s.handle))
        s.batch = None
        self.scenes.remove(s)

    def step(self, n: int = 1) -> None:
        A.check(self._L.bm_batch_step(self._h, int(n)))

    def set_tiles(self, graph_chunk: int, node_tile: int, brick_variant: int = 0) -> None:
        """Launch shape of later steps; see bm_batch_set_tiles (results do not
        depend on it)."""
        A.check(self._L.bm_batch_set_tiles(self._h, int(graph_chunk), int(node_tile),
                                           int(brick_variant)))

    def members(self) -> list:
        n = self._L.bm_batch_members(self._h, None, 0)
        arr = (C.c_void_p * max(n, 1))()
        self._L.bm_batch_members(self._h, arr, n)
        return [arr[i] for i in range(n)]

    def set_tool_states(self, states: np.ndarray) -> None:
        st = np.ascontiguousarray(states, dtype=np.float64)
        A.check(self._L.bm_batch_set_tool_states(self._h, st.ctypes.data_as(A.PD), st.shape[0], 0))

    def set_tool_states_ptr(self, ptr: int, n: int, on_device: bool) -> None:
        A.check(self._L.bm_batch_set_tool_states(self._h, C.cast(ptr, A.PD), n, int(on_device)))

    def tool_wrenches(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        n = len(self.scenes)
        out = np.zeros((n, 6)) if out is None else out
        A.check(self._L.bm_batch_tool_wrenches(self._h, out.ctypes.data_as(A.PD), n, 0))
        return out

    def tool_wrenches_ptr(self, ptr: int, n: int, on_device: bool) -> None:
        A.check(self._L.bm_batch_tool_wrenches(self._h, C.cast(ptr, A.PD), n, int(on_device)))

    def profile(self, n: int) -> Dict[str, tuple]:
        """Per-kernel (total ms, launches) over n eager substeps (CUDA events)."""
        ms = (C.c_double * 32)()
        cnt = (C.c_int * 32)()
        k = A.check(self._L.bm_batch_profile(self._h, int(n), ms, cnt, 32))
        return {self._L.bm_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(k)}

    def errors(self) -> int:
        b = C.c_uint32()
        A.check(self._L.bm_batch_errors(self._h, C.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            for s in list(self.scenes):
                s.close()
            self.scenes = []
            self._L.bm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
