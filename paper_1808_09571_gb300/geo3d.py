"""Python binding of the geo3d C ABI (include/geo3d.h).

Argument marshalling only: every step of distance / intersects runs in the
CUDA library.  Arrays may be numpy arrays (host) or torch tensors (host or
CUDA); torch supplies device memory and streams.  If the library cannot be
loaded, every entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

G3D_OK = 0
ERRORS = {
    -1: "G3D_ERR_INVALID_ARG", -2: "G3D_ERR_NAN_INPUT", -3: "G3D_ERR_INDEX_OOB",
    -4: "G3D_ERR_EMPTY_MESH", -5: "G3D_ERR_OOM", -6: "G3D_ERR_CAND_OVERFLOW",
    -7: "G3D_ERR_TIMEOUT", -8: "G3D_ERR_CUDA", -9: "G3D_ERR_RANGE", -10: "G3D_ERR_NO_BVH",
    -11: "G3D_ERR_TOO_LARGE",
    -12: "G3D_ERR_IO",
}
G3D_F32, G3D_F64 = 0, 1
OP_DISTANCE, OP_INTERSECTS = 0, 1


class G3DError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({code})")


class g3d_config(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("warps_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("stack_depth", C.c_int32), ("cand_capacity", C.c_int32), ("queue_capacity", C.c_int32),
                ("time_limit_ms", C.c_int32), ("isect_first", C.c_int32), ("morton_bits", C.c_int32),
                ("traversal", C.c_int32), ("count_visits", C.c_int32), ("frontier_capacity", C.c_int32),
                ("dives", C.c_int32), ("chunk_mfaces", C.c_int32), ("proposal_min_faces", C.c_int32),
                ("reserved", C.c_int32)]


class g3d_query(C.Structure):
    _fields_ = [("a", C.c_int64), ("b", C.c_int64), ("op", C.c_int32), ("pad", C.c_int32)]


class g3d_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "node_pairs", "leaf_pairs", "tri_prefilter", "tri_tests", "candidates", "fp64_tests",
        "exact_tests", "exact_orients", "queue_pushes", "second_passes", "launches", "warp_busy_ns",
        "warp_idle_ns", "seed_excess_ppm", "seed_queries", "distinct_nodes", "distinct_faces",
        "levels", "frontier_blocks")]


class g3d_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_uint64), ("total_ms", C.c_double), ("max_ms", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libgeo3d.so (building it in-tree first if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libgeo3d.so is not built; call paper_1808_09571_gb300.build()")
    L = C.CDLL(_build.LIB)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.g3d_create.argtypes = [C.POINTER(vp), i32, C.POINTER(g3d_config)]
    L.g3d_destroy.argtypes = [vp]
    L.g3d_mesh_load.argtypes = [vp, vp, i32, i64, vp, i64, i32, C.POINTER(i64), vp]
    L.g3d_mesh_build_bvh.argtypes = [vp, i64, vp]
    L.g3d_mesh_load_many.argtypes = [vp, i64, C.POINTER(vp), C.POINTER(C.c_int32), C.POINTER(i64), C.POINTER(vp),
                                     C.POINTER(i64), i32, C.POINTER(i64), C.POINTER(C.c_int32), vp]
    L.g3d_mesh_build_bvh_many.argtypes = [vp, i64, C.POINTER(i64), vp]
    L.g3d_mesh_free.argtypes = [vp, i64]
    L.g3d_mesh_free_many.argtypes = [vp, i64, C.POINTER(i64)]
    L.g3d_mesh_free_many_async.argtypes = [vp, i64, C.POINTER(i64), vp]
    L.g3d_mesh_size.argtypes = [vp, i64, C.POINTER(i64)]
    L.g3d_mesh_export.argtypes = [vp, i64, vp, vp, vp, C.POINTER(i64)]
    L.g3d_distance.argtypes = [vp, i64, i64, vp, vp]
    L.g3d_intersects.argtypes = [vp, i64, i64, vp, vp]
    L.g3d_batch.argtypes = [vp, C.POINTER(g3d_query), i64, vp, vp, vp, vp]
    L.g3d_sync.argtypes = [vp, vp]
    L.g3d_batch_ex.argtypes = [vp, C.POINTER(g3d_query), i64, vp, vp, vp, vp, vp]
    L.g3d_autotune.argtypes = [vp, C.POINTER(g3d_query), i64, i32, i32, C.POINTER(g3d_config), vp]
    L.g3d_volume.argtypes = [vp, i64, vp, vp]
    L.g3d_volume_many.argtypes = [vp, i64, C.POINTER(i64), vp, vp]
    L.g3d_segments.argtypes = [vp, i64, vp, i64, i32, vp, vp, vp, vp]
    L.g3d_batch_hint.argtypes = [vp, C.POINTER(g3d_query), i64, vp, vp, vp, vp, vp, vp]
    L.g3d_mlp_num_params.argtypes = []
    L.g3d_mlp_num_params.restype = C.c_int64
    L.g3d_mlp_create.argtypes = [vp, C.POINTER(vp)]
    L.g3d_mlp_destroy.argtypes = [vp, vp]
    L.g3d_mlp_set_params.argtypes = [vp, vp, vp]
    L.g3d_mlp_get_params.argtypes = [vp, vp, vp]
    L.g3d_mlp_save.argtypes = [vp, vp, C.c_char_p]
    L.g3d_mlp_train.argtypes = [vp, vp, vp, vp, i64, i64, i32, C.c_float, C.c_uint64, vp, vp]
    L.g3d_mlp_load.argtypes = [vp, vp, C.c_char_p]
    L.g3d_mlp_forward.argtypes = [vp, vp, vp, i64, vp, vp]
    L.g3d_mlp_gradients.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
    L.g3d_mlp_train_step.argtypes = [vp, vp, vp, vp, i64, C.c_float, vp, vp]
    L.g3d_pair_features.argtypes = [vp, C.POINTER(g3d_query), i64, vp, vp]
    L.g3d_set_proposal.argtypes = [vp, vp]
    L.g3d_proposal_topk.argtypes = [vp, vp, i64, i32, i32, vp, vp]
    L.g3d_level_trace.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_int), vp]
    L.g3d_plan_create.argtypes = [vp, C.POINTER(g3d_query), i64, vp, vp, vp, C.POINTER(vp), vp]
    L.g3d_plan_launch.argtypes = [vp, vp, vp]
    L.g3d_plan_destroy.argtypes = [vp, vp]
    L.g3d_stats_get.argtypes = [vp, C.POINTER(g3d_stats), vp]
    L.g3d_stats_reset.argtypes = [vp, vp]
    L.g3d_get_config.argtypes = [vp, C.POINTER(g3d_config)]
    L.g3d_set_config.argtypes = [vp, C.POINTER(g3d_config)]
    L.g3d_debug_words.argtypes = [vp, C.POINTER(C.c_int)]
    L.g3d_profile_begin.argtypes = [vp, C.c_char_p]
    L.g3d_profile_end.argtypes = [vp, C.POINTER(g3d_kernel_time), i32, C.POINTER(i32)]
    L.g3d_strerror.argtypes = [i32]
    L.g3d_strerror.restype = C.c_char_p
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != G3D_OK:
        raise G3DError(rc, what)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


_TORCH = None  # the torch module once imported (torch is optional for numpy callers)
_TORCH_DTYPES = {}  # torch dtype -> name


def _torch():
    global _TORCH
    if _TORCH is None:
        try:
            import torch
            _TORCH = torch
        except ImportError:
            _TORCH = False
    return _TORCH


def _ptr_of(x, dtype=None):
    """(pointer, keepalive, dtype-name, nrows) of a numpy array or torch tensor."""
    torch = _torch()
    if torch and isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            x = x.contiguous()
        name = _TORCH_DTYPES.get(x.dtype)
        if name is None:
            name = _TORCH_DTYPES.setdefault(x.dtype, str(x.dtype).replace("torch.", ""))
        return x.data_ptr(), x, name, x.shape[0]
    a = np.ascontiguousarray(x if dtype is None else np.asarray(x, dtype=dtype))
    return a.ctypes.data, a, str(a.dtype), a.shape[0]


def _handles(ms):
    """(ctypes int64 pointer, count, keepalive) of a list of Mesh or an array of handles."""
    if isinstance(ms, np.ndarray):
        a = np.ascontiguousarray(ms, np.int64)
    else:
        a = np.fromiter((m.handle for m in ms), np.int64, len(ms))
    return a.ctypes.data_as(C.POINTER(C.c_int64)), len(a), a


class Mesh:
    """A loaded mesh: its library handle and face count (slots only: calls
    that load tens of thousands of meshes create one per mesh)."""
    __slots__ = ("handle", "nt")

    def __init__(self, handle: int, nt: int):
        self.handle = handle
        self.nt = nt

    def __eq__(self, other):
        return isinstance(other, Mesh) and self.handle == other.handle and self.nt == other.nt

    __hash__ = None

    def __repr__(self):
        return f"Mesh(handle={self.handle}, nt={self.nt})"


class Context:
    """A geo3d context on one CUDA device (g3d_create)."""

    def __init__(self, device: int = 0, leaf_size: int = 0, warps_per_cta: int = 0, ctas_per_sm: int = 0,
                 stack_depth: int = 0, cand_capacity: int = 0, queue_capacity: int = 0,
                 time_limit_ms: int = 0, isect_first: int = 0, morton_bits: int = 0, traversal: int = 0,
                 count_visits: int = 0, frontier_capacity: int = 0, dives: int = 0, chunk_mfaces: int = 0,
                 proposal_min_faces: int = 0):
        self.lib = load()
        cfg = g3d_config(leaf_size, warps_per_cta, ctas_per_sm, stack_depth, cand_capacity, queue_capacity,
                         time_limit_ms, isect_first, morton_bits, traversal, count_visits, frontier_capacity, dives,
                         chunk_mfaces, proposal_min_faces)
        h = C.c_void_p()
        _check(self.lib.g3d_create(C.byref(h), device, C.byref(cfg)), "g3d_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.g3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def config(self) -> dict:
        c = g3d_config()
        _check(self.lib.g3d_get_config(self.h, C.byref(c)), "g3d_get_config")
        return {f: getattr(c, f) for f, _ in g3d_config._fields_ if f != "reserved"}

    def save_config(self, path: str):
        """The current configuration (e.g. as chosen by the autotuner) as JSON."""
        import json
        with open(path, "w") as f:
            json.dump(self.config(), f, indent=1)

    def load_config(self, path: str) -> dict:
        """Apply a configuration saved by save_config (g3d_set_config)."""
        import json
        with open(path) as f:
            cfg = json.load(f)
        return self.set_config(**{k: v for k, v in cfg.items()
                                  if k not in ("cand_capacity", "queue_capacity", "frontier_capacity")})

    def set_config(self, **changes) -> dict:
        """g3d_set_config with the given fields changed; returns the new configuration."""
        cur = self.config()
        cur.update(changes)
        c = g3d_config(*[cur[f] for f, _ in g3d_config._fields_ if f != "reserved"])
        _check(self.lib.g3d_set_config(self.h, C.byref(c)), "g3d_set_config")
        return self.config()

    # -- meshes ---------------------------------------------------------------
    def mesh_load(self, V, I, copy_fp64_master: bool = True, stream=None) -> Mesh:
        vp, vkeep, vdt, nv = _ptr_of(V)
        if vdt not in ("float32", "float64"):
            vp, vkeep, vdt, nv = _ptr_of(np.asarray(V, np.float64))
        ip, ikeep, idt, nt = _ptr_of(I)
        if idt not in ("uint32", "int32"):
            ip, ikeep, idt, nt = _ptr_of(np.asarray(I, np.uint32))
        out = C.c_int64()
        rc = self.lib.g3d_mesh_load(self.h, C.c_void_p(vp), G3D_F32 if vdt == "float32" else G3D_F64, nv,
                                    C.c_void_p(ip), nt, int(copy_fp64_master), C.byref(out), _stream_ptr(stream))
        _check(rc, "g3d_mesh_load")
        return Mesh(out.value, nt)

    def mesh_load_many(self, meshes, copy_fp64_master: bool = True, stream=None) -> list:
        """Load [(V, I), ...] together (g3d_mesh_load_many)."""
        n = len(meshes)
        torch = _torch()
        Vs = [m[0] for m in meshes]
        Is = [m[1] for m in meshes]
        fast = False
        if torch and n:
            T = torch.Tensor
            f32, f64, i32 = torch.float32, torch.float64, torch.int32
            fast = all(type(v) is T and (v.dtype is f32 or v.dtype is f64) and v.is_contiguous() for v in Vs) and \
                all(type(i) is T and i.dtype is i32 and i.is_contiguous() for i in Is)
        if fast:  # lists of contiguous torch tensors: no per-element conversion
            keep = (Vs, Is)
            vl = [v.data_ptr() for v in Vs]
            dl = [G3D_F32 if v.dtype is f32 else G3D_F64 for v in Vs]
            nvl = [v.shape[0] for v in Vs]
            il = [i.data_ptr() for i in Is]
            ntl = [i.shape[0] for i in Is]
        else:
            keep, vl, dl, nvl, il, ntl = [], [], [], [], [], []
            for V, I in meshes:
                vp, vk, vdt, nv = _ptr_of(V)
                if vdt != "float32" and vdt != "float64":
                    vp, vk, vdt, nv = _ptr_of(np.asarray(V, np.float64))
                ip, ik, idt, nt = _ptr_of(I)
                if idt != "int32" and idt != "uint32":
                    ip, ik, idt, nt = _ptr_of(np.asarray(I, np.uint32))
                keep.append(vk)
                keep.append(ik)
                vl.append(vp)
                dl.append(G3D_F32 if vdt == "float32" else G3D_F64)
                nvl.append(nv)
                il.append(ip)
                ntl.append(nt)
        vps, dts, nvs = (C.c_void_p * n)(*vl), (C.c_int32 * n)(*dl), (C.c_int64 * n)(*nvl)
        ips, nts = (C.c_void_p * n)(*il), (C.c_int64 * n)(*ntl)
        out = (C.c_int64 * n)()
        st = (C.c_int32 * n)()
        rc = self.lib.g3d_mesh_load_many(self.h, n, vps, dts, nvs, ips, nts, int(copy_fp64_master), out, st,
                                         _stream_ptr(stream))
        _check(rc, "g3d_mesh_load_many")
        return [Mesh(h, t) for h, t in zip(out, ntl)]

    def mesh_load_arrays(self, vptr, vdtype, nv, iptr, nt, copy_fp64_master: bool = True, stream=None):
        """g3d_mesh_load_many on meshes described by arrays, with no per-mesh
        Python work: vptr / iptr the (device or host) addresses of each mesh's
        vertices and indices (uint32 triples), vdtype G3D_F32 / G3D_F64, nv
        and nt the vertex and face counts.  The caller keeps that memory
        alive until the call returns.  Returns the handles (int64 array)."""
        n = len(vptr)
        vp = np.ascontiguousarray(vptr, np.uint64)
        ip = np.ascontiguousarray(iptr, np.uint64)
        dt = np.ascontiguousarray(vdtype, np.int32)
        nva = np.ascontiguousarray(nv, np.int64)
        nta = np.ascontiguousarray(nt, np.int64)
        out = np.zeros(n, np.int64)
        st = np.zeros(n, np.int32)
        P = C.POINTER
        rc = self.lib.g3d_mesh_load_many(self.h, n, vp.ctypes.data_as(P(C.c_void_p)), dt.ctypes.data_as(P(C.c_int32)),
                                         nva.ctypes.data_as(P(C.c_int64)), ip.ctypes.data_as(P(C.c_void_p)),
                                         nta.ctypes.data_as(P(C.c_int64)), int(copy_fp64_master),
                                         out.ctypes.data_as(P(C.c_int64)), st.ctypes.data_as(P(C.c_int32)),
                                         _stream_ptr(stream))
        _check(rc, "g3d_mesh_load_many")
        return out

    def mesh_build_bvh_many(self, ms, stream=None):
        """Build the BVHs of a list of Mesh, or of an int64 array of handles."""
        arr, n, _k = _handles(ms)
        _check(self.lib.g3d_mesh_build_bvh_many(self.h, n, arr, _stream_ptr(stream)), "g3d_mesh_build_bvh_many")

    def mesh_build_bvh(self, m: Mesh, stream=None):
        _check(self.lib.g3d_mesh_build_bvh(self.h, m.handle, _stream_ptr(stream)), "g3d_mesh_build_bvh")

    def mesh_free(self, m: Mesh):
        _check(self.lib.g3d_mesh_free(self.h, m.handle), "g3d_mesh_free")

    def mesh_export(self, mesh: Mesh) -> dict:
        """The BVH of a built mesh on the host (g3d_mesh_export): face_ids
        (input face id per face in BVH order), leaf_lo / leaf_hi [nleaf, 3],
        leaf_first / leaf_count, node_lo / node_hi [nleaf-1, 2, 3] (the two
        children's boxes), node_child [nleaf-1, 2] (>= 0 internal, < 0 leaf
        ~ref), node_below [nleaf-1, 2] (leaves below each child)."""
        nl = C.c_int64()
        _check(self.lib.g3d_mesh_export(self.h, mesh.handle, None, None, None, C.byref(nl)), "g3d_mesh_export")
        nleaf = nl.value
        ids = np.empty(mesh.nt, np.int32)
        lv = np.empty((nleaf, 8), np.float32)
        nd = np.empty((max(nleaf - 1, 0), 16), np.float32)
        _check(self.lib.g3d_mesh_export(self.h, mesh.handle, C.c_void_p(ids.ctypes.data), C.c_void_p(lv.ctypes.data),
                                        C.c_void_p(nd.ctypes.data) if nleaf > 1 else None, C.byref(nl)),
               "g3d_mesh_export")
        nd4 = nd.reshape(-1, 2, 8)
        return {"face_ids": ids, "leaf_lo": lv[:, 0:3], "leaf_hi": lv[:, 4:7],
                "leaf_first": lv[:, 3].view(np.int32), "leaf_count": lv[:, 7].view(np.int32),
                "node_lo": nd4[:, :, 0:3], "node_hi": nd4[:, :, 4:7],
                "node_child": np.ascontiguousarray(nd4[:, :, 3]).view(np.int32),
                "node_below": np.ascontiguousarray(nd4[:, :, 7]).view(np.int32)}

    def mesh_free_many(self, ms):
        """Free a list of Mesh, or an int64 array of handles."""
        arr, n, _k = _handles(ms)
        _check(self.lib.g3d_mesh_free_many(self.h, n, arr), "g3d_mesh_free_many")

    def mesh_free_many_async(self, ms, stream=None):
        """Stream-ordered release (g3d_mesh_free_many_async) of a list of Mesh or an array of handles."""
        arr, n, _k = _handles(ms)
        _check(self.lib.g3d_mesh_free_many_async(self.h, n, arr, _stream_ptr(stream)), "g3d_mesh_free_many_async")

    def load_and_build(self, V, I, copy_fp64_master: bool = True, stream=None) -> Mesh:
        m = self.mesh_load(V, I, copy_fp64_master, stream)
        self.mesh_build_bvh(m, stream)
        return m

    # -- queries --------------------------------------------------------------
    def distance(self, a: Mesh, b: Mesh, out=None, stream=None, sync: bool = True):
        """3D distance (g3d_distance).  Without `out`, waits and returns a float."""
        if out is None:
            buf = np.full(1, np.nan)
            _check(self.lib.g3d_distance(self.h, a.handle, b.handle, C.c_void_p(buf.ctypes.data),
                                         _stream_ptr(stream)), "g3d_distance")
            self.sync(stream)
            return float(buf[0])
        p, _, _, _ = _ptr_of(out)
        _check(self.lib.g3d_distance(self.h, a.handle, b.handle, C.c_void_p(p), _stream_ptr(stream)), "g3d_distance")
        if sync:
            self.sync(stream)
        return out

    def intersects(self, a: Mesh, b: Mesh, out=None, stream=None, sync: bool = True):
        """3D intersection (g3d_intersects).  Without `out`, waits and returns a bool."""
        if out is None:
            buf = np.full(1, 0xFF, np.uint8)
            _check(self.lib.g3d_intersects(self.h, a.handle, b.handle, C.c_void_p(buf.ctypes.data),
                                           _stream_ptr(stream)), "g3d_intersects")
            self.sync(stream)
            return bool(buf[0])
        p, _, _, _ = _ptr_of(out)
        _check(self.lib.g3d_intersects(self.h, a.handle, b.handle, C.c_void_p(p), _stream_ptr(stream)),
               "g3d_intersects")
        if sync:
            self.sync(stream)
        return out

    def batch(self, queries, dist_out=None, hit_out=None, status_out=None, stream=None, sync: bool = True):
        """Batched queries (g3d_batch).  `queries` = list of (Mesh a, Mesh b, op).
        Returns (dist float64[n], hit uint8[n], status int32[n])."""
        qa = np.fromiter((q[0].handle for q in queries), np.int64, len(queries))
        qb = np.fromiter((q[1].handle for q in queries), np.int64, len(queries))
        ops = np.fromiter((int(q[2]) for q in queries), np.int32, len(queries))
        return self.batch_arrays(qa, qb, ops, dist_out, hit_out, status_out, stream, sync)

    QUERY_DTYPE = np.dtype([("a", "<i8"), ("b", "<i8"), ("op", "<i4"), ("pad", "<i4")])

    def batch_arrays(self, qa, qb, ops, dist_out=None, hit_out=None, status_out=None, stream=None,
                     sync: bool = True):
        """g3d_batch on queries given as arrays of mesh handles (int64) and
        ops (int32): the same call as batch() without a Python loop."""
        n = len(qa)
        q = np.zeros(n, self.QUERY_DTYPE)
        q["a"], q["b"], q["op"] = qa, qb, ops
        d = np.full(n, np.nan) if dist_out is None else dist_out
        h = np.zeros(n, np.uint8) if hit_out is None else hit_out
        s = np.zeros(n, np.int32) if status_out is None else status_out
        dp, _, _, _ = _ptr_of(d)
        hp, _, _, _ = _ptr_of(h)
        sp, _, _, _ = _ptr_of(s)
        _check(self.lib.g3d_batch(self.h, q.ctypes.data_as(C.POINTER(g3d_query)), n, C.c_void_p(dp),
                                  C.c_void_p(hp), C.c_void_p(sp), _stream_ptr(stream)), "g3d_batch")
        if sync:
            self.sync(stream)
        return d, h, s

    def batch_witness(self, queries, stream=None):
        """Distance results with the witness face pair of each (g3d_batch_ex).
        Returns host arrays (dist float64[n], witness int64[n]: (a << 32) | b
        in input face ids or -1, status int32[n], cluster int32[n]: cA * 64 + cB
        of the witness or -1)."""
        import torch
        n = len(queries)
        arr = (g3d_query * n)()
        for i, (a, b, op) in enumerate(queries):
            arr[i].a, arr[i].b, arr[i].op = a.handle, b.handle, int(op)
        d = np.full(n, np.nan)
        h = np.zeros(n, np.uint8)
        s = np.zeros(n, np.int32)
        dev = f"cuda:{self.device}"
        w = torch.empty(n, dtype=torch.int64, device=dev)
        cl = torch.empty(n, dtype=torch.int32, device=dev)
        _check(self.lib.g3d_batch_ex(self.h, arr, n, C.c_void_p(d.ctypes.data), C.c_void_p(h.ctypes.data),
                                     C.c_void_p(s.ctypes.data), C.c_void_p(w.data_ptr()), C.c_void_p(cl.data_ptr()),
                                     _stream_ptr(stream)), "g3d_batch_ex")
        self.sync(stream)
        return d, w.cpu().numpy(), s, cl.cpu().numpy()

    def volume(self, meshes, out=None, stream=None):
        """Volumes of a mesh or a list of meshes (g3d_volume_many, Eq. 2).
        Returns a float for one mesh, else a float64 array (or fills `out`)."""
        one = isinstance(meshes, Mesh)
        ms = [meshes] if one else list(meshes)
        n = len(ms)
        hs = (C.c_int64 * max(n, 1))(*[m.handle for m in ms])
        res = np.zeros(n) if out is None else out
        rp, _, _, _ = _ptr_of(res)
        _check(self.lib.g3d_volume_many(self.h, n, hs, C.c_void_p(rp), _stream_ptr(stream)), "g3d_volume_many")
        return float(res[0]) if (one and out is None) else res

    def segments(self, mesh: Mesh, segs, op: int = OP_DISTANCE, dist_out=None, hit_out=None,
                 status_out=None, stream=None, sync: bool = True):
        """Segments / points against one mesh (g3d_segments).  segs: float32
        [n, 6] (P0, P1) as a numpy array or torch tensor (host or device).
        Returns (dist, hit, status); host numpy arrays unless outputs are given."""
        sp, skeep, sdt, n = _ptr_of(segs)
        if sdt != "float32":
            sp, skeep, sdt, n = _ptr_of(np.ascontiguousarray(np.asarray(segs, np.float32)))
        if tuple(skeep.shape[1:]) != (6,):
            raise ValueError("segments must be an [n, 6] array (P0, P1)")
        n = int(n)
        d = (np.full(n, np.nan) if op == OP_DISTANCE else None) if dist_out is None else dist_out
        h = np.zeros(n, np.uint8) if hit_out is None else hit_out
        s = np.zeros(n, np.int32) if status_out is None else status_out
        dp = _ptr_of(d)[0] if d is not None else 0
        hp, _, _, _ = _ptr_of(h)
        stp, _, _, _ = _ptr_of(s)
        _check(self.lib.g3d_segments(self.h, mesh.handle, C.c_void_p(sp), n, int(op), C.c_void_p(dp),
                                     C.c_void_p(hp), C.c_void_p(stp), _stream_ptr(stream)), "g3d_segments")
        if sync:
            self.sync(stream)
        return d, h, s

    def autotune(self, queries, tune_leaf_size: bool = False, reps: int = 3, count_build: bool = False,
                 stream=None) -> dict:
        """g3d_autotune on a sample batch [(a, b, op), ...]; returns the
        chosen configuration (now the context's).  count_build charges each
        leaf size its rebuild time too."""
        n = len(queries)
        arr = (g3d_query * n)()
        for i, (a, b, op) in enumerate(queries):
            arr[i].a, arr[i].b, arr[i].op = a.handle, b.handle, int(op)
        out = g3d_config()
        flags = (1 if tune_leaf_size else 0) | (2 if (tune_leaf_size and count_build) else 0)
        _check(self.lib.g3d_autotune(self.h, arr, n, flags, reps, C.byref(out),
                                     _stream_ptr(stream)), "g3d_autotune")
        return {f: getattr(out, f) for f, _ in g3d_config._fields_ if f != "reserved"}

    def batch_hint(self, queries, hint, witness: bool = False, stream=None):
        """g3d_batch_hint: queries with caller-supplied proposals hint[i] =
        cA * 64 + cB (or -1).  Returns (dist, hit, status[, witness, cluster]) on the host."""
        import torch
        n = len(queries)
        arr = (g3d_query * n)()
        for i, (a, b, op) in enumerate(queries):
            arr[i].a, arr[i].b, arr[i].op = a.handle, b.handle, int(op)
        hv = np.ascontiguousarray(np.asarray(hint, np.int32))
        if hv.shape != (n,):
            raise ValueError("one hint per query")
        d = np.full(n, np.nan)
        h = np.zeros(n, np.uint8)
        s = np.zeros(n, np.int32)
        w = torch.empty(n, dtype=torch.int64, device=f"cuda:{self.device}") if witness else None
        cl = torch.empty(n, dtype=torch.int32, device=f"cuda:{self.device}") if witness else None
        _check(self.lib.g3d_batch_hint(self.h, arr, n, C.c_void_p(hv.ctypes.data), C.c_void_p(d.ctypes.data),
                                       C.c_void_p(h.ctypes.data), C.c_void_p(s.ctypes.data),
                                       C.c_void_p(w.data_ptr() if witness else 0),
                                       C.c_void_p(cl.data_ptr() if witness else 0), _stream_ptr(stream)),
               "g3d_batch_hint")
        self.sync(stream)
        return (d, h, s, w.cpu().numpy(), cl.cpu().numpy()) if witness else (d, h, s)

    def pair_features(self, pairs, out=None, stream=None):
        """Features [n x 1536] (device tensor) of mesh pairs [(a, b), ...]."""
        import torch
        n = len(pairs)
        arr = (g3d_query * n)()
        for i, (a, b) in enumerate(pairs):
            arr[i].a, arr[i].b, arr[i].op = a.handle, b.handle, 0
        X = out if out is not None else torch.empty((n, 1536), dtype=torch.float32, device=f"cuda:{self.device}")
        _check(self.lib.g3d_pair_features(self.h, arr, n, C.c_void_p(X.data_ptr()), _stream_ptr(stream)),
               "g3d_pair_features")
        return X

    def proposal_topk(self, logits, k: int, stream=None):
        """Indices [B x k] (int32 device tensor) of the k largest logits of
        each row of a [B x N] float32 device tensor (g3d_proposal_topk)."""
        import torch
        B, N = logits.shape
        out = torch.empty((B, k), dtype=torch.int32, device=logits.device)
        _check(self.lib.g3d_proposal_topk(self.h, C.c_void_p(logits.data_ptr()), B, N, k,
                                          C.c_void_p(out.data_ptr()), _stream_ptr(stream)), "g3d_proposal_topk")
        return out

    def set_proposal(self, mlp):
        _check(self.lib.g3d_set_proposal(self.h, mlp.h if mlp is not None else None), "g3d_set_proposal")

    def plan_create(self, queries, dist_out, hit_out, status_out=None, stream=None):
        """Capture the batch of `queries` in a CUDA graph (g3d_plan_create);
        outputs are device tensors written by every plan_launch."""
        n = len(queries)
        arr = (g3d_query * n)()
        for i, (a, b, op) in enumerate(queries):
            arr[i].a, arr[i].b, arr[i].op = a.handle, b.handle, int(op)
        h = C.c_void_p()
        sp = C.c_void_p(status_out.data_ptr()) if status_out is not None else C.c_void_p(0)
        _check(self.lib.g3d_plan_create(self.h, arr, n, C.c_void_p(dist_out.data_ptr()),
                                        C.c_void_p(hit_out.data_ptr()), sp, C.byref(h), _stream_ptr(stream)),
               "g3d_plan_create")
        return h

    def plan_launch(self, plan, stream=None):
        _check(self.lib.g3d_plan_launch(self.h, plan, _stream_ptr(stream)), "g3d_plan_launch")

    def plan_destroy(self, plan):
        _check(self.lib.g3d_plan_destroy(self.h, plan), "g3d_plan_destroy")

    def sync(self, stream=None):
        _check(self.lib.g3d_sync(self.h, _stream_ptr(stream)), "g3d_sync")

    def stats(self, stream=None) -> dict:
        s = g3d_stats()
        _check(self.lib.g3d_stats_get(self.h, C.byref(s), _stream_ptr(stream)), "g3d_stats_get")
        return {f: getattr(s, f) for f, _ in g3d_stats._fields_ if f != "reserved"}

    def profile_begin(self, name_filter: str = ""):
        _check(self.lib.g3d_profile_begin(self.h, name_filter.encode()), "g3d_profile_begin")

    def profile_end(self) -> dict:
        """{kernel name: (launches, total_ms, max_ms)} since profile_begin."""
        cap = 64
        buf = (g3d_kernel_time * cap)()
        n = C.c_int()
        _check(self.lib.g3d_profile_end(self.h, buf, cap, C.byref(n)), "g3d_profile_end")
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms, buf[i].max_ms) for i in range(n.value)}

    def level_trace(self, cap: int = 1024, stream=None) -> np.ndarray:
        """The most recent levels of level-synchronous traversals (oldest
        first): rows of (ns since the launch started, level, node pairs,
        leaf pairs, block 0's expansion ns, block 0's ns until its leaf
        tests ended) (g3d_level_trace)."""
        buf = np.zeros((cap, 6), np.uint64)
        n = C.c_int()
        _check(self.lib.g3d_level_trace(self.h, C.c_void_p(buf.ctypes.data), cap, C.byref(n), _stream_ptr(stream)),
               "g3d_level_trace")
        return buf[:n.value]

    def debug_words(self) -> list:
        buf = (C.c_int * 8)()
        _check(self.lib.g3d_debug_words(self.h, buf), "g3d_debug_words")
        return list(buf)

    def stats_reset(self, stream=None):
        _check(self.lib.g3d_stats_reset(self.h, _stream_ptr(stream)), "g3d_stats_reset")


def linestring_mesh(P):
    """A line string (vertices P [n, 3], n >= 1, float32 or float64) as a
    mesh the operators take: face k = (P_k, P_k+1, P_k+1), a degenerate face
    whose closed point set is segment k; a single point becomes the face
    (P_0, P_0, P_0).  Line strings are one of the geometry types of Sec. 2.2;
    the mesh path decides degenerate faces exactly (as their segment or
    point), so distance and intersects of a line string against a surface,
    another line string or a point follow the same definitions (Sec. 3.2.2
    cases ii-iii, Sec. 3.2.3).  Returns (V, I uint32 [max(1, n-1), 3])."""
    V = np.ascontiguousarray(P)
    if V.ndim != 2 or V.shape[1] != 3 or V.shape[0] < 1:
        raise ValueError("a line string needs points [n >= 1, 3]")
    n = V.shape[0]
    if n == 1:
        return V, np.zeros((1, 3), np.uint32)
    k = np.arange(n - 1, dtype=np.uint32)
    return V, np.ascontiguousarray(np.stack([k, k + 1, k + 1], axis=1))


def collection_mesh(parts):
    """Several geometries (meshes, line strings as linestring_mesh gives
    them, points) as one geometry: the union of their faces, vertex arrays
    concatenated (in a common float type) and indices offset.  Distance and
    intersects of a collection are the minimum / any over its parts, which
    is what the union of faces gives.  Returns (V, I uint32)."""
    if not parts:
        raise ValueError("an empty collection has no faces")
    dt = np.float64 if any(np.asarray(V).dtype == np.float64 for V, _ in parts) else np.float32
    Vs, Is, off = [], [], 0
    for V, I in parts:
        V = np.asarray(V, dt).reshape(-1, 3)
        Is.append(np.asarray(I, np.uint32).reshape(-1, 3) + np.uint32(off))
        Vs.append(V)
        off += V.shape[0]
    return np.ascontiguousarray(np.concatenate(Vs)), np.ascontiguousarray(np.concatenate(Is))


def declared_functions(header: str | None = None) -> list[str]:
    """Names of the functions include/geo3d.h declares."""
    import re
    header = header or os.path.join(_build.INCLUDE, "geo3d.h")
    txt = open(header).read()
    return sorted(set(re.findall(r"\b(g3d_[a-z0-9_]+)\s*\(", txt)))


class MLP:
    """The learned-proposal network of a context (g3d_mlp_*)."""

    def __init__(self, ctx: Context, params=None):
        self.ctx = ctx
        self.lib = ctx.lib
        h = C.c_void_p()
        _check(self.lib.g3d_mlp_create(ctx.h, C.byref(h)), "g3d_mlp_create")
        self.h = h
        self.n = int(self.lib.g3d_mlp_num_params())
        if params is not None:
            self.set_params(params)

    def close(self):
        if getattr(self, "h", None):
            self.lib.g3d_mlp_destroy(self.ctx.h, self.h)
            self.h = None

    def set_params(self, params):
        p, keep, _, _ = _ptr_of(params if not isinstance(params, np.ndarray) else np.asarray(params, np.float32))
        if (params.numel() if hasattr(params, "numel") else np.asarray(params).size) != self.n:
            raise ValueError("wrong number of parameters")
        _check(self.lib.g3d_mlp_set_params(self.ctx.h, self.h, C.c_void_p(p)), "g3d_mlp_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n, np.float32)
        _check(self.lib.g3d_mlp_get_params(self.ctx.h, self.h, C.c_void_p(out.ctypes.data)), "g3d_mlp_get_params")
        return out

    def train(self, X, labels, steps: int, batch: int = 256, lr: float = 1e-3, seed: int = 0, stream=None) -> float:
        """g3d_mlp_train: `steps` Adam steps on minibatches drawn on the
        device from X [n x 1536] / labels [n] (device tensors); returns the
        last loss."""
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        _check(self.lib.g3d_mlp_train(self.ctx.h, self.h, C.c_void_p(X.data_ptr()), C.c_void_p(labels.data_ptr()),
                                      int(X.shape[0]), int(steps), int(batch), float(lr), int(seed),
                                      C.c_void_p(loss.data_ptr()), _stream_ptr(stream)), "g3d_mlp_train")
        return float(loss.item())

    def save(self, path: str):
        """g3d_mlp_save: the parameters to a checkpoint file."""
        _check(self.lib.g3d_mlp_save(self.ctx.h, self.h, os.fsencode(path)), "g3d_mlp_save")

    def load(self, path: str):
        """g3d_mlp_load: the parameters from a checkpoint file (Adam reset)."""
        _check(self.lib.g3d_mlp_load(self.ctx.h, self.h, os.fsencode(path)), "g3d_mlp_load")

    def forward(self, X, stream=None):
        import torch
        B = X.shape[0]
        z = torch.empty((B, 4096), dtype=torch.float32, device=X.device)
        _check(self.lib.g3d_mlp_forward(self.ctx.h, self.h, C.c_void_p(X.data_ptr()), B, C.c_void_p(z.data_ptr()),
                                        _stream_ptr(stream)), "g3d_mlp_forward")
        return z

    def gradients(self, X, labels, stream=None):
        g = np.empty(self.n, np.float32)
        loss = np.zeros(1, np.float32)
        _check(self.lib.g3d_mlp_gradients(self.ctx.h, self.h, C.c_void_p(X.data_ptr()), C.c_void_p(labels.data_ptr()),
                                          X.shape[0], C.c_void_p(g.ctypes.data), C.c_void_p(loss.ctypes.data),
                                          _stream_ptr(stream)), "g3d_mlp_gradients")
        return g, float(loss[0])

    def train_step(self, X, labels, lr: float, loss_out=None, stream=None):
        """One Adam step; loss_out (device float32[1] tensor) receives the loss."""
        lp = C.c_void_p(loss_out.data_ptr()) if loss_out is not None else C.c_void_p(0)
        _check(self.lib.g3d_mlp_train_step(self.ctx.h, self.h, C.c_void_p(X.data_ptr()),
                                           C.c_void_p(labels.data_ptr()), X.shape[0], C.c_float(lr), lp,
                                           _stream_ptr(stream)), "g3d_mlp_train_step")
