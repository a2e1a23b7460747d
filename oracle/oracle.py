"""ctypes wrapper of the C oracle (oracle.c).  Test infrastructure only.

Inputs are taken as float64 vertex arrays; float32 inputs are widened exactly.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (round-to-nearest, no contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lpthread", "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(os.environ.get("ORACLE_SO_OVERRIDE") or build())
            d, i64, i32 = C.POINTER(C.c_double), C.c_int64, C.c_int32
            u32 = C.POINTER(C.c_uint32)
            L.orc_orient3d.argtypes = [d, d, d, d]
            L.orc_orient2d.argtypes = [d, d, d]
            L.orc_tri_intersects.argtypes = [d, d]
            L.orc_tri_feature_d2.argtypes = [d, d]
            L.orc_tri_feature_d2.restype = C.c_double
            L.orc_tri_distance.argtypes = [d, d]
            L.orc_tri_distance.restype = C.c_double
            L.orc_pt_tri_d2.argtypes = [d, d, d, d]
            L.orc_pt_tri_d2.restype = C.c_double
            L.orc_pt_seg_d2.argtypes = [d, d, d]
            L.orc_pt_seg_d2.restype = C.c_double
            L.orc_seg_seg_d2.argtypes = [d, d, d, d]
            L.orc_seg_seg_d2.restype = C.c_double
            L.orc_mesh_distance_brute.argtypes = [d, u32, i64, d, u32, i64,
                                                  C.POINTER(i64), C.POINTER(i64)]
            L.orc_mesh_distance_brute.restype = C.c_double
            L.orc_mesh_intersects_brute.argtypes = [d, u32, i64, d, u32, i64]
            L.orc_mesh_distance_pruned.argtypes = [d, u32, i64, d, u32, i64, C.POINTER(i64)]
            L.orc_mesh_distance_pruned.restype = C.c_double
            L.orc_mesh_intersects_pruned.argtypes = [d, u32, i64, d, u32, i64, C.POINTER(i64)]
            L.orc_batch_pruned.argtypes = [i64, C.POINTER(d), C.POINTER(u32), C.POINTER(i64),
                                           C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_int32),
                                           d, C.POINTER(i64), C.c_int]
            L.orc_bigint_overflowed.argtypes = []
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _u32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint32))


def _check_overflow():
    if lib().orc_bigint_overflowed():
        raise OverflowError("oracle big-integer capacity exceeded")


def orient3d(a, b, c, d) -> int:
    a, b, c, d = map(_f64, (a, b, c, d))
    r = lib().orc_orient3d(_dp(a), _dp(b), _dp(c), _dp(d))
    _check_overflow()
    return r


def orient2d(a, b, c) -> int:
    a, b, c = map(_f64, (a, b, c))
    r = lib().orc_orient2d(_dp(a), _dp(b), _dp(c))
    _check_overflow()
    return r


def tri_intersects(T1, T2) -> bool:
    T1, T2 = _f64(T1).reshape(9), _f64(T2).reshape(9)
    return bool(lib().orc_tri_intersects(_dp(T1), _dp(T2)))


def tri_feature_d2(T1, T2) -> float:
    T1, T2 = _f64(T1).reshape(9), _f64(T2).reshape(9)
    return lib().orc_tri_feature_d2(_dp(T1), _dp(T2))


def tri_distance(T1, T2) -> float:
    T1, T2 = _f64(T1).reshape(9), _f64(T2).reshape(9)
    return lib().orc_tri_distance(_dp(T1), _dp(T2))


def pt_tri_d2(p, a, b, c) -> float:
    p, a, b, c = map(_f64, (p, a, b, c))
    return lib().orc_pt_tri_d2(_dp(p), _dp(a), _dp(b), _dp(c))


def pt_seg_d2(p, a, b) -> float:
    p, a, b = map(_f64, (p, a, b))
    return lib().orc_pt_seg_d2(_dp(p), _dp(a), _dp(b))


def seg_seg_d2(p0, p1, q0, q1) -> float:
    p0, p1, q0, q1 = map(_f64, (p0, p1, q0, q1))
    return lib().orc_seg_seg_d2(_dp(p0), _dp(p1), _dp(q0), _dp(q1))


def _mesh(V, I):
    V = _f64(V).reshape(-1, 3)
    I = _u32(I).reshape(-1, 3)
    if len(I) and int(I.max()) >= len(V):
        raise ValueError("index out of range")
    return V, I, len(I)


def _up(I):
    return I.ctypes.data_as(C.POINTER(C.c_uint32))


def mesh_distance_brute(VA, IA, VB, IB, return_arg: bool = False):
    VA, IA, na = _mesh(VA, IA)
    VB, IB, nb = _mesh(VB, IB)
    ai, aj = C.c_int64(-1), C.c_int64(-1)
    r = lib().orc_mesh_distance_brute(_dp(VA), _up(IA), na, _dp(VB), _up(IB), nb,
                                      C.byref(ai), C.byref(aj))
    _check_overflow()
    return (r, ai.value, aj.value) if return_arg else r


def mesh_intersects_brute(VA, IA, VB, IB) -> bool:
    VA, IA, na = _mesh(VA, IA)
    VB, IB, nb = _mesh(VB, IB)
    r = bool(lib().orc_mesh_intersects_brute(_dp(VA), _up(IA), na, _dp(VB), _up(IB), nb))
    _check_overflow()
    return r


def mesh_distance_pruned(VA, IA, VB, IB, return_tests: bool = False):
    VA, IA, na = _mesh(VA, IA)
    VB, IB, nb = _mesh(VB, IB)
    t = C.c_int64(0)
    r = lib().orc_mesh_distance_pruned(_dp(VA), _up(IA), na, _dp(VB), _up(IB), nb, C.byref(t))
    _check_overflow()
    return (r, t.value) if return_tests else r


def mesh_intersects_pruned(VA, IA, VB, IB, return_tests: bool = False):
    VA, IA, na = _mesh(VA, IA)
    VB, IB, nb = _mesh(VB, IB)
    t = C.c_int64(0)
    r = bool(lib().orc_mesh_intersects_pruned(_dp(VA), _up(IA), na, _dp(VB), _up(IB), nb,
                                              C.byref(t)))
    _check_overflow()
    return (r, t.value) if return_tests else r


def batch_pruned(meshes, qa, qb, op, nthreads: int = 1, return_tests: bool = False):
    """Independent queries over a mesh table on `nthreads` threads.
    meshes: list of (V, I); op: 0 distance, 1 intersects.  Returns float64
    results (distance, or 1.0/0.0)."""
    Ms = [_mesh(V, I) for (V, I) in meshes]
    n = len(qa)
    Vp = (C.POINTER(C.c_double) * len(Ms))(*[_dp(m[0]) for m in Ms])
    Ip = (C.POINTER(C.c_uint32) * len(Ms))(*[_up(m[1]) for m in Ms])
    nt = np.array([m[2] for m in Ms], np.int64)
    qa = np.ascontiguousarray(qa, np.int64)
    qb = np.ascontiguousarray(qb, np.int64)
    op = np.ascontiguousarray(op, np.int32)
    out = np.zeros(n, np.float64)
    tests = np.zeros(n, np.int64)
    i64p = C.POINTER(C.c_int64)
    rc = lib().orc_batch_pruned(n, Vp, Ip, nt.ctypes.data_as(i64p), qa.ctypes.data_as(i64p),
                                qb.ctypes.data_as(i64p), op.ctypes.data_as(C.POINTER(C.c_int32)),
                                _dp(out), tests.ctypes.data_as(i64p), int(nthreads))
    if rc != 0:
        raise MemoryError("oracle batch allocation failed")
    _check_overflow()
    return (out, tests) if return_tests else out
