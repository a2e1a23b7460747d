"""Host-side marshalling of the Python binding (no device, no library call)."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_09571_gb300 import geo3d


def test_handles_from_meshes_and_arrays_agree():
    ms = [geo3d.Mesh(h, 10 + h) for h in (5, 3, 9, 1)]
    p1, n1, k1 = geo3d._handles(ms)
    p2, n2, k2 = geo3d._handles(np.array([5, 3, 9, 1], np.int64))
    assert n1 == n2 == 4
    assert [p1[i] for i in range(4)] == [p2[i] for i in range(4)] == [5, 3, 9, 1]
    # a non-int64 or strided array is converted, not misread
    p3, n3, k3 = geo3d._handles(np.array([5, 3, 9, 1, 7, 7], np.int32)[:4])
    assert [p3[i] for i in range(n3)] == [5, 3, 9, 1]


def test_mesh_value_semantics():
    a, b = geo3d.Mesh(7, 100), geo3d.Mesh(7, 100)
    assert a == b and a != geo3d.Mesh(8, 100)
    assert repr(a) == "Mesh(handle=7, nt=100)"
    with pytest.raises(TypeError):
        hash(a)
    with pytest.raises(AttributeError):
        a.extra = 1  # slots only


def test_ptr_of_numpy_and_torch():
    V = np.arange(12, dtype=np.float32).reshape(4, 3)
    p, keep, name, rows = geo3d._ptr_of(V)
    assert p == V.ctypes.data and name == "float32" and rows == 4
    # non-contiguous input is copied into a contiguous array that is kept alive
    Vt = np.asfortranarray(V)
    p, keep, name, rows = geo3d._ptr_of(Vt)
    assert keep.flags["C_CONTIGUOUS"] and np.array_equal(keep, V) and p == keep.ctypes.data
    torch = pytest.importorskip("torch")
    T = torch.arange(12, dtype=torch.int32).reshape(4, 3)
    p, keep, name, rows = geo3d._ptr_of(T)
    assert p == T.data_ptr() and name == "int32" and rows == 4
    Tt = T.t()  # not contiguous: a contiguous copy
    p, keep, name, rows = geo3d._ptr_of(Tt)
    assert keep.is_contiguous() and p == keep.data_ptr() and rows == 3
    assert C.sizeof(C.c_int64) == 8
