"""The no-allocation entry point (g3d_distance_soup_noalloc) through the C
ABI.

It serves callers that cannot allocate device memory (a host whose device
memory belongs to its own allocator, a real-time pipeline that must not call
cudaMalloc once running); its working memory is a fixed array inside the
library.  Its results are checked against the CPU oracle's brute force and
against the regular entry point (meshes + BVH + g3d_distance), on calls in a
row over the shared array.  This file is collected last on purpose: a run
that stops at the first failure has run every other test first."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15


def _noalloc(lib, fa, fb, out, status):
    lib.g3d_distance_soup_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                              C.c_void_p, C.c_void_p]
    sp = C.c_void_p(status.data_ptr()) if status is not None else C.c_void_p(0)
    return lib.g3d_distance_soup_noalloc(C.c_void_p(fa.data_ptr()), fa.shape[0], C.c_void_p(fb.data_ptr()),
                                         fb.shape[0], C.c_void_p(out.data_ptr()), sp, C.c_void_p(0))


def _soup(rng, nt, shift):
    M = synth.tiny_random_mesh(nt, rng, spread=1.0, size=0.3, dtype=np.float32)
    M.V = (M.V + np.asarray(shift, np.float32)).astype(np.float32)
    return M


def _stacked(rng, nt, z):
    """nt large jittered faces in the plane z (every pair of an A and a B
    stack overlaps in projection, so all nt^2 pairs attain the distance)."""
    base = np.array([[-1.0, -1.0], [1.2, -0.9], [0.0, 1.1]])
    V = np.zeros((nt, 3, 3))
    V[:, :, :2] = base[None] + rng.uniform(-0.05, 0.05, size=(nt, 3, 2))
    V[:, :, 2] = z
    V = V.reshape(-1, 3).astype(np.float32)
    return synth.Mesh(V, np.arange(len(V), dtype=np.uint32).reshape(-1, 3))


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x.reshape(-1, 9))).cuda()


def test_noalloc_matches_oracle_and_regular_entry_point(g3d, orc):
    import torch
    lib = g3d.load()
    ctx = g3d.Context(0, time_limit_ms=10000)
    rng = np.random.default_rng(2024)
    pairs = [(_soup(rng, 300, (0, 0, 0)), _soup(rng, 250, (1.9, 0.2, 0.0))),   # separated
             (_soup(rng, 180, (0, 0, 0)), _soup(rng, 220, (0.4, 0.0, 0.1))),   # overlapping
             (_stacked(rng, 300, 0.0), _stacked(rng, 300, 0.5))]               # 90,000 pairs at 0.5
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda:0")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda:0")
    for A, B in pairs:  # calls in a row on the shared scratch array
        assert _noalloc(lib, _dev(A.V), _dev(B.V), out, status) == 0
        torch.cuda.synchronize()
        got = float(out.item())
        assert int(status.item()) == 0
        ref = orc.mesh_distance_brute(A.V.astype(np.float64), A.I, B.V.astype(np.float64), B.I)
        assert abs(got - ref) <= REL * abs(ref) + ABS, (got, ref)
        ma = ctx.load_and_build(A.V, A.I, copy_fp64_master=False)
        mb = ctx.load_and_build(B.V, B.I, copy_fp64_master=False)
        reg = ctx.distance(ma, mb)
        assert abs(got - reg) <= REL * abs(reg) + ABS, (got, reg)
        assert (got == 0.0) == ctx.intersects(ma, mb) == orc.mesh_intersects_brute(
            A.V.astype(np.float64), A.I, B.V.astype(np.float64), B.I)
        ctx.mesh_free_many([ma, mb])
    assert float(out.item()) == np.float64(np.float32(0.5))  # every stacked pair attains the gap
    ctx.close()


def test_noalloc_rejects_bad_input(g3d):
    import torch
    lib = g3d.load()
    rng = np.random.default_rng(5)
    A, B = _soup(rng, 40, (0, 0, 0)), _soup(rng, 30, (2.0, 0, 0))
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda:0")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda:0")
    for val, code in ((np.nan, -2), (np.inf, -2), (1e30, -9)):
        V = A.V.copy()
        V[7, 1] = val
        assert _noalloc(lib, _dev(V), _dev(B.V), out, status) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == code and np.isnan(out.item()), (val, status.item(), out.item())
    # the next call on the shared array starts clean
    assert _noalloc(lib, _dev(A.V), _dev(B.V), out, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and out.item() > 0
    # beyond the fixed size, without a status word, or with host memory:
    # refused before any work
    big = torch.zeros((9000, 9), dtype=torch.float32, device="cuda:0")
    assert _noalloc(lib, big, big, out, status) == -11
    assert _noalloc(lib, _dev(A.V), _dev(B.V), out, None) == -1
    host = torch.from_numpy(A.V.reshape(-1, 9).copy())
    assert _noalloc(lib, host, _dev(B.V), out, status) == -1


def test_noalloc_captured_in_a_graph(g3d, orc):
    """The call's main use: captured once into a CUDA graph (after a first
    direct call on the device), then replayed on new faces written into the
    same buffers."""
    import torch
    lib = g3d.load()
    rng = np.random.default_rng(77)
    cases = [(_soup(rng, 120, (0, 0, 0)), _soup(rng, 90, (1.7, 0.1, 0.0))),
             (_soup(rng, 120, (0, 0, 0)), _soup(rng, 90, (0.3, 0.0, 0.05))),
             (_soup(rng, 120, (0, 0, 0)), _soup(rng, 90, (0.0, 2.2, -0.4)))]
    fa = _dev(cases[0][0].V).clone()
    fb = _dev(cases[0][1].V).clone()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda:0")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda:0")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # first call, outside any capture
        assert _noalloc_on(lib, fa, fb, out, status, side) == 0
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        assert _noalloc_on(lib, fa, fb, out, status, torch.cuda.current_stream()) == 0
    for A, B in cases:
        fa.copy_(_dev(A.V))
        fb.copy_(_dev(B.V))
        out.fill_(-1.0)
        status.fill_(99)
        graph.replay()
        torch.cuda.synchronize()
        ref = orc.mesh_distance_brute(A.V.astype(np.float64), A.I, B.V.astype(np.float64), B.I)
        got = float(out.item())
        assert int(status.item()) == 0
        assert abs(got - ref) <= REL * abs(ref) + ABS, (got, ref)


def _noalloc_on(lib, fa, fb, out, status, stream):
    lib.g3d_distance_soup_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                              C.c_void_p, C.c_void_p]
    return lib.g3d_distance_soup_noalloc(C.c_void_p(fa.data_ptr()), fa.shape[0], C.c_void_p(fb.data_ptr()),
                                         fb.shape[0], C.c_void_p(out.data_ptr()),
                                         C.c_void_p(status.data_ptr()), C.c_void_p(stream.cuda_stream))
