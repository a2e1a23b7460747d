"""The no-allocation entry point (g3d_distance_soup_noalloc) through the C
ABI, against the regular entry point (meshes + BVH + g3d_distance).

It serves callers that cannot allocate device memory (graph capture, a host
that owns all device memory, real-time code); its working memory is a fixed
array inside the library.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15


def _noalloc(lib, fa, fb, out, status):
    lib.g3d_distance_soup_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                              C.c_void_p, C.c_void_p]
    return lib.g3d_distance_soup_noalloc(C.c_void_p(fa.data_ptr()), fa.shape[0], C.c_void_p(fb.data_ptr()),
                                         fb.shape[0], C.c_void_p(out.data_ptr()), C.c_void_p(status.data_ptr()),
                                         C.c_void_p(0))


def _soup(rng, nt, shift):
    M = synth.tiny_random_mesh(nt, rng, spread=1.0, size=0.3, dtype=np.float32)
    M.V = (M.V + np.asarray(shift, np.float32)).astype(np.float32)
    return M


def test_noalloc_matches_regular_entry_point_twice(g3d):
    import torch
    lib = g3d.load()
    ctx = g3d.Context(0, time_limit_ms=10000)
    rng = np.random.default_rng(2024)
    pairs = [(_soup(rng, 300, (0, 0, 0)), _soup(rng, 250, (1.9, 0.2, 0.0))),   # separated
             (_soup(rng, 180, (0, 0, 0)), _soup(rng, 220, (0.4, 0.0, 0.1)))]   # overlapping
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda:0")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda:0")
    for A, B in pairs:  # two calls in a row on the shared scratch array
        fa = torch.from_numpy(A.V.reshape(-1, 9).copy()).cuda()
        fb = torch.from_numpy(B.V.reshape(-1, 9).copy()).cuda()
        assert _noalloc(lib, fa, fb, out, status) == 0
        torch.cuda.synchronize()
        got = float(out.item())
        assert int(status.item()) == 0
        ma = ctx.load_and_build(A.V, A.I, copy_fp64_master=False)
        mb = ctx.load_and_build(B.V, B.I, copy_fp64_master=False)
        ref = ctx.distance(ma, mb)
        assert abs(got - ref) <= REL * abs(ref) + ABS, (got, ref)
        assert (got == 0.0) == ctx.intersects(ma, mb)
        ctx.mesh_free_many([ma, mb])
    # beyond the fixed scratch size the call is refused before any work
    big = torch.zeros((9000, 9), dtype=torch.float32, device="cuda:0")
    assert _noalloc(lib, big, big, out, status) == -11
    ctx.close()
