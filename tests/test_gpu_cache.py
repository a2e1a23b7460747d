"""The device-resident geometry cache (cache.GeometryCache) on the GPU:
whole-column evaluation over more geometry than its budget holds (so
geometries are evicted and loaded again on demand), and a mixed query list,
against the same queries on meshes loaded directly and against the CPU
oracle on a sample (Sec. 3.1: geometry mirrored on the device, loaded
asynchronously on demand; whole-column evaluation)."""
import numpy as np
import pytest

from paper_1808_09571_gb300 import synth
from paper_1808_09571_gb300.cache import GeometryCache

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15


def test_cache_whole_column_and_queries(g3d, orc):
    import torch
    meshes, queries, _ = synth.batch_workload(15, seed=77, t_min=200, t_max=3000, p_intersect=0.3)
    cat = {g: (V, I) for g, (V, I) in enumerate(meshes)}
    faces = sum(len(I) for _, I in meshes)
    ctx = g3d.Context(0, time_limit_ms=10000)
    try:
        cache = GeometryCache(ctx, cat, budget_bytes=73 * faces // 3)
        col = list(range(1, len(meshes)))
        d, h0, s0 = cache.whole_column(col, 0, op=0)
        _, h1, s1 = cache.whole_column(col, 0, op=1)
        assert (s0 == 0).all() and (s1 == 0).all()
        assert cache.evictions > 0 and cache.loads > len(meshes)
        qa = [a for a, _, _ in queries]
        qb = [b for _, b, _ in queries]
        ops = [op for _, _, op in queries]
        dq, hq, sq = cache.evaluate(qa, qb, ops)
        assert (sq == 0).all()
        cache.clear()
        # the same queries on meshes loaded directly
        hs = [ctx.load_and_build(V, I, copy_fp64_master=False) for V, I in meshes]
        rd, _, _ = ctx.batch([(hs[g], hs[0], 0) for g in col])
        _, rh, _ = ctx.batch([(hs[g], hs[0], 1) for g in col])
        assert np.array_equal(d, rd) and np.array_equal(h1, rh)
        qd, qh, _ = ctx.batch([(hs[a], hs[b], op) for a, b, op in queries])
        dist_q = np.array(ops) == 0
        assert np.array_equal(dq[dist_q], qd[dist_q]) and np.array_equal(hq[~dist_q], qh[~dist_q])
        # oracle on a sample of the column
        for g in col[::5]:
            A, B = meshes[g], meshes[0]
            ref = orc.mesh_distance_pruned(A[0].astype(np.float64), A[1], B[0].astype(np.float64), B[1])
            inter = orc.mesh_intersects_pruned(A[0].astype(np.float64), A[1], B[0].astype(np.float64), B[1])
            i = g - 1
            assert abs(d[i] - ref) <= REL * abs(ref) + ABS, (g, d[i], ref)
            assert bool(h1[i]) == inter
        ctx.mesh_free_many(hs)
        torch.cuda.synchronize()
    finally:
        ctx.close()
