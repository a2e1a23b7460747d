"""The independent-pairs workload at its full size against the oracle.

100,000 pairs (200,000 meshes, faces log-uniform in [20, 65,536], about 1.6
billion faces, 30 % sharing a vertex, 50 % distance and 50 % intersects
queries), loaded, built and queried through the array forms of the calls in
one batched launch, as the benchmark's pairs workload runs them.  The oracle
(exact-pruned, on all host cores) recomputes a seeded sample of 100 queries:
60 drawn uniformly and the 40 with the most face pairs.  This exercises the
paths only large launches take: deep stacks, queue donation under load, a
full candidate pool.  Definitions: Sec. 3.2.2 (Eq. 3) and Sec. 3.2.3 (Eq. 4).
"""
import os

import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15
N_PAIRS = 100000


def test_pairs_full_size_sampled_against_oracle(g3d, orc):
    from paper_1808_09571_gb300 import geo3d
    meshes, queries, info = synth.batch_workload(N_PAIRS)
    ctx = g3d.Context(0, time_limit_ms=60000)
    try:
        vptr = np.array([V.ctypes.data for V, _ in meshes], np.uint64)
        iptr = np.array([I.ctypes.data for _, I in meshes], np.uint64)
        vdt = np.full(len(meshes), geo3d.G3D_F32, np.int32)
        nvs = np.array([len(V) for V, _ in meshes], np.int64)
        nts = np.array([len(I) for _, I in meshes], np.int64)
        hs = ctx.mesh_load_arrays(vptr, vdt, nvs, iptr, nts, copy_fp64_master=False)
        for c0 in range(0, len(hs), 60000):
            ctx.mesh_build_bvh_many(hs[c0:c0 + 60000])
        qa = np.array([q[0] for q in queries], np.int64)
        qb = np.array([q[1] for q in queries], np.int64)
        qop = np.array([q[2] for q in queries], np.int32)
        d, h, s = ctx.batch_arrays(hs[qa], hs[qb], qop)
        assert (s == 0).all(), np.unique(s)
        ctx.mesh_free_many(hs)
    finally:
        ctx.close()

    rng = np.random.default_rng(2026)
    work = np.array([info[i]["faces"][0] * info[i]["faces"][1] for i in range(len(queries))], np.float64)
    big = np.argsort(-work)[:40]
    rest = np.setdiff1d(np.arange(len(queries)), big)
    sample = np.concatenate([big, rng.choice(rest, size=60, replace=False)])
    used = sorted({int(queries[i][0]) for i in sample} | {int(queries[i][1]) for i in sample})
    pos = {m: k for k, m in enumerate(used)}
    table = [(meshes[m][0].astype(np.float64), meshes[m][1]) for m in used]
    ref = orc.batch_pruned(table, [pos[queries[i][0]] for i in sample], [pos[queries[i][1]] for i in sample],
                           [queries[i][2] for i in sample], nthreads=os.cpu_count() or 1)
    assert max(info[i]["faces"][0] for i in big) > 40000
    n_hit = 0
    for k, i in enumerate(sample):
        op = queries[i][2]
        if op == 0:
            assert abs(d[i] - ref[k]) <= REL * ref[k] + ABS, (i, d[i], ref[k])
            assert h[i] == (ref[k] == 0.0)
        else:
            assert bool(h[i]) == bool(ref[k]), i
            assert np.isnan(d[i])
            n_hit += int(ref[k])
        if info[i]["shares_vertex"]:
            assert (d[i] == 0.0) if op == 0 else bool(h[i])
    assert n_hit > 0
