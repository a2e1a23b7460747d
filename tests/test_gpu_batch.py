"""Batched evaluation of many independent pairs (the persistent multi-query
launch and its CUDA-graph plan) against the CPU oracle."""
import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15


def close(d, ref):
    return abs(d - ref) <= REL * abs(ref) + ABS


@pytest.fixture(scope="module")
def loaded(g3d):
    ctx = g3d.Context(0, time_limit_ms=10000)
    meshes, queries, info = synth.batch_workload(400, seed=4242, t_max=4096)
    handles = ctx.mesh_load_many(meshes, copy_fp64_master=False)
    ctx.mesh_build_bvh_many(handles)
    qs = [(handles[a], handles[b], op) for (a, b, op) in queries]
    yield ctx, meshes, queries, info, handles, qs
    ctx.close()


def test_batch_pairs_against_oracle(loaded, orc):
    ctx, meshes, queries, info, handles, qs = loaded
    d, h, s = ctx.batch(qs)
    assert (s == 0).all()
    rng = np.random.default_rng(0)
    sample = rng.choice(len(queries), size=80, replace=False)
    n_hit = 0
    for i in sample:
        a, b, op = queries[i]
        VA, IA = meshes[a]
        VB, IB = meshes[b]
        if op == 0:
            ref = orc.mesh_distance_pruned(VA.astype(np.float64), IA, VB.astype(np.float64), IB)
            assert close(d[i], ref), (i, d[i], ref)
            assert h[i] == (ref == 0.0)
            if not info[i]["shares_vertex"]:  # placed at a known gap
                assert abs(d[i] - info[i]["gap"]) <= 1e-4 * info[i]["gap"] + 1e-4
        else:
            ref = orc.mesh_intersects_pruned(VA.astype(np.float64), IA, VB.astype(np.float64), IB)
            assert bool(h[i]) == ref, i
            assert np.isnan(d[i])
            n_hit += ref
        if info[i]["shares_vertex"]:
            assert (d[i] == 0.0) if op == 0 else bool(h[i])
    assert n_hit > 0


def test_batch_equals_single_queries(loaded):
    ctx, meshes, queries, info, handles, qs = loaded
    d, h, s = ctx.batch(qs)
    for i in range(0, len(qs), 7):
        a, b, op = qs[i]
        if op == 0:
            assert d[i] == ctx.distance(a, b)
        else:
            assert bool(h[i]) == ctx.intersects(a, b)


def test_plan_graph_replays_batch(loaded):
    import torch
    ctx, meshes, queries, info, handles, qs = loaded
    d, h, s = ctx.batch(qs)
    dev = torch.device("cuda:0")
    dd = torch.full((len(qs),), -1.0, dtype=torch.float64, device=dev)
    hh = torch.zeros(len(qs), dtype=torch.uint8, device=dev)
    ss = torch.full((len(qs),), 7, dtype=torch.int32, device=dev)
    plan = ctx.plan_create(qs, dd, hh, ss)
    for _ in range(3):
        dd.fill_(-1.0)
        ctx.plan_launch(plan)
        ctx.sync()
        assert (ss.cpu().numpy() == 0).all()
        np.testing.assert_array_equal(dd.cpu().numpy(), d)
        np.testing.assert_array_equal(hh.cpu().numpy(), h)
    ctx.plan_destroy(plan)


def test_distance_without_intersects_phase(loaded, g3d):
    """isect_first=2 sends distance queries straight to the distance
    traversal; results must be identical to the default two-phase order."""
    ctx, meshes, queries, info, handles, qs = loaded
    d, h, s = ctx.batch(qs)
    c2 = g3d.Context(0, time_limit_ms=10000, isect_first=2)
    assert c2.config()["isect_first"] == 2
    hs2 = c2.mesh_load_many(meshes, copy_fp64_master=False)
    c2.mesh_build_bvh_many(hs2)
    qs2 = [(hs2[a], hs2[b], op) for (a, b, op) in queries]
    for ops in (None, 0):  # the mixed batch, then every pair as a distance query
        q = qs2 if ops is None else [(a, b, 0) for (a, b, _) in qs2]
        ref = (d, h, s) if ops is None else ctx.batch([(a, b, 0) for (a, b, _) in qs])
        d2, h2, s2 = c2.batch(q)
        assert (s2 == 0).all()
        np.testing.assert_array_equal(d2, ref[0])
        np.testing.assert_array_equal(h2, ref[1])
    c2.close()


def test_hints_never_change_results(loaded):
    """Caller-supplied proposals (the true witness clusters, random clusters,
    none, out of range) leave every result unchanged; the true clusters
    lower the candidate count."""
    ctx, meshes, queries, info, handles, qs = loaded
    dq = [(a, b, 0) for (a, b, _) in qs]
    d, w, s, true = ctx.batch_witness(dq)
    _, h, _ = ctx.batch(dq)
    rng = np.random.default_rng(1)
    cands = {}
    for name, hint in (("none", None), ("true", true), ("random", rng.integers(0, 4096, len(dq))),
                       ("minus1", np.full(len(dq), -1)), ("oob", np.full(len(dq), 5000))):
        ctx.stats_reset()
        if hint is None:
            d1, h1, s1 = ctx.batch(dq)
        else:
            d1, h1, s1 = ctx.batch_hint(dq, hint)
        cands[name] = ctx.stats()["candidates"]
        assert (s1 == 0).all(), name
        np.testing.assert_array_equal(d1, d, err_msg=name)
        np.testing.assert_array_equal(h1, h, err_msg=name)
    assert cands["true"] < cands["none"], cands


def test_autotune_keeps_results(g3d):
    """The autotuner picks launch parameters and leaf sizes on a sample; the
    results of the whole batch, including meshes the sample did not rebuild
    (a batch mixing leaf sizes), stay identical."""
    meshes, queries, info = synth.batch_workload(120, seed=4343, t_max=3000)
    ctx = g3d.Context(0, time_limit_ms=10000)
    hs = ctx.mesh_load_many(meshes, copy_fp64_master=False)
    ctx.mesh_build_bvh_many(hs)
    qs = [(hs[a], hs[b], op) for (a, b, op) in queries]
    d0, h0, s0 = ctx.batch(qs)
    chosen = ctx.autotune(qs[:60], tune_leaf_size=True, reps=1)
    cfg = ctx.config()
    assert chosen == cfg
    assert cfg["leaf_size"] in (4, 8, 16) and cfg["isect_first"] in (1, 2) and cfg["morton_bits"] in (8, 10)
    assert 1 <= cfg["warps_per_cta"] <= 4 and cfg["stack_depth"] in (128, 256, 512)
    d1, h1, s1 = ctx.batch(qs)
    assert (s1 == 0).all()
    np.testing.assert_array_equal(d1, d0)
    np.testing.assert_array_equal(h1, h0)
    # a batch that mixes leaf sizes and Morton widths explicitly: every other
    # mesh rebuilt at leaf size 4 with 8-bit Morton axes
    ctx.set_config(leaf_size=4, morton_bits=8)
    assert ctx.config()["leaf_size"] == 4 and ctx.config()["morton_bits"] == 8
    ctx.mesh_build_bvh_many(hs[::2])
    d2, h2, s2 = ctx.batch(qs)
    assert (s2 == 0).all()
    np.testing.assert_array_equal(d2, d0)
    np.testing.assert_array_equal(h2, h0)
    with pytest.raises(g3d.G3DError):
        ctx.set_config(queue_capacity=1 << 12)
    with pytest.raises(g3d.G3DError):
        ctx.autotune([], reps=1)
    ctx.close()


def test_shared_allocations_outlive_partial_frees(g3d):
    """Meshes loaded / built by one call share one device block: freeing
    some of them, rebuilding others (with another leaf size) and querying
    the rest must leave every result unchanged until the last one is freed."""
    meshes, queries, info = synth.batch_workload(30, seed=515, t_max=3000)
    ctx = g3d.Context(0, time_limit_ms=10000)
    hs = ctx.mesh_load_many(meshes, copy_fp64_master=False)
    ctx.mesh_build_bvh_many(hs)
    qs = [(hs[a], hs[b], op) for (a, b, op) in queries]
    d0, h0, s0 = ctx.batch(qs)
    # free the meshes of the first 10 pairs (in stream order), rebuild those
    # of the next 10
    import torch
    ctx.mesh_free_many_async([m for (a, b, _) in queries[:10] for m in (hs[a], hs[b])],
                             stream=torch.cuda.current_stream())
    with pytest.raises(g3d.G3DError):  # the handles are gone at once
        ctx.distance(qs[0][0], qs[0][1])
    ctx.set_config(leaf_size=4)
    ctx.mesh_build_bvh_many([m for (a, b, _) in queries[10:20] for m in (hs[a], hs[b])])
    rest = qs[10:]
    d1, h1, s1 = ctx.batch(rest)
    assert (s1 == 0).all()
    np.testing.assert_array_equal(d1, d0[10:])
    np.testing.assert_array_equal(h1, h0[10:])
    for (a, b, _) in queries[10:]:
        ctx.mesh_free(hs[a])
        ctx.mesh_free(hs[b])
    assert ctx.volume(ctx.mesh_load(*meshes[0])) != 0.0  # the context still works
    ctx.close()


def test_results_repeat_bit_for_bit(loaded):
    """20 reruns of the batch give identical results (the final FP64 minimum
    does not depend on the order the warps found the candidates in)."""
    ctx, meshes, queries, info, handles, qs = loaded
    d0, h0, s0 = ctx.batch(qs)
    for _ in range(19):
        d, h, s = ctx.batch(qs)
        np.testing.assert_array_equal(d, d0)
        np.testing.assert_array_equal(h, h0)


def test_candidate_pool_overflow_takes_a_second_pass(g3d, loaded):
    """With the smallest candidate pool, the first pass overflows and the
    queries are re-run from their bounds with an empty pool: results equal
    those of a default context."""
    ctx, meshes, queries, info, handles, qs = loaded
    sub = list(range(24))
    d0, h0, _ = ctx.batch([qs[i] for i in sub])
    small = g3d.Context(0, cand_capacity=1024, time_limit_ms=10000)
    hs = small.mesh_load_many([meshes[k] for i in sub for k in queries[i][:2]], copy_fp64_master=False)
    small.mesh_build_bvh_many(hs)
    small.stats_reset()
    d1, h1, s1 = small.batch([(hs[2 * j], hs[2 * j + 1], queries[i][2]) for j, i in enumerate(sub)])
    st = small.stats()
    assert st["second_passes"] > 0, st
    assert (s1 == 0).all(), s1
    np.testing.assert_array_equal(d1, d0)
    np.testing.assert_array_equal(h1, h0)
    small.close()


def _sheet(n: int, z: float):
    """A flat n x n grid of squares (2 n^2 faces) at height z, float32."""
    xs = np.arange(n + 1, dtype=np.float64) / n
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], 1).astype(np.float32)
    k = np.arange(n)
    i, j = np.meshgrid(k, k, indexing="ij")
    a = (i * (n + 1) + j).ravel()
    I = np.concatenate([np.stack([a, a + n + 1, a + 1], 1), np.stack([a + 1, a + n + 1, a + n + 2], 1)])
    return V, I.astype(np.uint32)


def test_time_limit_reports_and_recovers(g3d):
    """A launch that outlives the configured limit stops by itself with
    G3D_ERR_TIMEOUT (every wait and the launch itself are bounded); after
    g3d_sync the context answers the same queries correctly.  Two parallel
    sheets of 320k faces 0.001 apart make the distance traversal test every
    nearby face pair, far longer than the 10 ms limit on one warp per SM."""
    A, B = _sheet(400, 0.0), _sheet(400, 1e-3)
    ctx = g3d.Context(0, time_limit_ms=10, warps_per_cta=1, ctas_per_sm=1, traversal=2)
    a, b = ctx.load_and_build(*A, copy_fp64_master=False), ctx.load_and_build(*B, copy_fp64_master=False)
    with pytest.raises(g3d.G3DError) as e:
        ctx.batch([(a, b, 0), (b, a, 0)])
    assert "TIMEOUT" in str(e.value)
    ctx.set_config(time_limit_ms=60000, warps_per_cta=4, ctas_per_sm=2)
    d, h, s = ctx.batch([(a, b, 0), (b, a, 1)])
    assert (s == 0).all() and h[1] == 0
    assert d[0] == np.float64(np.float32(1e-3))  # the sheets' exact gap
    ctx.close()


def test_frontier_overflow_finishes_in_the_queue(g3d, loaded):
    """With the smallest frontier (1,024 node pairs, 512 leaf pairs), the
    level-synchronous traversal hands what does not fit to the global queue
    and the persistent kernel finishes it: results equal those of a default
    context."""
    ctx, meshes, queries, info, handles, qs = loaded
    sub = list(range(400))
    d0, h0, _ = ctx.batch([qs[i] for i in sub])
    small = g3d.Context(0, frontier_capacity=1024, time_limit_ms=10000)
    hs = small.mesh_load_many([meshes[k] for i in sub for k in queries[i][:2]], copy_fp64_master=False)
    small.mesh_build_bvh_many(hs)
    small.stats_reset()
    d1, h1, s1 = small.batch([(hs[2 * j], hs[2 * j + 1], queries[i][2]) for j, i in enumerate(sub)])
    st = small.stats()
    assert st["queue_pushes"] > 0, st
    assert (s1 == 0).all(), s1
    np.testing.assert_array_equal(d1, d0)
    np.testing.assert_array_equal(h1, h0)
    small.close()


def test_work_that_fits_nowhere_is_rerun(g3d, loaded):
    """With the smallest frontier (1,024 node pairs) and the smallest global
    queue (8,192 entries, 4,096 of them usable), node pairs that fit neither
    are dropped and their queries marked; the second pass reruns those
    queries from their roots with the persistent kernel: no error, results
    equal those of a default context."""
    ctx, meshes, queries, info, handles, qs = loaded
    d0, h0, _ = ctx.batch(qs)
    small = g3d.Context(0, frontier_capacity=1024, queue_capacity=8192, time_limit_ms=20000)
    hs = small.mesh_load_many(meshes, copy_fp64_master=False)
    small.mesh_build_bvh_many(hs)
    small.stats_reset()
    d1, h1, s1 = small.batch([(hs[a], hs[b], op) for (a, b, op) in queries])
    st = small.stats()
    assert (s1 == 0).all(), s1
    assert st["second_passes"] > 0, st
    np.testing.assert_array_equal(d1, d0)
    np.testing.assert_array_equal(h1, h0)
    small.close()


def test_large_batch_runs_in_chunks(g3d, orc):
    """A level-synchronous batch whose queries reference more faces in all
    than chunk_mfaces runs as consecutive chunks (each with its own links
    between distance and intersects queries of one mesh pair): results with
    3 and with 6 chunks equal those of small batches of one mesh pair each
    (60 queries, never chunked) and the oracle on every distinct pair."""
    V, I = synth.icosphere(7, radius=1.0, seed=11)  # 327,680 faces
    V = np.asarray(V, np.float64)
    I = np.asarray(I, np.uint32)
    offs = [(0.0, 0.0, 0.0), (2.3, 0.0, 0.0), (0.0, 1.7, 0.4), (-1.0, -1.0, -1.0)]
    meshes = [((V + np.array(o)).astype(np.float32), I) for o in offs]
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    rng = np.random.default_rng(9)
    queries = [(*pairs[k], int(op)) for k, op in zip(rng.integers(0, 6, 1100), rng.integers(0, 2, 1100))]
    assert sum(2 * len(I) for _ in queries) > 2 * (256 << 20)
    res = []
    for cm in (256, 128):
        ctx = g3d.Context(0, time_limit_ms=20000, chunk_mfaces=cm)
        hs = ctx.mesh_load_many(meshes, copy_fp64_master=False)
        ctx.mesh_build_bvh_many(hs)
        d, h, s = ctx.batch([(hs[a], hs[b], op) for a, b, op in queries])
        assert (s == 0).all()
        res.append((d, h))
        if cm == 256:  # per mesh pair, small batches
            ref_d, ref_h = np.zeros(len(queries)), np.zeros(len(queries), np.uint8)
            for pr in pairs:
                idx = [i for i, q in enumerate(queries) if q[:2] == pr]
                for c0 in range(0, len(idx), 60):
                    part = idx[c0:c0 + 60]
                    dd, hh, ss = ctx.batch([(hs[queries[i][0]], hs[queries[i][1]], queries[i][2]) for i in part])
                    assert (ss == 0).all()
                    ref_d[part], ref_h[part] = dd, hh
        ctx.close()
    for d, h in res:
        dist_q = np.array([op == 0 for _, _, op in queries])
        np.testing.assert_array_equal(d[dist_q], ref_d[dist_q])
        np.testing.assert_array_equal(h[~dist_q], ref_h[~dist_q])
    d, h = res[0]
    for a, b in pairs:
        A, B = meshes[a], meshes[b]
        ref = orc.mesh_distance_pruned(A[0].astype(np.float64), A[1], B[0].astype(np.float64), B[1])
        inter = orc.mesh_intersects_pruned(A[0].astype(np.float64), A[1], B[0].astype(np.float64), B[1])
        for i, (qa, qb, op) in enumerate(queries):
            if (qa, qb) != (a, b):
                continue
            if op == 0:
                assert abs(d[i] - ref) <= 1e-12 * abs(ref) + 1e-15, (a, b, d[i], ref)
            else:
                assert bool(h[i]) == inter, (a, b)


def test_visit_counters(g3d, loaded):
    """count_visits: distinct nodes and faces read per query are counted
    (at most every internal node and face of both meshes per query), and
    the results do not change."""
    ctx, meshes, queries, info, handles, qs = loaded
    d0, h0, _ = ctx.batch(qs)
    cnt = g3d.Context(0, count_visits=1, time_limit_ms=10000)
    hs = cnt.mesh_load_many(meshes, copy_fp64_master=False)
    cnt.mesh_build_bvh_many(hs)
    cnt.stats_reset()
    d1, h1, s1 = cnt.batch([(hs[a], hs[b], op) for (a, b, op) in queries])
    st = cnt.stats()
    assert (s1 == 0).all()
    np.testing.assert_array_equal(d1, d0)
    np.testing.assert_array_equal(h1, h0)
    faces = sum(len(meshes[a][1]) + len(meshes[b][1]) for (a, b, _) in queries)
    assert 0 < st["distinct_faces"] <= faces, st
    assert 0 < st["distinct_nodes"] <= faces, st
    assert st["levels"] > 0
    cnt.close()


def test_config_file_round_trip(g3d, tmp_path):
    ctx = g3d.Context(0, leaf_size=8, ctas_per_sm=3, morton_bits=8)
    ctx.save_config(str(tmp_path / "tuned.json"))
    other = g3d.Context(0)
    cfg = other.load_config(str(tmp_path / "tuned.json"))
    assert cfg == ctx.config()
    other.close()
    ctx.close()


def test_array_forms_match_list_forms(loaded, g3d):
    """Loading by address arrays, building and querying by handle arrays, and
    freeing by handle array give the list forms' results bit for bit, for
    device (torch) and host (numpy) sources."""
    import torch
    ctx, meshes, queries, info, handles, qs = loaded
    d0, h0, s0 = ctx.batch(qs)
    dev = torch.device("cuda:0")
    for on_device in (True, False):
        if on_device:
            Vs = [torch.from_numpy(V).to(dev) for V, _ in meshes]
            Is = [torch.from_numpy(I.view(np.int32)).to(dev) for _, I in meshes]
            vptr = [t.data_ptr() for t in Vs]
            iptr = [t.data_ptr() for t in Is]
        else:
            Vs = [np.ascontiguousarray(V) for V, _ in meshes]
            Is = [np.ascontiguousarray(I) for _, I in meshes]
            vptr = [a.ctypes.data for a in Vs]
            iptr = [a.ctypes.data for a in Is]
        vdt = [g3d.G3D_F32 if V.dtype == np.float32 else g3d.G3D_F64 for V, _ in meshes]
        hs = ctx.mesh_load_arrays(vptr, vdt, [len(V) for V, _ in meshes], iptr, [len(I) for _, I in meshes],
                                  copy_fp64_master=False)
        assert hs.dtype == np.int64 and len(hs) == len(meshes) and len(set(hs.tolist())) == len(meshes)
        ctx.mesh_build_bvh_many(hs)
        qa = np.array([q[0] for q in queries], np.int64)
        qb = np.array([q[1] for q in queries], np.int64)
        op = np.array([q[2] for q in queries], np.int32)
        d1, h1, s1 = ctx.batch_arrays(hs[qa], hs[qb], op)
        assert (s1 == 0).all()
        assert np.array_equal(d1, d0, equal_nan=True) and np.array_equal(h1, h0)
        ctx.mesh_free_many(hs)
        torch.cuda.synchronize()
