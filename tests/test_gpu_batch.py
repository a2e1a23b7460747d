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
