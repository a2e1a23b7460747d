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
