"""Line segments and points against a polyhedral surface (g3d_segments)
against the CPU oracle: each segment is the oracle's degenerate face
(P0, P1, P1), whose distance and intersection the oracle pins separately."""
import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15


def close(d, ref):
    return abs(d - ref) <= REL * abs(ref) + ABS


def seg_mesh(seg):
    """A segment as the oracle's one-face degenerate mesh."""
    V = np.array([seg[:3], seg[3:], seg[3:]], np.float64)
    return V, np.array([[0, 1, 2]], np.uint32)


@pytest.fixture(scope="module")
def ctx(g3d):
    c = g3d.Context(0, time_limit_ms=10000)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ore(ctx):
    o = synth.small_ore_body()
    h = ctx.mesh_load(o.V, o.I, copy_fp64_master=False)
    ctx.mesh_build_bvh(h)
    return o, h


def test_drill_holes_against_oracle(ctx, ore, orc, g3d):
    o, h = ore
    segs = synth.drill_holes(150, 20, step=4.0, seed=91)
    d, hd, s = ctx.segments(h, segs, g3d.OP_DISTANCE)
    _, hi, si = ctx.segments(h, segs, g3d.OP_INTERSECTS)
    assert (s == 0).all() and (si == 0).all()
    OV = o.V.astype(np.float64)
    n_hit = n_near = 0
    for i, sg in enumerate(segs):
        V, I = seg_mesh(sg.astype(np.float64))
        ref = orc.mesh_distance_pruned(V, I, OV, o.I)
        inter = orc.mesh_intersects_pruned(V, I, OV, o.I)
        assert close(d[i], ref), (i, d[i], ref)
        assert bool(hi[i]) == inter, i
        assert bool(hd[i]) == (ref == 0.0), i
        n_hit += inter
        n_near += 0.0 < ref < 1.0
    assert n_hit > 20 and n_near > 20, (n_hit, n_near)


def test_points_and_exact_contacts(ctx, ore, orc, g3d):
    """Points (P0 == P1) inside, outside and on the surface; segments ending
    on a vertex, lying along an edge, in a face plane."""
    o, h = ore
    rng = np.random.default_rng(5)
    V, I = o.V, o.I
    rows = []
    for k in range(40):  # points on vertices, on edge midpoints (rounded), random
        v = V[I[k * 7 % len(I)]]
        rows.append(np.r_[v[0], v[0]])
        rows.append(np.r_[v[0], v[1]])                      # along an edge
        m = ((v[0].astype(np.float64) + v[1] + v[2]) / 3).astype(np.float32)
        rows.append(np.r_[m, m])                             # near the face centroid
        rows.append(np.r_[v[0] * 1.5, v[0] * 0.5])           # crosses the surface near a vertex
        p = rng.uniform(-45, 45, 3).astype(np.float32)
        rows.append(np.r_[p, p])
    segs = np.array(rows, np.float32)
    d, hd, s = ctx.segments(h, segs, g3d.OP_DISTANCE)
    _, hi, _ = ctx.segments(h, segs, g3d.OP_INTERSECTS)
    assert (s == 0).all()
    OV = V.astype(np.float64)
    for i, sg in enumerate(segs):
        SV, SI = seg_mesh(sg.astype(np.float64))
        ref = orc.mesh_distance_brute(SV, SI, OV, I)
        assert close(d[i], ref), (i, d[i], ref)
        assert bool(hi[i]) == orc.mesh_intersects_brute(SV, SI, OV, I), i
    assert hi[0::5].all()  # a vertex lies on the surface
    assert hi[1::5].all()  # so does an edge


def test_segments_equal_the_mesh_path(ctx, ore, g3d):
    """A segment through g3d_segments and as a one-face degenerate mesh
    through g3d_distance / g3d_intersects: the same intersections, distances
    within the tolerance (the FP64 recomputations use 5 and 15 feature
    terms respectively, so their roundings may differ)."""
    o, h = ore
    segs = synth.drill_holes(6, 10, step=6.0, seed=3)
    d, _, _ = ctx.segments(h, segs, g3d.OP_DISTANCE)
    _, hi, _ = ctx.segments(h, segs, g3d.OP_INTERSECTS)
    for i, sg in enumerate(segs):
        V = np.array([sg[:3], sg[3:], sg[3:]], np.float32)
        m = ctx.mesh_load(V, np.array([[0, 1, 2]], np.uint32), copy_fp64_master=False)
        ctx.mesh_build_bvh(m)
        assert close(ctx.distance(m, h), d[i]), i
        assert ctx.intersects(m, h) == bool(hi[i]), i
        ctx.mesh_free(m)


def test_fp64_mesh(ctx, orc, g3d):
    """A mesh loaded from FP64 vertices keeps its FP64 master copy: results
    are exact for the FP64 input (the FP32 filters widen by the rounding)."""
    A, _ = synth.small_pairs()["A"]
    m = ctx.mesh_load(A.V, A.I, copy_fp64_master=True)
    ctx.mesh_build_bvh(m)
    rng = np.random.default_rng(8)
    P0 = rng.normal(0, 1, (300, 3))
    P0 /= np.linalg.norm(P0, axis=1, keepdims=True)
    P0 *= rng.uniform(0.5, 1.6, (300, 1))
    segs = np.hstack([P0, P0 + rng.normal(0, 0.2, (300, 3))]).astype(np.float32)
    d, _, s = ctx.segments(m, segs, g3d.OP_DISTANCE)
    _, hi, _ = ctx.segments(m, segs, g3d.OP_INTERSECTS)
    assert (s == 0).all()
    for i in range(0, 300, 3):
        V, I = seg_mesh(segs[i].astype(np.float64))
        ref = orc.mesh_distance_pruned(V, I, A.V, A.I)
        assert close(d[i], ref), (i, d[i], ref)
        assert bool(hi[i]) == orc.mesh_intersects_pruned(V, I, A.V, A.I)
    ctx.mesh_free(m)


def test_device_inputs_and_errors(ctx, ore, g3d):
    import torch
    o, h = ore
    segs = synth.drill_holes(20, 10, step=6.0, seed=4)
    segs[7, 2] = np.nan
    segs[9, 4] = 3e18  # beyond 2^60
    d, hd, s = ctx.segments(h, segs, g3d.OP_DISTANCE)
    assert s[7] == -2 and np.isnan(d[7]) and hd[7] == 0xff
    assert s[9] == -9 and np.isnan(d[9])
    ok = np.ones(len(segs), bool)
    ok[[7, 9]] = False
    assert (s[ok] == 0).all() and np.isfinite(d[ok]).all()
    # device input and outputs give the same results
    dv = torch.from_numpy(segs).cuda()
    dd = torch.empty(len(segs), dtype=torch.float64, device="cuda")
    dh = torch.empty(len(segs), dtype=torch.uint8, device="cuda")
    ds = torch.empty(len(segs), dtype=torch.int32, device="cuda")
    ctx.segments(h, dv, g3d.OP_DISTANCE, dist_out=dd, hit_out=dh, status_out=ds)
    np.testing.assert_array_equal(dd.cpu().numpy()[ok], d[ok])
    np.testing.assert_array_equal(ds.cpu().numpy(), s)
    # empty input, bad op, bad shape
    d0, _, _ = ctx.segments(h, np.zeros((0, 6), np.float32))
    assert len(d0) == 0
    with pytest.raises(g3d.G3DError):
        ctx.segments(h, segs, 7)
    with pytest.raises(ValueError):
        ctx.segments(h, np.zeros((4, 3), np.float32))
