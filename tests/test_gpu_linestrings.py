"""Line strings, points and mixed collections through the mesh path
(geo3d.linestring_mesh / collection_mesh, g3d_batch) against the CPU oracle
on the same faces: drill-hole line strings against the 500-face ore body
and against each other, single points, and a collection of a surface and
line strings against a sphere (Sec. 2.2 geometry types; Sec. 3.2.2 cases
ii-iii; Sec. 3.2.3).  Intersects bit-exact, distance within 1e-12
relative (1e-15 absolute at zero)."""
import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15


def close(d, ref):
    return abs(d - ref) <= REL * abs(ref) + ABS


def hole_paths(n_holes, segs, step, seed):
    """Vertices of drill-hole line strings (the segments of
    synth.drill_holes joined end to end)."""
    S = synth.drill_holes(n_holes, segs, step=step, seed=seed).reshape(n_holes, segs, 6)
    return [np.concatenate([S[h, :1, :3], S[h, :, 3:]]).astype(np.float32) for h in range(n_holes)]


def check(ctx, orc, g3d, geoms_a, geoms_b):
    la = [ctx.load_and_build(V, I, copy_fp64_master=False) for V, I in geoms_a]
    lb = [ctx.load_and_build(V, I, copy_fp64_master=False) for V, I in geoms_b]
    qs = [(a, b, op) for a, b in zip(la, lb) for op in (0, 1)]
    d, h, s = ctx.batch(qs)
    assert (s == 0).all()
    n_hit = 0
    for i, ((VA, IA), (VB, IB)) in enumerate(zip(geoms_a, geoms_b)):
        VA64, VB64 = np.asarray(VA, np.float64), np.asarray(VB, np.float64)
        ref = orc.mesh_distance_pruned(VA64, IA, VB64, IB)
        inter = orc.mesh_intersects_pruned(VA64, IA, VB64, IB)
        assert close(d[2 * i], ref), (i, d[2 * i], ref)
        assert bool(h[2 * i + 1]) == inter, i
        assert (d[2 * i] == 0.0) == inter, i
        n_hit += inter
    ctx.mesh_free_many(la + lb)
    return n_hit


@pytest.fixture(scope="module")
def ctx(g3d):
    c = g3d.Context(0, time_limit_ms=10000)
    yield c
    c.close()


def test_drill_hole_line_strings_against_the_ore_body(ctx, orc, g3d):
    o = synth.small_ore_body()
    paths = hole_paths(40, 30, 3.0, seed=71)
    A = [g3d.linestring_mesh(P) for P in paths]
    n_hit = check(ctx, orc, g3d, A, [(o.V, o.I)] * len(A))
    assert 5 <= n_hit <= 35, n_hit  # both outcomes are exercised


def test_line_strings_against_line_strings(ctx, orc, g3d):
    paths = hole_paths(40, 25, 2.0, seed=72)
    A = [g3d.linestring_mesh(P) for P in paths[:20]]
    B = [g3d.linestring_mesh(P) for P in paths[20:]]
    # a line string that crosses its partner: the partner's middle vertex
    # moved onto a vertex of the first (a shared point)
    P0, P1 = paths[0].copy(), paths[20].copy()
    P1[12] = P0[7]
    A.append(g3d.linestring_mesh(P0))
    B.append(g3d.linestring_mesh(P1))
    assert check(ctx, orc, g3d, A, B) >= 1


def test_points_against_a_surface(ctx, orc, g3d):
    o = synth.small_ore_body()
    rng = np.random.default_rng(73)
    pts = rng.uniform([-50, -35, -25], [50, 35, 25], size=(30, 3)).astype(np.float32)
    pts[:3] = o.V[[5, 77, 140]]  # exactly on the surface
    A = [g3d.linestring_mesh(p[None]) for p in pts]
    assert check(ctx, orc, g3d, A, [(o.V, o.I)] * len(A)) >= 3


def test_collection_of_surface_and_line_strings(ctx, orc, g3d):
    o = synth.small_ore_body()
    paths = hole_paths(6, 20, 3.0, seed=74)
    G = g3d.collection_mesh([(o.V, o.I)] + [g3d.linestring_mesh(P) for P in paths])
    sph = synth.icosphere(2, radius=3.0, seed=5)
    geoms_b = []
    for c in ([0.0, 0.0, 60.0], [0.0, 0.0, 20.0], [45.0, 0.0, 0.0], [0.0, 0.0, 0.0]):
        V = (np.asarray(sph[0], np.float64) + c).astype(np.float32)
        geoms_b.append((V, np.asarray(sph[1], np.uint32)))
    check(ctx, orc, g3d, [G] * len(geoms_b), geoms_b)
