"""The exact stage of intersects on the GPU, on inputs only it can decide.

Near-coplanar face pairs (synth.near_coplanar_face_pairs): float64 vertices
at about 2^20 on a 2^-32 grid, with a vertex exactly on, or 2^-32 off, the
other face's plane.  The orientation determinants there are zero or below
2^7 against a double-precision forward error bound of about 2^8, so neither
the float32 filter nor the float64 filter certifies them and the expansion
arithmetic decides (Sec. 3.2.3, Eq. 4 in sign form).  The results must
match the oracle's big-integer predicates bit for bit, and the device
counter of expansion evaluations must show that stage ran.

Distance: the FP64 recomputation of both sides rounds at the frame scale
(about 2^20), so on these pairs both carry an absolute error of a few units
of 2^-53 * 2^20 (a few 1e-10, the size of the distance itself).  The bar here
is d == 0 exactly when the pair intersects, and agreement within
64 * 2^-53 * 2^21 absolute (the FP64 bound at this scale) otherwise.
"""
import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = synth.near_coplanar_face_pairs(60)
ABS_FRAME = 64 * 2.0 ** -53 * 2.0 ** 21
I1 = np.array([[0, 1, 2]], np.uint32)


@pytest.fixture(scope="module")
def ctx(g3d):
    c = g3d.Context(0, time_limit_ms=10000)
    yield c
    c.close()


def _distractors(rng, centre, n):
    """n small integer faces 2^18 away from `centre` (never nearest, never
    touching): they only give the BVH a few leaves to prune."""
    V = (np.asarray(centre) + rng.integers(1 << 18, (1 << 18) + 4096, size=(n, 3, 3))).reshape(-1, 3)
    return V.astype(np.float64)


def _run(ctx, pairs):
    hs = ctx.mesh_load_many([m for p in pairs for m in p], copy_fp64_master=True)
    ctx.mesh_build_bvh_many(hs)
    qs = [(hs[2 * k], hs[2 * k + 1], 1) for k in range(len(pairs))] + \
         [(hs[2 * k + 1], hs[2 * k], 0) for k in range(len(pairs))]
    ctx.stats_reset()
    d, h, s = ctx.batch(qs)
    st = ctx.stats()
    ctx.mesh_free_many(hs)
    n = len(pairs)
    assert (s == 0).all()
    return h[:n].astype(bool), d[n:], st


def test_single_faces_decided_exactly(ctx, orc):
    pairs = [((T1, I1), (T2, I1)) for T1, T2, _, _ in CASES]
    hit, dist, st = _run(ctx, pairs)
    assert st["exact_orients"] > 0, st
    for k, (T1, T2, exp, kind) in enumerate(CASES):
        ref = orc.tri_intersects(T1, T2)
        assert bool(hit[k]) == ref, (k, kind)
        if exp is not None:
            assert ref == exp
        assert (dist[k] == 0.0) == ref, (k, kind, dist[k])
        dref = orc.tri_distance(T1, T2)
        assert abs(dist[k] - dref) <= 1e-12 * dref + ABS_FRAME, (k, kind, dist[k], dref)


def test_small_meshes_decided_exactly(ctx, orc):
    """The same pairs inside small meshes (the pair's face plus distant
    faces), so the face pair is reached through the BVH traversal."""
    rng = np.random.default_rng(17)
    pairs, raw = [], []
    for T1, T2, _, _ in CASES:
        VA = np.concatenate([T1, _distractors(rng, T1[0], 7)])
        VB = np.concatenate([T2, _distractors(rng, -T2[0] / 2, 5)])
        IA = np.arange(len(VA), dtype=np.uint32).reshape(-1, 3)
        IB = np.arange(len(VB), dtype=np.uint32).reshape(-1, 3)
        pairs.append(((VA, IA), (VB, IB)))
        raw.append((VA, IA, VB, IB))
    hit, dist, st = _run(ctx, pairs)
    assert st["exact_orients"] > 0, st
    for k, (VA, IA, VB, IB) in enumerate(raw):
        ref = orc.mesh_intersects_brute(VA, IA, VB, IB)
        assert bool(hit[k]) == ref, k
        assert ref == orc.tri_intersects(CASES[k][0], CASES[k][1])
        assert (dist[k] == 0.0) == ref, (k, dist[k])
