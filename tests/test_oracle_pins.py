"""Pins of the CPU oracle against facts it does not compute itself:
hand-derived closed forms, an independent exact intersection method, an
independent convex-QP distance, exact rational determinants, geometric
invariants and the brute-force / pruned agreement."""
import os
from fractions import Fraction

import numpy as np
import pytest

from exact_ref import frac_orient3d, minkowski_intersects, qp_distance
from paper_1808_09571_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tri_pair_closed_forms.txt")


def load_golden():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, t1, t2, d, x, _why = [f.strip() for f in line.split("|")]
        cases.append((name, np.array(t1.split(), float), np.array(t2.split(), float),
                      float(d), bool(int(x))))
    return cases


GOLD = load_golden()


@pytest.mark.parametrize("case", GOLD, ids=[c[0] for c in GOLD])
def test_closed_form_cases(orc, case):
    name, T1, T2, d, x = case
    assert orc.tri_intersects(T1, T2) == x
    assert orc.tri_intersects(T2, T1) == x
    got = orc.tri_distance(T1, T2)
    assert got == pytest.approx(d, rel=1e-15, abs=1e-300), name
    assert orc.tri_distance(T2, T1) == pytest.approx(d, rel=1e-15, abs=1e-300), name


def test_point_triangle_closed_forms(orc):
    a, b, c = np.array([0., 0, 0]), np.array([3., 0, 0]), np.array([0., 3, 0])
    # above the interior: |h|
    assert orc.pt_tri_d2([1, 1, -2.5], a, b, c) == 6.25
    # coplanar outside, nearest a vertex
    assert orc.pt_tri_d2([-3, -4, 0], a, b, c) == 25.0
    # coplanar outside, nearest the hypotenuse interior: distance |x+y-3|/sqrt 2
    assert orc.pt_tri_d2([3, 3, 0], a, b, c) == pytest.approx(4.5, rel=1e-15)
    # above and outside: nearest edge point, Pythagoras
    assert orc.pt_tri_d2([1, -2, 2], a, b, c) == pytest.approx(8.0, rel=1e-15)
    # on the triangle
    assert orc.pt_tri_d2([1, 1, 0], a, b, c) == 0.0
    assert orc.pt_tri_d2([1.5, 1.5, 0], a, b, c) == 0.0
    # degenerate triangle (segment)
    assert orc.pt_tri_d2([1, 1, 0], a, b, [1.5, 0, 0]) == 1.0


def test_segment_closed_forms(orc):
    # skew perpendicular
    assert orc.seg_seg_d2([-1, 0, 0], [1, 0, 0], [0, -1, 2], [0, 1, 2]) == 4.0
    # skew, closest point outside one segment: clamps to the endpoint
    assert orc.seg_seg_d2([-1, 0, 0], [1, 0, 0], [3, -1, 2], [3, 1, 2]) == pytest.approx(8.0)
    # parallel overlapping: the perpendicular distance
    assert orc.seg_seg_d2([0, 0, 0], [2, 0, 0], [1, 1, 0], [3, 1, 0]) == 1.0
    # collinear disjoint: endpoint gap
    assert orc.seg_seg_d2([0, 0, 0], [1, 0, 0], [2.5, 0, 0], [4, 0, 0]) == 2.25
    # degenerate segment
    assert orc.seg_seg_d2([0, 0, 0], [0, 0, 0], [1, -1, 1], [1, 1, 1]) == 2.0
    assert orc.pt_seg_d2([0, 5, 0], [0, 0, 0], [0, 0, 0]) == 25.0


@pytest.mark.parametrize("h", [1e-6, 0.25, 3.0])
def test_parallel_planes(orc, h):
    rng = np.random.default_rng(7)
    for _ in range(20):
        T1 = np.c_[rng.uniform(-1, 1, (3, 2)), np.zeros(3)]
        # overlapping shadows: T2's shadow contains T1's centroid
        c = T1.mean(0)
        w = rng.uniform(0.05, 0.3)
        T2 = np.c_[c[:2] + w * np.array([[-1.0, -1.0], [2.0, -1.0], [-1.0, 2.0]]), np.full(3, h)]
        assert orc.tri_distance(T1, T2) == pytest.approx(h, rel=1e-12)


def test_icosphere_pair_support_function(orc):
    """A vertex on +x and its antipode on -x: copies c apart along x are
    exactly c - 2r apart (the support planes x = r and x = c - r meet the
    meshes only in those vertices)."""
    V, I = synth.icosphere(3, 1.0, 0.0, None, vertex_on_x=True)
    for c in (2.0 + 2 ** -20, 2.5, 4.0):
        VB = V + np.array([c, 0.0, 0.0])
        d = orc.mesh_distance_pruned(V, I, VB, I)
        assert d == pytest.approx(c - 2.0, rel=1e-14, abs=1e-15)
        assert not orc.mesh_intersects_pruned(V, I, VB, I)
    VB = V + np.array([1.5, 0.0, 0.0])
    assert orc.mesh_intersects_pruned(V, I, VB, I)
    assert orc.mesh_distance_pruned(V, I, VB, I) == 0.0


def test_jittered_icosphere_bracket(orc):
    """Jittered spheres at centre distance c: every vertex radius lies in
    [0.95, 1.05], so c - 2.1 <= d <= c - 2 * 0.95 * cos(theta_max) with the
    facet angular radius theta_max < 0.2 rad for subdivision 3."""
    pairs = synth.small_pairs()
    A, B = pairs["A"]
    d = orc.mesh_distance_brute(A.V, A.I, B.V, B.I)
    assert 2.5 - 2.1 <= d <= 2.5 - 2 * 0.95 * np.cos(0.2)


def _rand_tri_pairs(rng, n, kind):
    out = []
    for _ in range(n):
        if kind == "int":  # small integers: many coplanar / touching cases
            T1 = rng.integers(-2, 3, (3, 3)).astype(float)
            T2 = rng.integers(-2, 3, (3, 3)).astype(float)
        elif kind == "dyadic":
            T1 = rng.integers(-8, 9, (3, 3)) / 8.0
            T2 = rng.integers(-8, 9, (3, 3)) / 8.0
        else:
            T1 = rng.uniform(-1, 1, (3, 3))
            T2 = rng.uniform(-1, 1, (3, 3)) + rng.uniform(-0.6, 0.6, 3)
        out.append((T1.reshape(9), T2.reshape(9)))
    return out


@pytest.mark.parametrize("kind,n", [("int", 250), ("dyadic", 150), ("real", 100)])
def test_intersects_vs_minkowski(orc, kind, n):
    rng = np.random.default_rng({"int": 1, "dyadic": 2, "real": 3}[kind])
    hits = 0
    for T1, T2 in _rand_tri_pairs(rng, n, kind):
        ref = minkowski_intersects(T1, T2)
        hits += ref
        assert orc.tri_intersects(T1, T2) == ref, (T1.tolist(), T2.tolist())
    assert 0 < hits < n  # both outcomes exercised


def test_intersects_constructed_degenerate(orc):
    """Touching configurations built exactly, checked against Minkowski."""
    rng = np.random.default_rng(11)
    for _ in range(60):
        T1 = rng.integers(-4, 5, (3, 3)).astype(float)
        choices = [(1, 0, 0), (0.5, 0.5, 0), (0.25, 0.25, 0.5), (0.5, 0.25, 0.25),
                   (0, 0.75, 0.25), (0.125, 0.375, 0.5)]
        bary = np.array(choices[int(rng.integers(0, len(choices)))])[rng.permutation(3)]
        p = bary @ T1
        T2 = np.stack([p, p + rng.integers(-2, 3, 3), p + rng.integers(-2, 3, 3)])
        ref = minkowski_intersects(T1.reshape(9), T2.reshape(9))
        assert orc.tri_intersects(T1.reshape(9), T2.reshape(9)) == ref


@pytest.mark.parametrize("kind", ["int", "real"])
def test_distance_vs_qp(orc, kind):
    rng = np.random.default_rng(5 if kind == "int" else 6)
    n = 0
    for T1, T2 in _rand_tri_pairs(rng, 120, kind):
        d = orc.tri_distance(T1, T2)
        ref = qp_distance(T1, T2)
        if orc.tri_intersects(T1, T2):
            assert d == 0.0 and ref < 1e-7
            continue
        n += 1
        assert d == pytest.approx(ref, rel=1e-6, abs=1e-8), (T1.tolist(), T2.tolist())
    assert n > 20


def test_distance_zero_iff_intersects(orc):
    rng = np.random.default_rng(9)
    for T1, T2 in _rand_tri_pairs(rng, 300, "int"):
        assert (orc.tri_distance(T1, T2) == 0.0) == orc.tri_intersects(T1, T2)


def test_orient_bigint_vs_fractions(orc):
    rng = np.random.default_rng(3)
    for _ in range(300):
        e = rng.integers(-60, 60, (4, 3))
        P = rng.uniform(-1, 1, (4, 3)) * np.exp2(e)
        if rng.random() < 0.3:  # force coplanarity with exact dyadics
            P = rng.integers(-3, 4, (4, 3)).astype(float) * 2.0 ** rng.integers(-30, 30)
            P[3] = P[0] + (P[1] - P[0]) + (P[2] - P[0])
        assert orc.orient3d(*P) == frac_orient3d(*P)
    # extreme exponent spread within the supported range
    a = np.array([2.0 ** 190, 1.0, 0.0])
    b = np.array([2.0 ** -190, 3.0, 1.0])
    c = np.array([1.0, 2.0 ** -150, 2.0 ** 150])
    d = np.array([0.5, 0.25, -2.0 ** -199])
    assert orc.orient3d(a, b, c, d) == frac_orient3d(a, b, c, d)
    # orient2d
    for _ in range(200):
        P = rng.integers(-5, 6, (3, 2)).astype(float) * 2.0 ** rng.integers(-40, 40)
        F = [[Fraction(float(x)) for x in p] for p in P]
        det = (F[0][0] - F[2][0]) * (F[1][1] - F[2][1]) - (F[0][1] - F[2][1]) * (F[1][0] - F[2][0])
        assert orc.orient2d(*P) == (det > 0) - (det < 0)


def _perturb_meshes(rng, A, B, how):
    VA, VB = A.V.copy(), B.V.copy()
    if how == "translate":
        t = rng.integers(-64, 64, 3) / 4.0
        return VA + t, VB + t
    if how == "reflect":
        s = np.array([-1.0, 1.0, -1.0])
        return VA * s, VB * s
    if how == "permute":
        p = [2, 0, 1]
        return VA[:, p], VB[:, p]
    raise ValueError(how)


@pytest.mark.parametrize("how", ["translate", "reflect", "permute"])
def test_rigid_motion_invariance(orc, how):
    rng = np.random.default_rng(21)
    A = synth.tiny_random_mesh(30, rng, spread=1.0, size=0.4)
    B = synth.tiny_random_mesh(30, rng, spread=1.0, size=0.4)
    B.V = B.V + np.array([0.7, 0.0, 0.0])
    d0 = orc.mesh_distance_brute(A.V, A.I, B.V, B.I)
    x0 = orc.mesh_intersects_brute(A.V, A.I, B.V, B.I)
    VA, VB = _perturb_meshes(rng, A, B, how)
    d1 = orc.mesh_distance_brute(VA, A.I, VB, B.I)
    x1 = orc.mesh_intersects_brute(VA, A.I, VB, B.I)
    assert x0 == x1
    if how in ("translate", "reflect"):
        assert d1 == d0  # exact: same differences, same rounding
    else:
        assert d1 == pytest.approx(d0, rel=1e-13, abs=1e-15)


def test_symmetry_and_order_invariance(orc):
    rng = np.random.default_rng(22)
    for sep in (0.0, 0.5, 1.5):
        A = synth.tiny_random_mesh(25, rng, spread=1.0, size=0.4)
        B = synth.tiny_random_mesh(25, rng, spread=1.0, size=0.4)
        B.V = B.V + np.array([sep, 0.0, 0.0])
        d = orc.mesh_distance_brute(A.V, A.I, B.V, B.I)
        x = orc.mesh_intersects_brute(A.V, A.I, B.V, B.I)
        assert orc.mesh_intersects_brute(B.V, B.I, A.V, A.I) == x
        assert orc.mesh_distance_brute(B.V, B.I, A.V, A.I) == pytest.approx(d, rel=1e-13, abs=1e-15)
        p = rng.permutation(A.nt)
        assert orc.mesh_distance_brute(A.V, A.I[p], B.V, B.I) == d
        assert (d == 0.0) == x


def test_pruned_equals_brute(orc):
    pairs = synth.small_pairs()
    for key, (A, B) in pairs.items():
        assert orc.mesh_distance_pruned(A.V, A.I, B.V, B.I) == orc.mesh_distance_brute(A.V, A.I, B.V, B.I)
        assert orc.mesh_intersects_pruned(A.V, A.I, B.V, B.I) == orc.mesh_intersects_brute(A.V, A.I, B.V, B.I)
    rng = np.random.default_rng(31)
    for sep in (0.2, 0.8, 1.6, 3.0):
        A = synth.tiny_random_mesh(300, rng, spread=1.0, size=0.15)
        B = synth.tiny_random_mesh(300, rng, spread=1.0, size=0.15)
        B.V = B.V + np.array([sep, 0.3, 0.0])
        assert orc.mesh_distance_pruned(A.V, A.I, B.V, B.I) == orc.mesh_distance_brute(A.V, A.I, B.V, B.I)
        assert orc.mesh_intersects_pruned(A.V, A.I, B.V, B.I) == orc.mesh_intersects_brute(A.V, A.I, B.V, B.I)


def test_batch_threads_match_single(orc):
    rng = np.random.default_rng(41)
    meshes = []
    for k in range(6):
        M = synth.tiny_random_mesh(80, rng, spread=1.0, size=0.2)
        M.V = M.V + np.array([0.9 * k, 0.0, 0.0])
        meshes.append((M.V, M.I))
    qa = [0, 1, 2, 3, 0, 5]
    qb = [1, 2, 3, 4, 5, 4]
    op = [0, 1, 0, 1, 0, 0]
    out = orc.batch_pruned(meshes, qa, qb, op, nthreads=3)
    for q in range(len(qa)):
        (VA, IA), (VB, IB) = meshes[qa[q]], meshes[qb[q]]
        if op[q] == 0:
            assert out[q] == orc.mesh_distance_brute(VA, IA, VB, IB)
        else:
            assert out[q] == float(orc.mesh_intersects_brute(VA, IA, VB, IB))
