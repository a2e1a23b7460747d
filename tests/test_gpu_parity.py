"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: intersects bit-exact; distance |d - d_oracle| <= 1e-12 d_oracle + 1e-15
(the tolerance the operators are specified to; the FP64 recomputation and the
oracle differ only in rounding order, a few ulps of the local-frame scale).
"""
import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15


def close(d, ref):
    return abs(d - ref) <= REL * abs(ref) + ABS


@pytest.fixture(scope="module", params=[1, 2], ids=["levelsync", "persistent"])
def ctx(g3d, request):
    """Both traversal forms: level-synchronous (1, the default) and the
    persistent per-warp depth-first kernel (2)."""
    c = g3d.Context(0, time_limit_ms=5000, traversal=request.param)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_small_leaves(g3d):
    c = g3d.Context(0, leaf_size=2, warps_per_cta=2, ctas_per_sm=1, stack_depth=64, time_limit_ms=5000)
    yield c
    c.close()


def _check_pair(ctx, orc, VA, IA, VB, IB, master=True, brute=True):
    A = ctx.load_and_build(VA, IA, copy_fp64_master=master)
    B = ctx.load_and_build(VB, IB, copy_fp64_master=master)
    d = ctx.distance(A, B)
    x = ctx.intersects(A, B)
    d2 = ctx.distance(B, A)
    x2 = ctx.intersects(B, A)
    VA64, VB64 = np.asarray(VA, np.float64), np.asarray(VB, np.float64)
    if not master:  # the engine computed on the float32 rounding of the input
        VA64 = np.asarray(VA, np.float32).astype(np.float64)
        VB64 = np.asarray(VB, np.float32).astype(np.float64)
    if brute:
        ref = orc.mesh_distance_brute(VA64, IA, VB64, IB)
        refx = orc.mesh_intersects_brute(VA64, IA, VB64, IB)
    else:
        ref = orc.mesh_distance_pruned(VA64, IA, VB64, IB)
        refx = orc.mesh_intersects_pruned(VA64, IA, VB64, IB)
    ctx.mesh_free(A)
    ctx.mesh_free(B)
    assert x == refx and x2 == refx, (x, x2, refx)
    assert close(d, ref), (d, ref, d - ref)
    assert close(d2, ref), (d2, ref, d2 - ref)
    assert (d == 0.0) == x
    return d, x


@pytest.mark.parametrize("pair", ["A", "B"])
def test_icosphere_pairs_fp64(ctx, orc, pair):
    A, B = synth.small_pairs()[pair]
    d, x = _check_pair(ctx, orc, A.V, A.I, B.V, B.I, master=True)
    assert x == (pair == "B")


@pytest.mark.parametrize("pair", ["A", "B"])
def test_icosphere_pairs_fp32(ctx, orc, pair):
    A, B = synth.small_pairs()[pair]
    _check_pair(ctx, orc, A.V.astype(np.float32), A.I, B.V.astype(np.float32), B.I, master=False)


@pytest.mark.parametrize("k", [-40, 40])
@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("pair", ["A", "B"])
def test_power_of_two_scaling(ctx, orc, pair, fp64, k):
    """Scaling both meshes by 2^k is exact in binary floating point and
    multiplies the distance by 2^k exactly (the square root of 2^(2k) d^2 is
    2^k d).  The scaled pair, far from unit magnitude, must meet the parity
    bar against the oracle on the scaled input, give the same intersects
    answer, and give 2^k times the unscaled distance bit for bit: the float32
    error bounds and the FP64 stage hold at any scale."""
    A, B = synth.small_pairs()[pair]
    VA, VB = (A.V, B.V) if fp64 else (A.V.astype(np.float32), B.V.astype(np.float32))
    a, b = ctx.load_and_build(VA, A.I, copy_fp64_master=fp64), ctx.load_and_build(VB, B.I, copy_fp64_master=fp64)
    d0, x0 = ctx.distance(a, b), ctx.intersects(a, b)
    ctx.mesh_free(a)
    ctx.mesh_free(b)
    s = VA.dtype.type(2.0 ** k)
    d1, x1 = _check_pair(ctx, orc, VA * s, A.I, VB * s, B.I, master=fp64)
    assert x1 == x0 == (pair == "B")
    assert d1 == d0 * 2.0 ** k, (d1, d0 * 2.0 ** k)


def test_icosphere_closed_form(ctx):
    V, I = synth.icosphere(3, 1.0, 0.0, None, vertex_on_x=True)
    A = ctx.load_and_build(V, I)
    for c in (2.5, 3.0, 2.0 + 2 ** -20):
        B = ctx.load_and_build(V + np.array([c, 0.0, 0.0]), I)
        assert close(ctx.distance(A, B), c - 2.0)
        assert not ctx.intersects(A, B)
        ctx.mesh_free(B)
    ctx.mesh_free(A)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("sep", [0.0, 0.35, 0.9, 2.5])
def test_random_soups(ctx, orc, seed, sep):
    rng = np.random.default_rng(100 + seed)
    na, nb = int(rng.integers(1, 120)), int(rng.integers(1, 120))
    A = synth.tiny_random_mesh(na, rng, spread=0.6, size=0.25)
    B = synth.tiny_random_mesh(nb, rng, spread=0.6, size=0.25)
    B.V = B.V + np.array([sep, 0.1, -0.05])
    _check_pair(ctx, orc, A.V, A.I, B.V, B.I, master=bool(seed % 2))


@pytest.fixture(scope="module")
def ctx_coarse_morton(g3d):
    c = g3d.Context(0, leaf_size=8, morton_bits=8, time_limit_ms=5000)
    yield c
    c.close()


@pytest.mark.parametrize("seed", range(4))
def test_random_soups_coarse_morton(ctx_coarse_morton, orc, seed):
    """8-bit Morton axes (24-bit keys, 3 sort passes): a coarser order, the
    same exact results."""
    rng = np.random.default_rng(300 + seed)
    A = synth.tiny_random_mesh(400, rng, spread=1.0, size=0.12)
    B = synth.tiny_random_mesh(350, rng, spread=1.0, size=0.12)
    B.V = B.V + np.array([0.4 * seed, 0.05, 0.0])
    _check_pair(ctx_coarse_morton, orc, A.V, A.I, B.V, B.I, master=bool(seed % 2))


@pytest.mark.parametrize("seed", range(4))
def test_random_soups_small_leaves(ctx_small_leaves, orc, seed):
    rng = np.random.default_rng(200 + seed)
    A = synth.tiny_random_mesh(300, rng, spread=1.0, size=0.15)
    B = synth.tiny_random_mesh(257, rng, spread=1.0, size=0.15)
    B.V = B.V + np.array([0.5 * seed, 0.0, 0.0])
    _check_pair(ctx_small_leaves, orc, A.V, A.I, B.V, B.I, master=False)


def _golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tri_pair_closed_forms.txt")
    out = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [x.strip() for x in line.split("|")]
        out.append((f[0], np.array(f[1].split(), float).reshape(3, 3), np.array(f[2].split(), float).reshape(3, 3),
                    float(f[3]), bool(int(f[4]))))
    return out


@pytest.mark.parametrize("case", _golden(), ids=[c[0] for c in _golden()])
def test_closed_form_face_pairs(ctx, case):
    """Degenerate, touching and coplanar single-face meshes (both dtypes)."""
    name, T1, T2, d, x = case
    I = np.array([[0, 1, 2]], np.uint32)
    for dt, master in ((np.float64, True), (np.float32, False)):
        A = ctx.load_and_build(T1.astype(dt), I, copy_fp64_master=master)
        B = ctx.load_and_build(T2.astype(dt), I, copy_fp64_master=master)
        assert ctx.intersects(A, B) == x, (name, dt)
        assert ctx.intersects(B, A) == x, (name, dt)
        got = ctx.distance(A, B)
        assert close(got, d), (name, dt, got, d)
        ctx.mesh_free(A)
        ctx.mesh_free(B)


def test_integer_grid_degeneracies(ctx, orc):
    """Faces on a small integer grid: many coplanar, collinear, touching and
    degenerate pairs, where every decision needs the exact stage."""
    rng = np.random.default_rng(7)
    for trial in range(6):
        nA, nB = 40, 40
        VA = rng.integers(-2, 3, (3 * nA, 3)).astype(np.float32)
        VB = rng.integers(-2, 3, (3 * nB, 3)).astype(np.float32) + np.float32(trial % 3)
        IA = np.arange(3 * nA, dtype=np.uint32).reshape(-1, 3)
        IB = np.arange(3 * nB, dtype=np.uint32).reshape(-1, 3)
        _check_pair(ctx, orc, VA, IA, VB, IB, master=False)


@pytest.mark.parametrize("nt", [1, 2, 3, 7, 8, 9, 17, 1000])
def test_ragged_sizes(ctx, orc, nt):
    rng = np.random.default_rng(nt)
    A = synth.tiny_random_mesh(nt, rng, spread=1.0, size=0.3)
    B = synth.tiny_random_mesh(max(1, nt // 2), rng, spread=1.0, size=0.3)
    B.V = B.V + np.array([1.2, 0.0, 0.0])
    _check_pair(ctx, orc, A.V, A.I, B.V, B.I, master=True)


def test_input_errors(ctx, g3d):
    from paper_1808_09571_gb300.geo3d import G3DError
    V = np.zeros((3, 3))
    I = np.array([[0, 1, 2]], np.uint32)
    with pytest.raises(G3DError) as e:
        ctx.mesh_load(V, np.zeros((0, 3), np.uint32))
    assert e.value.code == -4
    with pytest.raises(G3DError) as e:
        ctx.mesh_load(V, np.array([[0, 1, 3]], np.uint32))
    assert e.value.code == -3
    Vn = V.copy()
    Vn[1, 2] = np.nan
    with pytest.raises(G3DError) as e:
        ctx.mesh_load(Vn, I)
    assert e.value.code == -2
    Vr = V.copy()
    Vr[0, 0] = 1e30
    with pytest.raises(G3DError) as e:
        ctx.mesh_load(Vr, I)
    assert e.value.code == -9
    m = ctx.mesh_load(V, I)
    with pytest.raises(G3DError) as e:
        ctx.distance(m, m)
    assert e.value.code == -10
    ctx.mesh_free(m)


def test_tube_ellipsoid_reduced(ctx, orc):
    """The large plain-method workload at reduced resolution: tube (2,048
    segments, 65,536 faces) against a 128 x 128 ore body, 6 placements."""
    ore, tI, tubes, info = synth.large_placements(n_place=6, seed=2001, n_steps=2048, n_lon=128, n_lat=128)
    O = ctx.load_and_build(ore.V, ore.I, copy_fp64_master=False)
    for k, V in enumerate(tubes):
        T = ctx.load_and_build(V, tI, copy_fp64_master=False)
        d, x = ctx.distance(T, O), ctx.intersects(T, O)
        V64 = V.astype(np.float64)
        O64 = ore.V.astype(np.float64)
        ref = orc.mesh_distance_pruned(V64, tI, O64, ore.I)
        refx = orc.mesh_intersects_pruned(V64, tI, O64, ore.I)
        assert x == refx, k
        assert close(d, ref), (k, d, ref)
        ctx.mesh_free(T)
    ctx.mesh_free(O)


def test_batch_matches_single(ctx):
    rng = np.random.default_rng(77)
    meshes = []
    for k in range(8):
        M = synth.tiny_random_mesh(int(rng.integers(5, 400)), rng, spread=1.0, size=0.2)
        M.V = M.V + np.array([0.8 * k, 0.0, 0.0])
        meshes.append(ctx.load_and_build(M.V.astype(np.float32), M.I, copy_fp64_master=False))
    qs = [(meshes[int(rng.integers(0, 8))], meshes[int(rng.integers(0, 8))], int(rng.integers(0, 2)))
          for _ in range(64)]
    d, h, s = ctx.batch(qs)
    assert (s == 0).all()
    for i, (a, b, op) in enumerate(qs):
        if op == 0:
            assert d[i] == ctx.distance(a, b)
            assert h[i] == (d[i] == 0.0)
        else:
            assert bool(h[i]) == ctx.intersects(a, b)
    for m in meshes:
        ctx.mesh_free(m)


def test_stats_counters(ctx):
    A, B = synth.small_pairs()["A"]
    a = ctx.load_and_build(A.V.astype(np.float32), A.I, copy_fp64_master=False)
    b = ctx.load_and_build(B.V.astype(np.float32), B.I, copy_fp64_master=False)
    ctx.stats_reset()
    ctx.distance(a, b)
    st = ctx.stats()
    assert st["node_pairs"] > 0 and st["leaf_pairs"] > 0
    assert 0 < st["tri_tests"] <= st["tri_prefilter"] <= 1280 * 1280
    assert 1 <= st["fp64_tests"] <= st["candidates"]
    ctx.mesh_free(a)
    ctx.mesh_free(b)


def test_batched_build_matches_single_builds(ctx, orc):
    """Meshes built together by one batched build answer exactly as meshes
    built one by one (same tree per mesh: the mesh index only prefixes the
    sort key)."""
    rng = np.random.default_rng(91)
    ms = []
    for k in range(7):
        M = synth.tiny_random_mesh(int(rng.integers(1, 3000)), rng, spread=1.5, size=0.2)
        M.V = (M.V + np.array([0.9 * k, 0.0, 0.0])).astype(np.float32)
        ms.append(M)
    many = ctx.mesh_load_many([(M.V, M.I) for M in ms], copy_fp64_master=False)
    ctx.mesh_build_bvh_many(many)
    single = [ctx.load_and_build(M.V, M.I, copy_fp64_master=False) for M in ms]
    for i in range(len(ms) - 1):
        j = i + 1
        a = ctx.distance(many[i], many[j])
        b = ctx.distance(single[i], single[j])
        assert a == b
        assert ctx.intersects(many[i], many[j]) == ctx.intersects(single[i], single[j])
        ref = orc.mesh_distance_pruned(ms[i].V.astype(np.float64), ms[i].I, ms[j].V.astype(np.float64), ms[j].I)
        assert close(a, ref)
    for m in many + single:
        ctx.mesh_free(m)


def test_load_many_reports_each_mesh(ctx, g3d):
    from paper_1808_09571_gb300.geo3d import G3DError
    V = np.zeros((3, 3), np.float32)
    I = np.array([[0, 1, 2]], np.uint32)
    bad = np.array([[0, 1, 5]], np.uint32)
    with pytest.raises(G3DError) as e:
        ctx.mesh_load_many([(V, I), (V, bad), (V, I)])
    assert e.value.code == -3


def test_batch_links_distance_to_intersects(ctx, orc):
    """A batch holding both operators for the same mesh pairs (either order)
    answers exactly as the single queries."""
    rng = np.random.default_rng(5)
    ms, raw = [], []
    for k in range(6):
        M = synth.tiny_random_mesh(int(rng.integers(20, 600)), rng, spread=1.0, size=0.25)
        M.V = (M.V + np.array([0.6 * k, 0.0, 0.0])).astype(np.float32)
        raw.append(M)
        ms.append(ctx.load_and_build(M.V, M.I, copy_fp64_master=False))
    qs = []
    for i in range(5):
        qs += [(ms[i], ms[i + 1], 0), (ms[i + 1], ms[i], 1)]
    d, h, s = ctx.batch(qs)
    assert (s == 0).all()
    for k in range(0, len(qs), 2):
        a, b, _ = qs[k]
        ref = orc.mesh_distance_brute(raw[k // 2].V.astype(np.float64), raw[k // 2].I,
                                      raw[k // 2 + 1].V.astype(np.float64), raw[k // 2 + 1].I)
        assert close(d[k], ref)
        assert d[k] == ctx.distance(a, b)
        assert bool(h[k + 1]) == (ref == 0.0) == ctx.intersects(b, a)
    for m in ms:
        ctx.mesh_free(m)


def test_witness_is_the_oracle_argmin(ctx, orc):
    """g3d_batch_ex's witness (input face ids) against the oracle's brute
    force argmin, which takes the lowest (i, j) among ties.  The distance is
    unique; the witness must attain it (oracle distance of the witness pair
    within the tolerance) and, when the minimum is not tied within rounding,
    be the oracle's pair exactly."""
    rng = np.random.default_rng(77)
    meshes, queries, refs = [], [], []
    sp = synth.small_pairs()
    for key in ("A", "B"):
        MA, MB = sp[key]
        meshes += [(MA.V, MA.I), (MB.V, MB.I)]
    for k in range(8):
        A = synth.tiny_random_mesh(int(rng.integers(20, 300)), rng)
        B = synth.tiny_random_mesh(int(rng.integers(20, 300)), rng)
        B = synth.Mesh(B.V + np.array([2.0 + 0.15 * k, 0.1, 0.0]), B.I)  # mostly separated
        meshes += [(A.V, A.I), (B.V, B.I)]
    hs = [ctx.mesh_load(V, I) for V, I in meshes]
    for h in hs:
        ctx.mesh_build_bvh(h)
    qs = [(hs[2 * i], hs[2 * i + 1], 0) for i in range(len(hs) // 2)]
    d, w, s, cl = ctx.batch_witness(qs)
    assert (s == 0).all()
    exact = n_sep = 0
    for i in range(len(qs)):
        VA, IA = meshes[2 * i]
        VB, IB = meshes[2 * i + 1]
        ref, ai, aj = orc.mesh_distance_brute(VA, IA, VB, IB, return_arg=True)
        assert close(d[i], ref), (i, d[i], ref)
        if ref == 0.0:
            assert w[i] == -1 and cl[i] == -1
            continue
        n_sep += 1
        wa, wb = int(w[i]) >> 32, int(w[i]) & 0xffffffff
        assert 0 <= wa < len(IA) and 0 <= wb < len(IB)
        dw = orc.tri_distance(VA[IA[wa]], VB[IB[wb]])
        assert close(dw, ref), (i, dw, ref)
        exact += (wa, wb) == (ai, aj)
        assert 0 <= cl[i] < 4096
    # icosphere pair A may be tied within rounding (faces share vertices);
    # the soups have no shared vertices, so their argmin is unique
    assert n_sep >= 7 and exact >= n_sep - 1, (exact, n_sep)
    for h in hs:
        ctx.mesh_free(h)
