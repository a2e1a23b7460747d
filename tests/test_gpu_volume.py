"""Mesh volume (Eq. 2) on the GPU against the exact oracle.

Tolerance: each face term is a triple product evaluated in FP64 (two
differences, a cross product and a dot product), whose rounding error is at
most a few units of 2^-53 times |u| |v - u| |w - u|; the compensated sum adds
about one unit of the result.  The tests allow 16 units of 2^-53 times
sum_i |u_i| |v_i - u_i| |w_i - u_i| (the oracle's rounding_scale times 6)."""
import numpy as np
import pytest

from oracle import volume as VO
from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def tol(V, I):
    return 16 * EPS * 6 * VO.rounding_scale(V, I) + 1e-300


@pytest.fixture(scope="module")
def ctx(g3d):
    c = g3d.Context(0, time_limit_ms=10000)
    yield c
    c.close()


def test_closed_forms_exact(ctx):
    V, I = synth.box_mesh(2.0, 3.0, 5.0, origin=(-1.0, 0.5, 2.0))
    m = ctx.mesh_load(V, I)
    assert ctx.volume(m) == 30.0
    T = np.array([[0, 0, 0], [2, 0, 0], [0, 3, 0], [0, 0, 0.5]], np.float32)
    TI = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.uint32)
    t = ctx.mesh_load(T, TI)
    assert ctx.volume(t) == 0.5
    ctx.mesh_free(m)
    ctx.mesh_free(t)


@pytest.mark.parametrize("case", ["ore500", "ellipsoid_256", "icosphere_fp64", "tube"])
def test_against_exact_oracle(ctx, case):
    if case == "ore500":
        o = synth.small_ore_body()
        V, I = o.V, o.I
    elif case == "ellipsoid_256":
        V, I = synth.uv_ellipsoid((40.0, 25.0, 15.0), 256, 256, jitter=0.01, seed=3)
        V = V.astype(np.float32)
    elif case == "icosphere_fp64":
        A, _ = synth.small_pairs()["A"]
        V, I = A.V, A.I
    else:  # an open surface far from the origin: the formula's value
        m, _ = synth.drill_hole(2000, seed=7)
        V, I = (m.V + np.array([100.0, -50.0, 20.0])).astype(np.float32), m.I
    h = ctx.mesh_load(V, I)
    got = ctx.volume(h)
    ref = VO.volume_exact(V, I)
    assert abs(got - float(ref)) <= tol(V, I), (case, got, float(ref), tol(V, I))
    ctx.mesh_free(h)


def test_orientation_batch_and_determinism(ctx):
    """Reversed faces give exactly the negated volume; a batch equals the
    single calls bit for bit; repeated calls repeat bit for bit."""
    import torch
    o = synth.small_ore_body()
    meshes = [(o.V, o.I), (o.V, o.I[:, ::-1].copy())]
    rng = np.random.default_rng(2)
    for k in range(6):
        V, I = synth.uv_ellipsoid(tuple(rng.uniform(1, 30, 3)), int(rng.integers(8, 300)),
                                  int(rng.integers(8, 300)), jitter=0.02, seed=k)
        meshes.append((V.astype(np.float32) + rng.normal(0, 50, 3).astype(np.float32), I))
    hs = [ctx.mesh_load(V, I, copy_fp64_master=False) for V, I in meshes]
    vb = ctx.volume(hs)
    assert vb[1] == -vb[0]
    for h, v in zip(hs, vb):
        assert ctx.volume(h) == v
    for _ in range(3):
        np.testing.assert_array_equal(ctx.volume(hs), vb)
    dev = torch.empty(len(hs), dtype=torch.float64, device="cuda")
    ctx.volume(hs, out=dev)
    ctx.sync()
    np.testing.assert_array_equal(dev.cpu().numpy(), vb)
    for (V, I), v in zip(meshes[2:], vb[2:]):
        assert abs(v - VO.volume(V, I)) <= tol(V, I)
    for h in hs:
        ctx.mesh_free(h)


@pytest.mark.parametrize("case", ["ore500", "ellipsoid_256", "tube_far", "box_offset"])
def test_float32_meshes_rounded_from_the_exact_value(ctx, case):
    """Float32 meshes whose coordinates span at most 50 binary orders of
    magnitude are summed exactly (integers on the mesh's coordinate grid):
    the result is the exact Eq. 2 value with two roundings (the conversion
    of the exact sum, the division by 6), so within 2 units in the last
    place of the exact value -- far inside the FP64 bound."""
    if case == "ore500":
        o = synth.small_ore_body()
        V, I = o.V.astype(np.float32), o.I
    elif case == "ellipsoid_256":
        V, I = synth.uv_ellipsoid((40.0, 25.0, 15.0), 256, 256, jitter=0.01, seed=3)
        V = V.astype(np.float32)
    elif case == "tube_far":
        m, _ = synth.drill_hole(2000, seed=7)
        V, I = (m.V + np.array([100.0, -50.0, 20.0])).astype(np.float32), m.I
    else:
        V, I = synth.box_mesh(2.5, 3.25, 0.75, origin=(1e3, -2e2, 7.0))
        V = V.astype(np.float32)
    h = ctx.mesh_load(V, I, copy_fp64_master=False)
    got = ctx.volume(h)
    ref = VO.volume_exact(V, I)
    refd = float(ref)
    assert abs(got - refd) <= 2 * np.spacing(abs(refd)), (case, got, refd)
    ctx.mesh_free(h)


def test_wide_coordinate_range_takes_the_fp64_path(ctx):
    """A float32 mesh with coordinates from 1e-30 to 1e3 (beyond the 50 bits
    of the integer grid) is summed in FP64 and meets the FP64 bound."""
    o = synth.small_ore_body()
    V = o.V.astype(np.float32).copy()
    V[3, 0] = np.float32(1e-30)
    h = ctx.mesh_load(V, o.I, copy_fp64_master=False)
    got = ctx.volume(h)
    assert abs(got - float(VO.volume_exact(V, o.I))) <= tol(V, o.I)
    ctx.mesh_free(h)
