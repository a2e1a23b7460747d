"""Line strings and collections as meshes (geo3d.linestring_mesh,
geo3d.collection_mesh) in the CPU oracle, pinned to closed forms: parallel
and skew straight line strings, crossing ones, a point over a face, a line
string through a face, and a collection's distance as the minimum over its
parts (Sec. 2.2 geometry types; Sec. 3.2.2 cases ii-iii; Sec. 3.2.3)."""
import numpy as np
import pytest

from paper_1808_09571_gb300 import geo3d


def straight(p0, p1, n):
    t = np.linspace(0.0, 1.0, n)[:, None]
    return (1 - t) * np.asarray(p0, float) + t * np.asarray(p1, float)


def test_linestring_mesh_layout():
    V, I = geo3d.linestring_mesh(np.zeros((5, 3)))
    assert I.tolist() == [[0, 1, 1], [1, 2, 2], [2, 3, 3], [3, 4, 4]]
    V, I = geo3d.linestring_mesh(np.ones((1, 3), np.float32))
    assert V.dtype == np.float32 and I.tolist() == [[0, 0, 0]]
    with pytest.raises(ValueError):
        geo3d.linestring_mesh(np.zeros((0, 3)))


@pytest.mark.parametrize("h", [0.5, 1e-3, 3.0])
def test_parallel_line_strings(orc, h):
    """Two straight line strings along x, offset by h in y (overlapping x
    ranges, vertices not aligned): the distance is exactly h."""
    A = geo3d.linestring_mesh(straight((0, 0, 0), (8, 0, 0), 9))
    B = geo3d.linestring_mesh(straight((0.25, h, 0), (6.25, h, 0), 7))
    assert orc.mesh_distance_brute(*A, *B) == pytest.approx(h, rel=1e-15)
    assert not orc.mesh_intersects_brute(*A, *B)


def test_skew_and_crossing_line_strings(orc):
    A = geo3d.linestring_mesh(straight((-4, 0, 0), (4, 0, 0), 5))     # along x at z = 0
    B = geo3d.linestring_mesh(straight((0.5, -3, 2), (0.5, 3, 2), 4))  # along y at z = 2
    assert orc.mesh_distance_brute(*A, *B) == pytest.approx(2.0, rel=1e-15)
    C = geo3d.linestring_mesh(straight((0.5, -3, 0), (0.5, 3, 0), 4))  # crosses A at (0.5, 0, 0)
    assert orc.mesh_intersects_brute(*A, *C) and orc.mesh_distance_brute(*A, *C) == 0.0


def test_point_and_line_string_against_a_face(orc):
    T = (np.array([[0, 0, 0], [4, 0, 0], [0, 4, 0]], float), np.array([[0, 1, 2]], np.uint32))
    P = geo3d.linestring_mesh(np.array([[1.0, 1.0, 0.75]]))
    assert orc.mesh_distance_brute(*P, *T) == pytest.approx(0.75, rel=1e-15)
    L = geo3d.linestring_mesh(np.array([[1.0, 1.0, 2.0], [1.0, 1.0, -2.0], [3.0, 3.0, -2.0]]))
    assert orc.mesh_intersects_brute(*L, *T) and orc.mesh_distance_brute(*L, *T) == 0.0
    # ends on the face's edge: closed sets touch
    E = geo3d.linestring_mesh(np.array([[2.0, 0.0, 0.0], [2.0, -1.0, 0.0]]))
    assert orc.mesh_intersects_brute(*E, *T)


def test_collection_is_the_minimum_over_its_parts(orc):
    rng = np.random.default_rng(3)
    parts = [geo3d.linestring_mesh(rng.normal(0, 1, (6, 3)) + [5, 0, 0]),
             geo3d.linestring_mesh(np.array([[0.0, 4.0, 0.0]])),
             (rng.normal(0, 1, (6, 3)) + [0, -5, 0], np.array([[0, 1, 2], [3, 4, 5]], np.uint32))]
    G = geo3d.collection_mesh(parts)
    B = (rng.normal(0, 0.5, (9, 3)), np.arange(9, dtype=np.uint32).reshape(3, 3))
    whole = orc.mesh_distance_brute(*G, *B)
    assert whole == min(orc.mesh_distance_brute(np.asarray(V, float), I, *B) for V, I in parts)
