"""Pins of the proposal oracle (oracle/proposal.py): the face order, the
cluster partition, the cluster statistics, the pair features and the top-k
selection, against facts it does not compute itself -- a hand-derived
single-face case (tests/golden/proposal_single_face.txt), the closed-surface
identity (the area-weighted normals of a closed, consistently oriented mesh
sum to zero), the Morton order of points on the corners of a box (the
lexicographic (x, y, z) order), counting, and invariance of the features
under a dyadic translation and a power-of-two scale of both meshes."""
import os

import numpy as np
import pytest

from oracle import proposal as P
from paper_1808_09571_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "proposal_single_face.txt")


def test_single_face_pair_features_by_hand():
    A = np.array([[0, 0, 0], [2, 0, 0], [0, 2, 0]], float)
    B = np.array([[0, 0, 2], [2, 0, 2], [0, 2, 2]], float)
    I = np.array([[0, 1, 2]])
    X = P.mesh_pair_features(A, I, B, I, 10).reshape(128, 12)
    want = np.zeros((128, 12))
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        side, c, vals = [f.strip() for f in line.split("|")]
        v = np.array(vals.split(), float)
        v[:9] /= np.sqrt(3.0)
        want[(0 if side == "A" else 64) + int(c)] = v
    np.testing.assert_allclose(X, want, rtol=0, atol=1e-15)


def test_cluster_partition_counts():
    for nt in (1, 5, 63, 64, 65, 127, 1000, 4097):
        r = P.cluster_ranges(nt)
        assert r[0][0] == 0 and r[-1][1] == nt
        assert all(r[c][1] == r[c + 1][0] for c in range(63))
        sizes = [b - a for a, b in r]
        assert sum(sizes) == nt
        assert set(sizes) <= {nt // 64, -(-nt // 64)}
        # position f is in cluster floor(64 f / nt)
        for f in range(0, nt, max(1, nt // 50)):
            c = 64 * f // nt
            assert r[c][0] <= f < r[c][1]


def test_closed_box_normals_sum_to_zero():
    V, I = synth.box_mesh(3.0, 2.0, 5.0, origin=(1.0, -2.0, 0.5))
    for bits in (8, 10):
        st = P.cluster_stats(V, I, P.morton_order(V, I, bits))
        total = sum(s["normal_sum"] for s in st if s["count"])
        area = sum(s["area"] for s in st if s["count"])
        assert np.array_equal(total, np.zeros(3))
        assert area == 2 * (3 * 2 + 3 * 5 + 2 * 5)
        assert sum(s["count"] for s in st) == len(I)
        # every face's normal points out of the box: its mean normal is the
        # outward axis of the face's side
        for s in st:
            if s["count"] == 1:
                n = s["normal_sum"] / s["area"]
                assert sorted(np.abs(n)) == [0.0, 0.0, 1.0]


def test_morton_order_of_box_corners():
    """Eight degenerate faces (points) on the corners of a box: every cell
    coordinate is 0 or 2^bits - 1, so the key order is the lexicographic
    (x, y, z) order of the corners."""
    corners = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], float) * [4.0, 2.0, 1.0]
    perm = np.random.default_rng(3).permutation(8)
    V = corners[perm]
    I = np.repeat(np.arange(8)[:, None], 3, axis=1)
    order = P.morton_order(V, I, 8)
    want = sorted(range(8), key=lambda f: tuple(V[f]))
    assert list(order) == want
    # equal keys keep the input order (faces 8..15 repeat faces 0..7)
    V2 = np.concatenate([V, V])
    I2 = np.concatenate([I, I + 8])
    order2 = P.morton_order(V2, I2, 8)
    assert list(order2) == [f for w in want for f in (w, w + 8)]


def test_features_invariant_under_translation_and_scale():
    """Vertices on a 2^-12 grid below 2^4, so a translation by multiples of
    2^-12 and a scale by 4 are exact in float32: the face order is the same
    and the features agree to float64 rounding (scale: exactly)."""
    rng = np.random.default_rng(11)
    A = rng.integers(-4096, 4096, size=(900, 3)) / 4096.0
    B = rng.integers(-4096, 4096, size=(270, 3)) / 4096.0
    IA = np.arange(900).reshape(-1, 3)
    IB = np.arange(270).reshape(-1, 3)
    X0 = P.mesh_pair_features(A, IA, B, IB, 10)
    t = np.array([0.5, -0.25, 2.0])
    X1 = P.mesh_pair_features(A + t, IA, B + t, IB, 10)
    X2 = P.mesh_pair_features(A * 4.0, IA, B * 4.0, IB, 10)
    np.testing.assert_allclose(X1, X0, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(X2, X0)
    assert (X0.reshape(128, 12)[:, :9] >= -1 - 1e-12).all() and (X0.reshape(128, 12)[:, :9] <= 1 + 1e-12).all()


def test_empty_clusters_are_zero():
    rng = np.random.default_rng(2)
    A = synth.tiny_random_mesh(10, rng)
    B = synth.tiny_random_mesh(70, rng)
    X = P.mesh_pair_features(A.V, A.I, B.V, B.I, 10).reshape(128, 12)
    sizes_a = [b - a for a, b in P.cluster_ranges(10)]
    for c in range(64):
        assert (X[c] == 0).all() == (sizes_a[c] == 0)
    assert all((X[64 + c] != 0).any() for c in range(64))


@pytest.mark.parametrize("k", [1, 3, 8])
def test_topk_by_hand_and_counting(k):
    row = np.array([1.0, 3.0, 3.0, 2.0, -1.0, 3.0, 0.0, 2.0, 5.0])
    want = [8, 1, 2, 5, 3, 7, 0, 6][:k]
    assert list(P.topk(row, k)[0]) == want
    rng = np.random.default_rng(k)
    Z = rng.integers(0, 20, size=(5, 300)).astype(float)
    T = P.topk(Z, k)
    for r in range(5):
        # each chosen value is >= every unchosen one; among equal values the
        # chosen indices are the lowest
        chosen = set(T[r])
        vmin = min(Z[r, j] for j in chosen)
        for j in range(300):
            if j not in chosen:
                assert Z[r, j] < vmin or (Z[r, j] == vmin and j > max(i for i in chosen if Z[r, i] == vmin))
