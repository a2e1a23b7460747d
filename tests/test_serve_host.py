"""Host logic of the served stream (no GPU): arrivals, requests, admission
by the candidate budget and the queue limit, the split by size."""
import numpy as np

from paper_1808_09571_gb300 import serve


def test_poisson_arrivals():
    rng = np.random.default_rng(0)
    t = serve.poisson_arrivals(5000.0, 200_000, rng)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 5000) < 0.01 / 5000
    assert abs(gaps.std() - 1 / 5000) < 0.02 / 5000  # exponential: std == mean
    counts = np.bincount((t / 0.01).astype(int))[:-1]  # per 10 ms: Poisson(50)
    assert abs(counts.mean() - 50) < 1 and abs(counts.var() - 50) < 5


def test_random_requests_distinct_pairs():
    rng = np.random.default_rng(1)
    a, b, op = serve.random_requests(7, 50_000, rng)
    assert np.all(a != b) and a.min() == 0 and b.max() == 6
    assert set(np.unique(op)) == {0, 1}
    # every ordered pair of distinct meshes is about equally likely
    c = np.bincount(a * 7 + b, minlength=49).reshape(7, 7)
    assert np.all(np.diag(c) == 0)
    off = c[~np.eye(7, dtype=bool)]
    assert off.min() > 0.8 * off.mean() and off.max() < 1.2 * off.mean()


def test_admission():
    ops = np.array([0] * 10 + [1] * 10, np.int32)
    pending = list(range(20))
    # queue limit
    assert serve.admit(pending, ops, 4, 10**9) == 4
    # candidate budget: 3 distance queries fit in 3 * 512
    assert serve.admit(pending, ops, 100, 3 * serve.CAND_EST[0]) == 3
    # at least one request per round even if it alone exceeds the budget
    assert serve.admit(pending, ops, 100, 1) == 1
    # intersects queries are cheaper
    assert serve.admit(list(range(10, 20)), ops, 100, 5 * serve.CAND_EST[1]) == 5
    # the face budget: requests of 300 faces each, 1,000 faces a round
    faces = np.full(20, 300)
    assert serve.admit(pending, ops, 100, 10**9, faces, face_budget=1000) == 3
    assert serve.admit(pending, ops, 100, 10**9, faces, face_budget=10) == 1


def test_split_by_size():
    faces = np.array([100, 70000, 500, 2_000_000])
    a = np.array([0, 0, 2, 1, 3])
    b = np.array([2, 1, 0, 3, 0])
    small, large = serve.split_by_size(np.arange(5), a, b, faces, 65536)
    assert list(small) == [0, 2] and list(large) == [1, 3, 4]
