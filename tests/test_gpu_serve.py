"""The served stream on a small store: every request answered, results equal
to one batch of the same requests and, on a sample, to the CPU oracle on
the store's own input arrays; latencies measured."""
import numpy as np
import pytest

from paper_1808_09571_gb300 import serve

pytestmark = pytest.mark.gpu


def test_serve_matches_one_batch(g3d, orc):
    ctx = g3d.Context(0, time_limit_ms=10000)
    store = serve.build_store(ctx, 40, t_min=1000, t_max=20000, region=8.0, budget_bytes=1 << 40,
                              chunk_faces=100_000, keep_sources=True)
    assert len(store.handles) == 40 and store.refused == 0
    rng = np.random.default_rng(3)
    n = 3000
    arr = serve.poisson_arrivals(20000.0, n, rng)
    a, b, op = serve.random_requests(40, n, rng)
    r = serve.serve(ctx, store, arr, a, b, op)
    assert (r.status == 0).all()
    d, h, s = ctx.batch_arrays(store.handles[a], store.handles[b], op)
    assert (s == 0).all()
    np.testing.assert_array_equal(r.dist, d)
    np.testing.assert_array_equal(r.hit, h)
    assert r.rounds >= 2 and r.batches >= r.rounds
    assert np.all(r.latency_ms > 0) and np.isfinite(r.latency_ms).all()
    assert r.throughput > 0
    # a sample against the oracle (distance within 1e-12 relative, intersects bit-exact)
    src = [(V.cpu().numpy().astype(np.float64), I.cpu().numpy().view(np.uint32)) for V, I in store.sources]
    checked = 0
    for i in range(0, n, 150):
        A, B = src[a[i]], src[b[i]]
        if op[i] == 0:
            ref = orc.mesh_distance_pruned(A[0], A[1], B[0], B[1])
            assert abs(r.dist[i] - ref) <= 1e-12 * abs(ref) + 1e-15, (i, r.dist[i], ref)
        else:
            assert bool(r.hit[i]) == orc.mesh_intersects_pruned(A[0], A[1], B[0], B[1]), i
        checked += 1
    assert checked == 20


def test_store_budget_refuses(g3d):
    ctx = g3d.Context(0, time_limit_ms=10000)
    store = serve.build_store(ctx, 30, t_min=1000, t_max=4000, budget_bytes=serve.BYTES_PER_FACE * 20000)
    assert store.refused > 0 and store.bytes_est <= serve.BYTES_PER_FACE * 20000
    assert len(store.handles) + store.refused == 30
