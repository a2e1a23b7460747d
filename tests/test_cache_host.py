"""Host logic of the geometry cache (no GPU): rounds that fit half the
budget, least-recently-used eviction that spares the geometries of the
round in flight, loads issued on the load stream with the query stream
waiting on their event, stream-ordered releases, whole-column evaluation
over more geometry than the budget holds."""
import numpy as np
import pytest

from paper_1808_09571_gb300.cache import GeometryCache


class FakeMesh:
    def __init__(self, handle):
        self.handle = handle


class FakeEvent:
    def __init__(self, log):
        self.log = log

    def record(self, stream):
        self.log.append(("record", stream.name))


class FakeStream:
    def __init__(self, name, log):
        self.name, self.log = name, log

    def wait_event(self, ev):
        self.log.append(("wait", self.name))


class FakeCtx:
    """Records the calls; batch results encode the handles' geometry ids."""

    def __init__(self, log):
        self.log = log
        self.next = 1
        self.live = {}   # handle -> geometry vertex array id

    def mesh_load_many(self, meshes, copy_fp64_master=False, stream=None):
        out = []
        for V, I in meshes:
            m = FakeMesh(self.next)
            self.live[self.next] = int(V[0, 0])
            self.next += 1
            out.append(m)
        self.log.append(("load", stream.name, [self.live[m.handle] for m in out]))
        return out

    def mesh_build_bvh_many(self, ms, stream=None):
        self.log.append(("build", stream.name, len(ms)))

    def mesh_free_many_async(self, ms, stream=None):
        self.log.append(("free", stream.name, sorted(self.live.pop(m.handle) for m in ms)))

    def batch_arrays(self, ha, hb, ops, dist_out=None, hit_out=None, status_out=None, stream=None, sync=True):
        for h in list(ha) + list(hb):
            assert int(h) in self.live, "a batch used an evicted geometry"
        ga = np.array([self.live[int(h)] for h in ha], np.float64)
        gb = np.array([self.live[int(h)] for h in hb], np.float64)
        import torch
        dist_out.copy_(torch.from_numpy(ga * 1000 + gb + ops))
        hit_out.fill_(1)
        status_out.fill_(0)
        self.log.append(("batch", stream.name, len(ha)))

    def sync(self, stream=None):
        self.log.append(("sync", stream.name))


def catalog(sizes):
    """geometry g: a mesh of sizes[g] faces whose first coordinate is g"""
    return {g: (np.full((3, 3), float(g), np.float32), np.zeros((n, 3), np.uint32)) for g, n in enumerate(sizes)}


def make(sizes, budget_faces):
    log = []
    c = GeometryCache(FakeCtx(log), catalog(sizes), budget_bytes=budget_faces, bytes_per_face=1,
                      query_stream=FakeStream("q", log), load_stream=FakeStream("l", log),
                      event_factory=lambda: FakeEvent(log), device="cpu")
    return c, log


def test_rounds_fit_half_the_budget():
    c, _ = make([10] * 8, budget_faces=60)
    qa, qb = [0, 1, 2, 3, 4, 5], [7, 7, 7, 7, 6, 6]
    rs = c.rounds(qa, qb)
    assert [i for r in rs for i in r] == list(range(6))
    for r in rs:
        g = {qa[i] for i in r} | {qb[i] for i in r}
        assert 10 * len(g) <= 30
    with pytest.raises(MemoryError):
        make([40, 10], budget_faces=60)[0].rounds([0], [1])


def test_lru_eviction_spares_keep_and_recent():
    c, log = make([10] * 6, budget_faces=30)
    c.prefetch([0, 1, 2])
    c.acquire([0])                 # 0 is now the most recent
    c.prefetch([3], keep=[1])      # evicts the least recent outside {1, 3}: 2
    assert list(c.resident) == [1, 0, 3] and c.used == 30
    frees = [e for e in log if e[0] == "free"]
    assert frees == [("free", "q", [2])]
    assert c.loads == 4 and c.evictions == 1


def test_loads_on_the_load_stream_and_queries_wait():
    c, log = make([10] * 4, budget_faces=100)
    h = c.acquire([2, 3])
    assert ("load", "l", [2, 3]) in log and ("build", "l", 2) in log
    i = log.index(("record", "l"))
    assert log[i + 1] == ("wait", "q")
    assert len(h) == 2 and h.dtype == np.int64


def test_whole_column_over_more_than_the_budget():
    sizes = [5] * 40 + [20]
    c, log = make(sizes, budget_faces=60)   # 8 geometries of 5 faces plus the 20-face one per round
    d, hit, s = c.whole_column(list(range(40)), 40, op=1)
    assert (s == 0).all() and hit.all()
    assert np.array_equal(d, np.arange(40) * 1000.0 + 40 + 1)
    assert c.evictions > 0 and c.used <= 60
    # every geometry of the column was loaded once; the shared one stayed resident
    loaded = [g for e in log if e[0] == "load" for g in e[2]]
    assert sorted(loaded) == list(range(41))
    assert log[-1] == ("sync", "q")


def test_repeated_evaluation_reuses_resident_geometry():
    c, log = make([10] * 4, budget_faces=100)
    c.evaluate([0, 1], [2, 3], [0, 0])
    n = c.loads
    d, _, _ = c.evaluate([1, 0], [3, 2], [1, 1])
    assert c.loads == n and np.array_equal(d, [1003.0 + 1, 2.0 + 1])
