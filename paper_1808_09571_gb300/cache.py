"""Device-resident geometry cache with on-demand asynchronous loading and
whole-column evaluation (host orchestration; every load, build and query
runs in the library).

The geometry of a column lives on the host (a catalog: geometry id ->
vertex / index arrays).  The cache mirrors part of it on the device under a
byte budget, the way the paper's accelerator keeps a copy of the geometry
column in GPU memory that is filled asynchronously, on demand or at start-up
(Sec. 3.1), and evaluates an operator over a whole column at once (Sec. 3.1,
whole-column evaluation):

- `prefetch(ids)` starts the loads (host -> device copies made by the
  library, then the BVH builds) of the geometries not yet resident on a
  separate load stream and returns at once; queries that need them wait on
  the load's event, on the device, not on the host.
- `evaluate(qa, qb, ops)` runs a list of queries over geometry ids: it
  splits them into rounds whose distinct geometries fit half the budget,
  makes each round's geometries resident (evicting the least recently used
  ones that neither it nor the round in flight uses) and launches the round
  as one batch; the next round's loads are issued right after, so they
  overlap the batch in flight.
- `whole_column(column, other, op)` is evaluate() of one geometry against
  every geometry of a column.

Eviction releases a mesh stream-ordered on the query stream, after the
batches already launched there, so a batch in flight never loses its
geometry; the library allocates and frees mesh memory stream-ordered, so a
load on the load stream reuses an evicted mesh's memory only once the
query stream has released it.  Resident bytes are estimated per face
(serve.BYTES_PER_FACE); memory an eviction frees is counted as free at
once, so the device may hold up to one round more than the budget while
the batch in flight finishes.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np

from .serve import BYTES_PER_FACE


class GeometryCache:
    def __init__(self, ctx, catalog, budget_bytes: int, query_stream=None, load_stream=None,
                 bytes_per_face: int = BYTES_PER_FACE, event_factory=None, device="cuda:0"):
        """catalog: geometry id -> (V float32/float64 [nv, 3], I uint32/int32
        [nt, 3]) host arrays (pinned host memory makes the copies
        asynchronous).  Streams default to torch's current stream (queries)
        and a new side stream (loads); events come from torch.cuda.Event
        unless `event_factory` is given."""
        self.ctx = ctx
        self.catalog = catalog
        self.budget = int(budget_bytes)
        self.bpf = int(bytes_per_face)
        self.qs = query_stream
        self.ls = load_stream
        if self.qs is None or self.ls is None:
            import torch
            self.qs = self.qs if self.qs is not None else torch.cuda.current_stream()
            self.ls = self.ls if self.ls is not None else torch.cuda.Stream()
        self.event_factory = event_factory
        self.device = device
        self.resident: OrderedDict = OrderedDict()  # id -> Mesh, least recently used first
        self.used = 0
        self.pending_event = None                   # event after the latest loads on the load stream
        self.loads = self.evictions = 0

    # -- sizes -------------------------------------------------------------
    def cost(self, gid) -> int:
        return self.bpf * int(np.asarray(self.catalog[gid][1]).reshape(-1, 3).shape[0])

    # -- residency ---------------------------------------------------------
    def _make_room(self, need: int, keep: set):
        """Evict least recently used geometries outside `keep` until `need`
        more bytes fit the budget."""
        victims = []
        for gid in list(self.resident.keys()):
            if self.used + need <= self.budget:
                break
            if gid in keep:
                continue
            m = self.resident.pop(gid)
            self.used -= self.cost(gid)
            victims.append(m)
        if victims:
            # released after every batch already launched on the query stream
            self.ctx.mesh_free_many_async(victims, stream=self.qs)
            self.evictions += len(victims)
        if self.used + need > self.budget:
            raise MemoryError(f"geometries of one round need {self.used + need} bytes, budget {self.budget}")

    def prefetch(self, ids, keep=()):
        """Start loading the geometries of `ids` that are not resident (on
        the load stream; returns without waiting)."""
        miss = [g for g in dict.fromkeys(ids) if g not in self.resident]
        for g in dict.fromkeys(ids):
            if g in self.resident:
                self.resident.move_to_end(g)
        if not miss:
            return []
        need = sum(self.cost(g) for g in miss)
        self._make_room(need, set(ids) | set(keep))
        if self.pending_event is None:
            if self.event_factory is None:
                import torch
                self.event_factory = torch.cuda.Event
            self.pending_event = self.event_factory()
        ms = self.ctx.mesh_load_many([self.catalog[g] for g in miss], copy_fp64_master=False, stream=self.ls)
        self.ctx.mesh_build_bvh_many(ms, stream=self.ls)
        self.pending_event.record(self.ls)
        for g, m in zip(miss, ms):
            self.resident[g] = m
            self.used += self.cost(g)
        self.loads += len(miss)
        return miss

    def acquire(self, ids):
        """Handles (int64) of `ids`, every one resident once the query
        stream reaches the next launch (loads are waited for on the device)."""
        self.prefetch(ids)
        if self.pending_event is not None:
            self.qs.wait_event(self.pending_event)
        return np.array([self.resident[g].handle for g in ids], np.int64)

    # -- evaluation --------------------------------------------------------
    def rounds(self, qa, qb):
        """Split query indices into consecutive rounds whose distinct
        geometries fit half the budget (a query needs both of its
        geometries; two rounds are resident at once while one runs and the
        next loads)."""
        cap = self.budget // 2
        out, cur, ids, size = [], [], set(), 0
        for i, (a, b) in enumerate(zip(qa, qb)):
            add = [g for g in dict.fromkeys((a, b)) if g not in ids]
            extra = sum(self.cost(g) for g in add)
            if cur and size + extra > cap:
                out.append(cur)
                cur, ids, size = [], set(), 0
                add = list(dict.fromkeys((a, b)))
                extra = sum(self.cost(g) for g in add)
            if extra > cap:
                raise MemoryError(f"query {i} needs {extra} bytes, half the budget is {cap}")
            cur.append(i)
            ids.update(add)
            size += extra
        if cur:
            out.append(cur)
        return out

    def evaluate(self, qa, qb, ops):
        """Results (dist float64, hit uint8, status int32 numpy arrays) of the
        queries (geometry ids qa[i], qb[i], op ops[i])."""
        import torch
        qa, qb = list(qa), list(qb)
        ops = np.asarray(ops, np.int32)
        n = len(qa)
        d = torch.full((n,), float("nan"), dtype=torch.float64, device=self.device)
        h = torch.zeros(n, dtype=torch.uint8, device=self.device)
        s = torch.full((n,), -1, dtype=torch.int32, device=self.device)
        rs = self.rounds(qa, qb)

        def ids(r):
            return [qa[i] for i in r] + [qb[i] for i in r]

        if rs:
            self.prefetch(ids(rs[0]))
        for k, r in enumerate(rs):
            cur = ids(r)
            hd = self.acquire(cur)
            m = len(r)
            i0, i1 = r[0], r[-1] + 1  # rounds are consecutive runs of queries
            self.ctx.batch_arrays(hd[:m], hd[m:], ops[i0:i1], dist_out=d[i0:i1], hit_out=h[i0:i1],
                                  status_out=s[i0:i1], stream=self.qs, sync=False)
            if k + 1 < len(rs):  # the next round's loads overlap this batch
                self.prefetch(ids(rs[k + 1]), keep=cur)
        self.ctx.sync(self.qs)
        return d.cpu().numpy(), h.cpu().numpy(), s.cpu().numpy()

    def whole_column(self, column, other, op: int):
        """op(geometry c, geometry `other`) for every c of `column`."""
        column = list(column)
        return self.evaluate(column, [other] * len(column), np.full(len(column), op, np.int32))

    def clear(self):
        if self.resident:
            self.ctx.mesh_free_many_async(list(self.resident.values()), stream=self.qs)
        self.resident.clear()
        self.used = 0
