"""Served stream: a device-resident mesh store and an open-loop request
service over it (host orchestration; every query runs in the library).

- The store holds meshes loaded once (vertex / index copies, BVH) under a
  device-memory budget: a mesh is admitted only while the estimated bytes of
  the admitted meshes stay within it; the others are refused and reported.
- Requests (mesh a, mesh b, op) arrive at given times (Poisson arrivals for
  the benchmark).  The server keeps one batch in flight: each round takes the
  requests that have arrived (FIFO), admits them into the round while the
  round's estimated candidate memory and the work queue allow, and launches
  them as two batches by size -- pairs whose larger mesh is small first, then
  the rest -- so small requests are not held back by large ones.  A request's
  completion time is the GPU time of its batch's completion event.
- Latency = completion - arrival; throughput = completed / (last completion -
  first arrival).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import synth

# estimated device bytes per face of a loaded, built mesh: float4 SoA (48),
# index copy (12), about half a vertex per face (6), nodes + leaves + ranges (7)
BYTES_PER_FACE = 73
# estimated candidate-pool entries a query needs (a round is admitted while
# the sum stays within half of the pool; an overflow is still handled by the
# library's second pass)
CAND_EST = {0: 512, 1: 64}
# faces (both meshes of every request) a round admits: random pairs of the
# store lie far apart relative to their size, and thousands of them on
# meshes of up to 1M faces outgrow the level-synchronous traversal's
# frontier lists (measured: 2,048 such requests, 568 M faces, peak 4.1 M node
# pairs of 8.4 M; 4,096 requests, 1.18 G faces, overflow)
FACE_BUDGET = 600 << 20


@dataclass
class Store:
    handles: np.ndarray          # int64 mesh handles
    faces: np.ndarray            # faces per mesh
    meshes: list                 # Mesh objects
    bytes_est: int
    refused: int
    build_s: float
    budget: int
    sources: list = field(default_factory=list)  # (V, I) device tensors per mesh when kept


def build_store(ctx, n_meshes: int, t_min: int = 1000, t_max: int = 1_000_000, budget_bytes: int | None = None,
                region: float = 20.0, seed: int = synth.BASE_SEED + 7, device: str = "cuda:0",
                chunk_faces: int = 200_000_000, keep_sources: bool = False) -> Store:
    """n_meshes jittered UV spheres / 8-sided tubes (50/50) with face counts
    log-uniform in [t_min, t_max] (half-octave templates, each scaled to a
    bounding radius of 1 about its centroid), each under a random rotation,
    centred uniformly in a cube of side `region`; float32.  Loaded and built
    in chunks of about `chunk_faces` faces.  With keep_sources the input
    vertex / index tensors stay in Store.sources (for checks against a CPU
    reference)."""
    import torch
    rng = np.random.default_rng(seed)
    bank = synth.TemplateBank(seed)
    if budget_bytes is None:
        free, _ = torch.cuda.mem_get_info(torch.device(device))
        budget_bytes = int(0.6 * free)
    lo, hi = math.log(t_min), math.log(t_max)
    plan = []
    est = refused = 0
    for _ in range(n_meshes):
        kind = "sphere" if rng.random() < 0.5 else "tube"
        T = int(round(math.exp(rng.uniform(lo, hi))))
        V, I = bank.get(kind, T, 0)
        b = BYTES_PER_FACE * len(I)
        R = synth.random_rotation(rng)
        t = rng.uniform(-region / 2, region / 2, 3)
        if est + b > budget_bytes:
            refused += 1
            continue
        est += b
        plan.append((kind, T, R, t))
    dev = torch.device(device)
    tmpl = {}
    handles, faces, meshes, sources = [], [], [], []
    t0 = time.perf_counter()
    i = 0
    while i < len(plan):
        chunk, nf = [], 0
        while i < len(plan) and (not chunk or nf < chunk_faces):
            kind, T, R, t = plan[i]
            key = (kind, int(round(2 * math.log2(max(T, 2)))))
            if key not in tmpl:
                V, I = bank.get(kind, T, 0)
                V = V - V.mean(axis=0)
                V = V / np.linalg.norm(V, axis=1).max()
                tmpl[key] = (torch.from_numpy(V.astype(np.float32)).to(dev),
                             torch.from_numpy(I.view(np.int32)).to(dev))
            Vt, It = tmpl[key]
            Rt = torch.from_numpy(R.astype(np.float32)).to(dev)
            tt = torch.from_numpy(t.astype(np.float32)).to(dev)
            chunk.append(((Vt @ Rt.T + tt).contiguous(), It))
            nf += It.shape[0]
            i += 1
        hs = ctx.mesh_load_many(chunk, copy_fp64_master=False)
        ctx.mesh_build_bvh_many(hs)
        ctx.sync()
        handles += [h.handle for h in hs]
        faces += [h.nt for h in hs]
        meshes += hs
        if keep_sources:
            sources += chunk
        del chunk
    torch.cuda.synchronize()
    return Store(np.array(handles, np.int64), np.array(faces, np.int64), meshes, est, refused,
                 time.perf_counter() - t0, budget_bytes, sources)


def poisson_arrivals(rate: float, n: int, rng: np.random.Generator) -> np.ndarray:
    """Arrival times (s) of a Poisson process of `rate` per second."""
    return np.cumsum(rng.exponential(1.0 / rate, n))


def random_requests(n_meshes: int, n: int, rng: np.random.Generator):
    """Uniform random pairs of distinct meshes, op 0 / 1 with probability 1/2."""
    a = rng.integers(0, n_meshes, n)
    b = rng.integers(0, n_meshes - 1, n)
    b = b + (b >= a)
    return a, b, rng.integers(0, 2, n).astype(np.int32)


def admit(pending: list, ops: np.ndarray, max_queries: int, cand_budget: int, faces: np.ndarray | None = None,
          face_budget: int = FACE_BUDGET) -> int:
    """How many of the pending requests (FIFO) the next round takes: at
    least one, then while the queue limit, the candidate budget and (given
    the faces of each request) the face budget hold."""
    k, used, nf = 0, 0, 0
    for r in pending:
        c = CAND_EST[int(ops[r])]
        f = int(faces[r]) if faces is not None else 0
        if k and (k >= max_queries or used + c > cand_budget or nf + f > face_budget):
            break
        used += c
        nf += f
        k += 1
    return k


def split_by_size(ids: np.ndarray, a: np.ndarray, b: np.ndarray, faces: np.ndarray, small_faces: int):
    """(small, large): requests whose larger mesh has at most small_faces faces, and the rest."""
    big = np.maximum(faces[a[ids]], faces[b[ids]]) > small_faces
    return ids[~big], ids[big]


@dataclass
class ServeResult:
    rate: float
    n: int
    latency_ms: np.ndarray
    throughput: float
    rounds: int
    batches: int
    mean_round_size: float
    elapsed_s: float
    dist: np.ndarray = field(repr=False)
    hit: np.ndarray = field(repr=False)
    status: np.ndarray = field(repr=False)


def serve(ctx, store: Store, arrivals: np.ndarray, qa: np.ndarray, qb: np.ndarray, ops: np.ndarray,
          small_faces: int = 65536, device: str = "cuda:0", max_round: int = 0) -> ServeResult:
    """Run the requests (indices into the store) arriving at `arrivals` (s,
    increasing) through the open-loop server; returns per-request results
    and latencies.  A round admits at most `max_round` requests (0: a
    quarter of the library's work queue)."""
    import torch
    dev = torch.device(device)
    n = len(arrivals)
    cfg = ctx.config()
    max_q = cfg["queue_capacity"] // 4
    if max_round > 0:
        max_q = min(max_q, max_round)
    cand_budget = cfg["cand_capacity"] // 2
    H = store.handles
    req_faces = store.faces[qa] + store.faces[qb]
    dist = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    hit = torch.zeros(n, dtype=torch.uint8, device=dev)
    stat = torch.full((n,), -1, dtype=torch.int32, device=dev)
    bd = torch.empty(max_q, dtype=torch.float64, device=dev)
    bh = torch.empty(max_q, dtype=torch.uint8, device=dev)
    bs = torch.empty(max_q, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    done_ms = np.zeros(n)
    pending: list = []
    nxt = rounds = batches = 0
    sizes = []
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t0 = time.perf_counter()
    while nxt < n or pending:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            pending.append(nxt)
            nxt += 1
        if not pending:
            wait = arrivals[nxt] - (time.perf_counter() - t0)
            if wait > 2e-4:
                time.sleep(wait - 1e-4)
            continue
        k = admit(pending, ops, max_q, cand_budget, req_faces)
        ids = np.array(pending[:k], np.int64)
        del pending[:k]
        rounds += 1
        sizes.append(k)
        marks = []
        for part in split_by_size(ids, qa, qb, store.faces, small_faces):
            m = len(part)
            if m == 0:
                continue
            ctx.batch_arrays(H[qa[part]], H[qb[part]], ops[part], dist_out=bd[:m], hit_out=bh[:m],
                             status_out=bs[:m], stream=stream, sync=False)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            it = torch.from_numpy(part).to(dev, non_blocking=True)
            dist[it] = bd[:m]
            hit[it] = bh[:m]
            stat[it] = bs[:m]
            marks.append((part, ev))
            batches += 1
        marks[-1][1].synchronize()
        for part, ev in marks:
            done_ms[part] = ev0.elapsed_time(ev)
    ctx.sync()
    torch.cuda.synchronize()
    lat = done_ms - arrivals * 1000.0
    span = (done_ms.max() - arrivals[0] * 1000.0) / 1000.0
    offered = n / arrivals[-1] if n and arrivals[-1] > 0 else 0.0
    return ServeResult(offered, n, lat, n / max(span, 1e-9), rounds, batches,
                       float(np.mean(sizes)) if sizes else 0.0, span,
                       dist.cpu().numpy(), hit.cpu().numpy(), stat.cpu().numpy())
