#!/usr/bin/env python3
"""Benchmark of the 3D distance / 3D intersects engine on GB300.

Workload (one GPU): the large plain-method case -- a drill-hole tube
(radius 0.5, 16 sides, 65,536-segment persistent random walk, 2,097,152
faces) against an ore-body ellipsoid shell (40/25/15, 1024 x 1024 UV,
2,095,104 faces), 64 rigid placements (32 crossing the shell, 32 separated
by a gap log-uniform in [0.01, 10]), float32 vertices.  One step = ingest of
the 65 meshes from device-resident vertex/index buffers, BVH build of each,
and the 128 queries (distance + intersects per placement) in one batched
launch.  Metric: geometry pairs per second (queries completed / s).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on
a bounded sample of the same queries instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3DDistance/3DIntersects geometry-pairs/s"
UNIT = "geometry-pairs/s"
WORKLOAD = "tube_vs_orebody_2.1Mx2.1M_64_placements"

# Algorithmic cost of each kernel per unit of work (see the design notes):
# bytes for memory-bound kernels, FP32 operations for the leaf tests.
FLOP_FULL_TEST = 900.0   # certified face-pair distance bounds (15 feature terms)
FLOP_PREFILTER = 40.0    # two face boxes + box gap
FLOP_NODE = 20.0         # node-pair box gap
FLOP_SEG_TEST = 260.0    # certified segment-face bounds (5 feature terms)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic
# byte of k_frontier, from an ncu capture of this workload at 8 placements
# (27.26 MB of DRAM traffic per launch against 22.90 MB of distinct faces and
# nodes); the bench scales it to its launches by their algorithmic bytes
FRONTIER_DRAM_PER_ALG_BYTE = 27.26 / 22.90
# DRAM bytes per k_frontier launch of the 64-placement step itself (one-pass
# ncu capture of dram__bytes_read.sum + dram__bytes_write.sum on the two
# launches of a step: 125.2 MB and 96.4 MB): less than the algorithmic bytes,
# which count the ore body's faces and nodes once per query while the 64
# queries read the one ore body, which L2 keeps
FRONTIER_DRAM_PER_LAUNCH_64 = (125.24e6 + 96.37e6) / 2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--places", type=int, default=64)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the other configurations reported beside the headline (small icosphere pairs, "
                        "100,000 independent pairs, learned proposal, served stream)")
    p.add_argument("--extras-pairs", type=int, default=100000, help="pairs of the independent-pairs extra")
    p.add_argument("--leaf-size", type=int, default=0, help="faces per BVH leaf (0 = library default)")
    p.add_argument("--traversal", type=int, default=0, choices=[0, 1, 2],
                   help="1 level-synchronous, 2 persistent depth-first (0 = library default, then autotuned)")
    p.add_argument("--morton-bits", type=int, default=0, help="Morton bits per axis (0 = library default)")
    p.add_argument("--isect-first", type=int, default=0, choices=[0, 1, 2],
                   help="distance queries: 1 intersects phase first, 2 straight (0 = library default)")
    p.add_argument("--workload", default="large",
                   choices=["large", "pairs", "segments", "volume", "serve", "learned", "mlp"],
                   help="large: tube vs ore body (the headline); pairs: many independent small pairs; "
                        "segments: drill-hole segments vs the 500-face ore shape; "
                        "volume: ST_3DVolume of the large workload's 65 meshes; "
                        "serve: Poisson request stream over a device-resident store; "
                        "learned: train the proposal network, compare with / without it; "
                        "mlp: the proposal network's forward pass (tcgen05 GEMMs) on --rows rows")
    p.add_argument("--train-pairs", type=int, default=200000, help="training pairs of 'learned'")
    p.add_argument("--train-tmin", type=int, default=10000, help="smallest training mesh of 'learned' (faces)")
    p.add_argument("--train-tmax", type=int, default=100000, help="largest training mesh of 'learned' (faces)")
    p.add_argument("--eval-pairs", type=int, default=10000, help="held-out pairs of 'learned' (100k faces)")
    p.add_argument("--eval-chunk", type=int, default=2000, help="held-out pairs per batch of 'learned'")
    p.add_argument("--rows", type=int, default=2048, help="rows (queries) of the 'mlp' forward")
    p.add_argument("--frontier-capacity", type=int, default=0,
                   help="node pairs per frontier of the level-synchronous traversal in 'learned' (0 = library "
                        "default)")
    p.add_argument("--train-steps", type=int, default=20000, help="Adam steps of 'learned'")
    p.add_argument("--proposal-gates", default="8192",
                   help="proposal_min_faces values the independent pairs are measured at with the learned "
                        "proposal (comma list; the first is reported)")
    p.add_argument("--train-variants", type=int, default=16, help="template shapes per kind and size of 'learned'")
    p.add_argument("--store", type=int, default=10000, help="meshes of the 'serve' store (faces log-uniform 1k-1M)")
    p.add_argument("--rates", default="2000,5000,10000,20000,50000", help="offered request rates of 'serve' (req/s)")
    p.add_argument("--serve-seconds", type=float, default=2.0, help="arrival window per rate of 'serve'")
    p.add_argument("--serve-max-round", type=int, default=0,
                   help="most requests one round of 'serve' admits (0 = a quarter of the work queue)")
    p.add_argument("--holes", type=int, default=50000, help="drill holes of the 'segments' workload (100 segments each)")
    p.add_argument("--pairs", type=int, default=20000, help="pairs of the 'pairs' workload")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip g3d_autotune (launch shape, stack depth, intersects phase, leaf size) before warm-up")
    return p.parse_args()


def build_bytes_per_face(ore, tubes, tI):
    """Algorithmic bytes per face of one launch of each build kernel over the
    step's meshes (float32), every distinct byte counted once: ingest reads
    each source array once (the 64 placements share one index array, read
    once) and writes the library's copies (12 B indices per face, 12 B per
    vertex); Morton reads a mesh's indices (12 B per face) and vertices
    (12 B each, about half a vertex per face) and writes key and value (8 B);
    a sort pass reads the keys (counts: 4 B) or reads and writes key and
    value (16 B); the gather reads the sorted key and value (8 B), the
    indices (12 B) and the vertices, writes the 48 B face record and per
    leaf of 16 faces a 32 B box and a 4 B key."""
    nf = ore.nt + len(tubes) * len(tI)
    nv = len(ore.V) + sum(len(v) for v in tubes)
    vpf = 12.0 * nv / nf
    ingest = (12.0 * nv + 12.0 * (ore.nt + len(tI)) + 12.0 * nv + 12.0 * nf) / nf
    return {"k_ingest_many": ingest, "k_morton_tiles": 12.0 + vpf + 8.0, "k_seg_hist": 4.0, "k_seg_scatter": 16.0,
            "k_gather_many": 8.0 + 12.0 + vpf + 48.0 + 36.0 / 16.0}


def make_workload(n_place):
    import numpy as np
    from paper_1808_09571_gb300 import synth
    ore, tI, tubes, info = synth.large_placements(n_place=n_place)
    return ore, tI, tubes, info, np


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def cpu_baseline(ore, tI, tubes, info, np):
    """The oracle, single-threaded, on a bounded sample of the step's queries."""
    import oracle
    oracle.build()
    O64 = ore.V.astype(np.float64)
    sample = [(0, 0), (0, 1), (32, 0), (32, 1)] if len(tubes) > 32 else [(0, 0), (0, 1)]
    refs = []
    t0 = time.perf_counter()
    for k, op in sample:
        V64 = tubes[k].astype(np.float64)
        if op == 0:
            refs.append(oracle.mesh_distance_pruned(V64, tI, O64, ore.I))
        else:
            refs.append(oracle.mesh_intersects_pruned(V64, tI, O64, ore.I))
    dt = time.perf_counter() - t0
    return {"value": len(sample) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(sample)} of the step's queries (placements 0 and 32, distance and intersects), "
                      f"exact-pruned CPU oracle incl. its tree builds, 1 thread, {dt:.1f} s"}, list(zip(sample, refs))


def check_sampled_parity(checked, dist, hit, n_place):
    """The GPU results of the sampled queries (from the timed run) against the
    oracle's: intersects bit-exact, distance within 1e-12 relative + 1e-15.
    Query k of the batch is placement k's distance, n_place + k its
    intersects.  Raises on a mismatch; returns the number checked."""
    n = 0
    for (k, op), ref in checked:
        if op == 0:
            d = float(dist[k])
            if not abs(d - ref) <= 1e-12 * abs(ref) + 1e-15:
                raise AssertionError(f"parity: placement {k} distance {d!r} vs oracle {ref!r}")
            if (d == 0.0) != (int(hit[k]) == 1):
                raise AssertionError(f"parity: placement {k} distance {d!r} with hit flag {int(hit[k])}")
        else:
            x = int(hit[n_place + k])
            if x != int(bool(ref)):
                raise AssertionError(f"parity: placement {k} intersects {x} vs oracle {bool(ref)}")
        n += 1
    return n


def cpu_baseline_all_cores(ore, tI, tubes, np):
    """The oracle's threaded batch (one query per thread) on all host cores,
    on as many of the step's queries as there are cores."""
    import oracle
    oracle.build()
    ncores = os.cpu_count() or 1
    k = min(ncores, 2 * len(tubes))
    meshes = [(ore.V.astype(np.float64), ore.I)] + [(tubes[j].astype(np.float64), tI) for j in range(len(tubes))]
    qa = [1 + (j % len(tubes)) for j in range(k)]
    ops = [j // len(tubes) for j in range(k)]
    t0 = time.perf_counter()
    oracle.batch_pruned(meshes, qa, [0] * k, ops, nthreads=ncores)
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"{k} of the step's queries on {ncores} threads (exact-pruned CPU oracle, "
                      f"one query per thread, tree builds included), {dt:.1f} s"}


def run_reference(args):
    from paper_1808_09571_gb300 import replicas
    ws, rank, _ = replicas.env()
    if rank != 0:  # the CPU oracle runs on rank 0 only; the other ranks exit without work
        return
    ore, tI, tubes, info, np = make_workload(args.places)
    import oracle
    oracle.build()
    O64 = ore.V.astype(np.float64)
    queries = [(k, 0) for k in range(len(tubes))] + [(k, 1) for k in range(len(tubes))]
    order = [queries[(i * 37) % len(queries)] for i in range(len(queries))]

    def one(i):
        k, op = order[i % len(order)]
        V64 = tubes[k].astype(np.float64)
        if op == 0:
            oracle.mesh_distance_pruned(V64, tI, O64, ore.I)
        else:
            oracle.mesh_intersects_pruned(V64, tI, O64, ore.I)

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one(args.warmup + i)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "step": "one query of the workload (bounded sample)",
                      "queries_per_full_step": len(queries)},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} queries cycling through the 128, exact-pruned CPU oracle, "
                                      "1 thread"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def small_bench(reps=50):
    """The small plain-method case: two pairs of 1,280-face icospheres (FP64
    vertices, FP64 master copy), pair A separated, pair B intersecting.
    Per-call latency (p50 / p99 over `reps` rounds of the 4 queries, single
    g3d_distance / g3d_intersects calls on prebuilt BVHs, CUDA events) and
    throughput of single calls and of one batch of the 4 queries."""
    import torch
    from paper_1808_09571_gb300 import geo3d, synth
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = geo3d.Context(0)
    sp = synth.small_pairs()
    hs = []
    for key in ("A", "B"):
        A, B = sp[key]
        hs.append((ctx.load_and_build(A.V, A.I, copy_fp64_master=True),
                   ctx.load_and_build(B.V, B.I, copy_fp64_master=True)))
    one = torch.empty(1, dtype=torch.float64, device=dev)
    oneh = torch.empty(1, dtype=torch.uint8, device=dev)
    lat = []
    for rep in range(reps + 3):
        for a, b in hs:
            for op in (0, 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if op == 0:
                    ctx.distance(a, b, out=one, sync=False)
                else:
                    ctx.intersects(a, b, out=oneh, sync=False)
                e1.record(stream)
                e1.synchronize()
                if rep >= 3:
                    lat.append(e0.elapsed_time(e1))
    qs = [(a, b, op) for a, b in hs for op in (0, 1)]
    d_dist = torch.empty(4, dtype=torch.float64, device=dev)
    d_hit = torch.empty(4, dtype=torch.uint8, device=dev)
    d_stat = torch.empty(4, dtype=torch.int32, device=dev)
    for _ in range(3):
        ctx.batch(qs, dist_out=d_dist, hit_out=d_hit, status_out=d_stat)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.batch(qs, dist_out=d_dist, hit_out=d_hit, status_out=d_stat, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    b_ms = e0.elapsed_time(e1) / reps
    ctx.sync()
    assert (d_stat.cpu().numpy() == 0).all()
    lat.sort()
    ctx.close()
    return {"workload": "icosphere_1280x1280_fp64_2_pairs", "queries": 4,
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "pairs_per_s_single_calls": len(lat) / (sum(lat) / 1000.0),
            "batch_of_4_ms": b_ms, "pairs_per_s_batched": 4 / (b_ms / 1000.0),
            "distance_A": float(d_dist[0].item()), "intersects_B": int(d_hit[3].item())}


def run_pairs(args):
    print(json.dumps(pairs_bench(args, args.pairs, args.steps, args.warmup)), flush=True)


def pairs_bench(args, n_pairs, steps, warmup, proposal_params=None):
    """Many independent pairs (jittered spheres / tubes, faces log-uniform in
    [20, 65536], ~30 % sharing a vertex, mixed operators): one step = batched
    ingest + BVH build of all meshes + one batched launch of all queries.
    Also reports the same queries as single calls (a sample), as a
    CUDA-graph replay and, given trained network parameters, as one batch
    with the learned proposal (results checked identical)."""
    import numpy as np
    import torch
    from paper_1808_09571_gb300 import geo3d, synth
    dev = torch.device("cuda:0")
    t0 = time.perf_counter()
    meshes, queries, info = synth.batch_workload(n_pairs)
    gen_s = time.perf_counter() - t0
    ctx = geo3d.Context(0, leaf_size=args.leaf_size)
    stream = torch.cuda.current_stream(dev)
    uniq = {}
    dI = []
    for V, I in meshes:
        k = I.ctypes.data
        if k not in uniq:
            uniq[k] = torch.from_numpy(I.view(np.int32)).to(dev)
        dI.append(uniq[k])
    dV = [torch.from_numpy(V).to(dev) for V, _ in meshes]
    nq = len(queries)
    d_dist = torch.empty(nq, dtype=torch.float64, device=dev)
    d_hit = torch.empty(nq, dtype=torch.uint8, device=dev)
    d_stat = torch.empty(nq, dtype=torch.int32, device=dev)

    # the step goes through the array forms of the calls (addresses, counts,
    # handles as arrays): no per-mesh or per-query Python work
    vptr = np.array([t.data_ptr() for t in dV], np.uint64)
    iptr = np.array([t.data_ptr() for t in dI], np.uint64)
    vdt = np.array([geo3d.G3D_F32 if t.dtype == torch.float32 else geo3d.G3D_F64 for t in dV], np.int32)
    nvs = np.array([t.shape[0] for t in dV], np.int64)
    nts = np.array([t.shape[0] for t in dI], np.int64)
    qa = np.array([q[0] for q in queries], np.int64)
    qb = np.array([q[1] for q in queries], np.int64)
    qop = np.array([q[2] for q in queries], np.int32)

    def load_all():
        return ctx.mesh_load_arrays(vptr, vdt, nvs, iptr, nts, copy_fp64_master=False)

    def build_all(hs):
        for c0 in range(0, len(hs), 60000):
            ctx.mesh_build_bvh_many(hs[c0:c0 + 60000])

    def step():
        hs = load_all()
        build_all(hs)
        ctx.batch_arrays(hs[qa], hs[qb], qop, dist_out=d_dist, hit_out=d_hit, status_out=d_stat, sync=False)
        ctx.mesh_free_many_async(hs, stream=stream)

    tuned = None
    if not args.no_autotune:  # untimed: on a quarter of the queries, before warm-up
        hs = ctx.mesh_load_many(list(zip(dV, dI)), copy_fp64_master=False)
        for c0 in range(0, len(hs), 60000):
            ctx.mesh_build_bvh_many(hs[c0:c0 + 60000])
        t0 = time.perf_counter()
        tuned = ctx.autotune([(hs[a], hs[b], op) for (a, b, op) in queries[: max(1, nq // 4)]],
                             tune_leaf_size=True, reps=3, count_build=True)
        tuned = {"chosen": {k: tuned[k] for k in ("leaf_size", "warps_per_cta", "ctas_per_sm", "stack_depth",
                                                   "isect_first", "morton_bits", "traversal", "dives")},
                 "tuning_s": round(time.perf_counter() - t0, 2)}
        ctx.mesh_free_many(hs)

    for _ in range(warmup):
        step()
    ctx.sync()
    torch.cuda.synchronize()
    # one extra untimed step with a wall-clock split of its phases
    phases = {}
    t = time.perf_counter()
    hs = load_all()
    torch.cuda.synchronize()
    phases["load_s"] = time.perf_counter() - t
    t = time.perf_counter()
    build_all(hs)
    torch.cuda.synchronize()
    phases["build_s"] = time.perf_counter() - t
    t = time.perf_counter()
    ctx.batch_arrays(hs[qa], hs[qb], qop, dist_out=d_dist, hit_out=d_hit, status_out=d_stat)
    phases["batch_s"] = time.perf_counter() - t
    t = time.perf_counter()
    ctx.mesh_free_many(hs)
    phases["free_s"] = time.perf_counter() - t
    st0 = ctx.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.sync()
    st1 = ctx.stats()
    assert (d_stat.cpu().numpy() == 0).all()
    # prebuilt: batched queries only, CUDA-graph replay, single calls (sample)
    hs = ctx.mesh_load_many(list(zip(dV, dI)), copy_fp64_master=False)
    for c0 in range(0, len(hs), 60000):
        ctx.mesh_build_bvh_many(hs[c0:c0 + 60000])
    qs = [(hs[a], hs[b], op) for (a, b, op) in queries]
    # the array form of the batch call: no per-query Python work
    ha = np.array([m.handle for m in hs], np.int64)
    qa_h, qb_h = ha[qa], ha[qb]

    def run_batch(sync=False):
        ctx.batch_arrays(qa_h, qb_h, qop, dist_out=d_dist, hit_out=d_hit, status_out=d_stat, sync=sync)

    def batched_x3():
        # 3 batches back to back, then the same 3 again under the library's
        # per-kernel timer (its events do not enter the first timing)
        run_batch(sync=True)
        e0.record(stream)
        for _ in range(3):
            run_batch()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 3
        ctx.stats_reset()
        ctx.profile_begin("")
        for _ in range(3):
            run_batch()
        ctx.sync()
        prof = ctx.profile_end()
        st = ctx.stats()
        work = {"node_pairs": st["node_pairs"] // 3, "tri_tests": st["tri_tests"] // 3,
                "kernels_ms": {k: round(v[1] / 3, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])[:8]}}
        return t, work

    q_ms, q_work = batched_x3()
    learned = None
    if proposal_params is not None:
        ref = (d_dist.cpu().numpy().copy(), d_hit.cpu().numpy().copy())
        mlp = geo3d.MLP(ctx, proposal_params)
        dist_q = qop == 0
        small = np.array([min(len(meshes[a][1]), len(meshes[b][1])) for (a, b, _) in queries])
        gate0 = ctx.config()["proposal_min_faces"]

        def one(prop):
            # one batch from an idle device (its host-side preparation
            # included), with or without the proposal
            ctx.set_proposal(prop)
            torch.cuda.synchronize()
            e0.record(stream)
            run_batch()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        by_gate = []
        for g in [int(x) for x in str(args.proposal_gates).split(",")]:
            ctx.set_config(proposal_min_faces=g)
            one(mlp)  # untimed: the clusters' statistics are computed on first use
            same = bool(np.array_equal(d_dist.cpu().numpy()[dist_q], ref[0][dist_q]) and
                        np.array_equal(d_hit.cpu().numpy()[~dist_q], ref[1][~dist_q]))
            assert same
            tp, tl = [], []
            for _ in range(7):  # the two forms alternate, so drifts of the device hit both
                tp.append(one(None))
                tl.append(one(mlp))
            r = {"proposal_min_faces": g, "proposal_rows": int((small >= g).sum()), "ms": float(np.median(tl)),
                 "ms_without": float(np.median(tp)), "results_identical": same}
            r["pairs_per_s"] = nq / (r["ms"] / 1000.0)
            r["vs_batched"] = r["ms_without"] / r["ms"]
            if not by_gate:  # per-kernel work at the reported gate
                ctx.set_proposal(mlp)
                r["work"] = batched_x3()[1]
                r["work_without"] = q_work
            by_gate.append(r)
        ctx.set_proposal(None)
        ctx.set_config(proposal_min_faces=gate0)
        learned = dict(by_gate[0])
        learned["timing"] = "median of 7 single batches from an idle device, alternating with the plain form"
        if len(by_gate) > 1:
            learned["by_gate"] = [{k: r[k] for k in ("proposal_min_faces", "proposal_rows", "ms", "ms_without",
                                                     "vs_batched")} for r in by_gate]
        mlp.close()
    plan = ctx.plan_create(qs, d_dist, d_hit, d_stat)
    ctx.plan_launch(plan)
    e0.record(stream)
    for _ in range(3):
        ctx.plan_launch(plan)
    e1.record(stream)
    torch.cuda.synchronize()
    g_ms = e0.elapsed_time(e1) / 3
    ctx.plan_destroy(plan)
    n_single = min(nq, 500)
    one = torch.empty(1, dtype=torch.float64, device=dev)
    oneh = torch.empty(1, dtype=torch.uint8, device=dev)
    e0.record(stream)
    for (a, b, op) in qs[:n_single]:
        if op == 0:
            ctx.distance(a, b, out=one, sync=False)
        else:
            ctx.intersects(a, b, out=oneh, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    s_ms = e0.elapsed_time(e1)
    ctx.sync()
    faces = sum(len(I) for _, I in meshes)
    out = {"metric": METRIC, "value": nq * steps / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (FP64/exact on certified candidates)", "data": "synthetic",
           "config": {"workload": f"independent_pairs_{n_pairs}", "meshes": len(meshes), "faces_total": int(faces),
                      "faces_per_mesh": "log-uniform [20, 65536] (half-octave templates)",
                      "shared_vertex_fraction": float(np.mean([i["shares_vertex"] for i in info])),
                      "step": "ingest + batched BVH build of all meshes + one batched launch of all queries",
                      "generation_s": round(gen_s, 1), "autotune": tuned,
                      "phases_of_one_step_s": {k: round(v, 4) for k, v in phases.items()}},
           "batched_queries_only": {"ms": q_ms, "pairs_per_s": nq / (q_ms / 1000.0)},
           "batched_queries_learned": learned,
           "graph_replay": {"ms": g_ms, "pairs_per_s": nq / (g_ms / 1000.0)},
           "plain_single_calls": {"queries": n_single, "ms": s_ms, "pairs_per_s": n_single / (s_ms / 1000.0)},
           "tri_pair_tests_per_step": (st1["tri_tests"] - st0["tri_tests"]) / steps,
           "gpu_launches": int(st1["launches"] - st0["launches"])}
    ctx.close()
    return out


def run_segments(args):
    """The paper's own workload: drill-hole line segments against one
    500-face ore shape.  One step = ST_3DDistance and ST_3DIntersects of
    every segment against the ore shape (two g3d_segments calls over
    device-resident segments); a geometry pair is one (segment, ore) query."""
    import numpy as np
    import torch
    from paper_1808_09571_gb300 import geo3d, synth
    dev = torch.device("cuda:0")
    ore = synth.small_ore_body()
    t0 = time.perf_counter()
    segs = synth.drill_holes(args.holes, 100)
    gen_s = time.perf_counter() - t0
    n = len(segs)
    ctx = geo3d.Context(0)
    stream = torch.cuda.current_stream(dev)
    h = ctx.mesh_load(ore.V, ore.I, copy_fp64_master=False)
    ctx.mesh_build_bvh(h)
    d_segs = torch.from_numpy(segs).to(dev)
    d_dist = torch.empty(n, dtype=torch.float64, device=dev)
    d_hit = torch.empty(n, dtype=torch.uint8, device=dev)
    d_hit2 = torch.empty(n, dtype=torch.uint8, device=dev)
    d_stat = torch.empty(n, dtype=torch.int32, device=dev)

    def step(sv, dd, dh, dh2, ds):
        ctx.segments(h, sv, geo3d.OP_DISTANCE, dist_out=dd, hit_out=dh, status_out=ds, sync=False)
        ctx.segments(h, sv, geo3d.OP_INTERSECTS, hit_out=dh2, status_out=ds, sync=False)

    for _ in range(args.warmup):
        step(d_segs, d_dist, d_hit, d_hit2, d_stat)
    ctx.sync()
    torch.cuda.synchronize()
    ctx.stats_reset()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    ctx.profile_begin("")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step(d_segs, d_dist, d_hit, d_hit2, d_stat)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_end()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ctx.sync()
    st = ctx.stats()
    assert (d_stat.cpu().numpy() == 0).all()
    hits = d_hit2.cpu().numpy()
    assert np.array_equal(hits, d_hit.cpu().numpy())
    pairs = 2 * n * args.steps
    # roofline of k_segments: FP32 work from the device counters
    flops = st["tri_tests"] * FLOP_SEG_TEST + st["node_pairs"] * FLOP_NODE
    kl, kms, _ = prof["k_segments"]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks() or {}
    peak = sms * 128 * 2 * (peaks.get("sm_max_mhz", 2070.0) * 1e6) / 1e12
    ach = flops / (kms / 1000.0) / 1e12
    roof = {"bound": "alu", "kernel": "k_segments", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None,
            "peak_note": f"FP32 non-tensor: {sms} SMs x 128 lanes x 2 x sm_max {peaks.get('sm_max_mhz', 2070.0)} MHz"}
    # end to end from pinned host memory: segments in, results out, every step
    h_segs = torch.from_numpy(segs).pin_memory()
    h_dist = torch.empty(n, dtype=torch.float64).pin_memory()
    h_hit = torch.empty(n, dtype=torch.uint8).pin_memory()
    h_hit2 = torch.empty(n, dtype=torch.uint8).pin_memory()
    h_stat = torch.empty(n, dtype=torch.int32).pin_memory()
    step(h_segs, h_dist, h_hit, h_hit2, h_stat)
    ctx.sync()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t1 = time.perf_counter()
    f0.record(stream)
    for _ in range(args.steps):
        step(h_segs, h_dist, h_hit, h_hit2, h_stat)
    f1.record(stream)
    torch.cuda.synchronize()
    ems = max(f0.elapsed_time(f1), 1000 * (time.perf_counter() - t1))
    ctx.sync()
    assert np.array_equal(h_dist.numpy(), d_dist.cpu().numpy())
    # CPU oracle on a bounded sample (each segment as a one-face mesh)
    cpu = None
    if not args.no_cpu:
        import oracle
        oracle.build()
        OV = ore.V.astype(np.float64)
        idx = np.arange(0, n, max(1, n // 4000))
        I1 = np.array([[0, 1, 2]], np.uint32)
        tc = time.perf_counter()
        for k in idx:
            sg = segs[k].astype(np.float64)
            V = np.array([sg[:3], sg[3:], sg[3:]])
            oracle.mesh_distance_pruned(V, I1, OV, ore.I)
            oracle.mesh_intersects_pruned(V, I1, OV, ore.I)
        dt = time.perf_counter() - tc
        cpu = {"value": 2 * len(idx) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{len(idx)} segments (every {max(1, n // 4000)}th), distance + intersects each, "
                         "exact-pruned CPU oracle, 1 thread"}
    kern_table = {k: {"launches": v[0], "total_ms": round(v[1], 3), "share": round(v[1] / ms, 4)}
                  for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    out = {"metric": METRIC, "value": pairs / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (FP64/exact on certified candidates)", "data": "synthetic",
           "config": {"workload": f"drill_hole_segments_{n}_vs_ore_shape_500",
                      "segments": n, "ore_faces": int(ore.nt),
                      "step": "ST_3DDistance + ST_3DIntersects of every segment against the ore shape",
                      "intersecting_segments": int(hits.sum()), "generation_s": round(gen_s, 1),
                      "l2": f"segments {segs.nbytes / 1e6:.0f} MB + results per step > 129 MB L2"},
           "tri_pair_tests_per_s": st["tri_tests"] / (ms / 1000.0),
           "exact_tests_per_step": st["exact_tests"] / args.steps,
           "roofline": roof, "kernels": kern_table, "clocks": clocks,
           "gpu_launches": int(sum(v[0] for v in prof.values())),
           "e2e": {"value": pairs / (ems / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(segs.nbytes),
                   "d2h_bytes_per_step": int(n * (8 + 1 + 1 + 4))},
           "cpu_baseline": cpu}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_volume(args):
    """ST_3DVolume (Eq. 2) of a column of meshes: the ore body and the 64
    tube placements of the large workload (136M faces), one g3d_volume_many
    call per step over device-resident meshes.  HBM-bound: per face 12 B of
    indices and 3 vertices of 12 B (float32) are read."""
    import numpy as np
    import torch
    from paper_1808_09571_gb300 import geo3d
    ore, tI, tubes, info, np = make_workload(args.places)
    dev = torch.device("cuda:0")
    ctx = geo3d.Context(0)
    stream = torch.cuda.current_stream(dev)
    oreV = torch.from_numpy(ore.V).to(dev)
    oreI = torch.from_numpy(ore.I.view(np.int32)).to(dev)
    tI_d = torch.from_numpy(tI.view(np.int32)).to(dev)
    hs = ctx.mesh_load_many([(oreV, oreI)] + [(torch.from_numpy(v).to(dev), tI_d) for v in tubes],
                            copy_fp64_master=False)
    out = torch.empty(len(hs), dtype=torch.float64, device=dev)
    faces = ore.nt + len(tubes) * len(tI)
    verts = len(ore.V) + sum(len(v) for v in tubes)
    for _ in range(args.warmup):
        ctx.volume(hs, out=out)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    ctx.profile_begin("")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.volume(hs, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_end()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    vols = out.cpu().numpy()
    kl, kms, _ = prof["k_volume_chunks"]
    # algorithmic bytes: indices once, every vertex once (each is shared by ~6 faces)
    alg = 12 * faces + 12 * verts
    peaks = measured_peaks() or {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    ach = alg / (kms / kl / 1000.0) / 1e9
    rl, rms, _ = prof.get("k_volume_range", (0, 0.0, 0.0))
    kern_table = {k: {"launches": v[0], "total_ms": round(v[1], 3), "share": round(v[1] / ms, 4)}
                  for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    res = {"metric": "3DVolume meshes/s", "value": len(hs) * args.steps / (ms / 1000.0), "unit": "meshes/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "exact integers (float32 meshes on their coordinate grid), f64 fallback", "data": "synthetic",
           "config": {"workload": WORKLOAD + "_volume", "meshes": len(hs), "faces": int(faces),
                      "step": "one g3d_volume_many over the 65 device-resident meshes",
                      "l2": f"{alg / 1e9:.2f} GB read per step > 129 MB L2"},
           "faces_per_s": faces * args.steps / (ms / 1000.0),
           "roofline": {"bound": "hbm", "kernel": "k_volume_chunks", "achieved": ach, "peak": hbm,
                        "unit": "GB/s", "frac": ach / hbm, "traffic": None,
                        "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                        "bytes_note": "12 B indices per face + 12 B per vertex, each read once",
                        "range_pass": {"kernel": "k_volume_range", "ms_per_launch": rms / max(1, rl),
                                       "bytes_per_launch": 12 * verts}},
           "kernels": kern_table, "clocks": clocks, "gpu_launches": int(sum(v[0] for v in prof.values())),
           "ore_volume": float(vols[0]), "ore_volume_closed_form": 4.0 / 3.0 * 3.141592653589793 * 40 * 25 * 15}
    print(json.dumps(res), flush=True)
    ctx.close()


def run_serve(args):
    print(json.dumps(serve_bench(args, args.rates)), flush=True)


def serve_bench(args, rates_arg):
    """Served stream: Poisson arrivals of distance / intersects requests on
    uniform random pairs of a device-resident store of meshes (faces
    log-uniform in [1k, 1M]), admitted by memory and batched by size, at each
    offered rate; reports throughput and p50 / p99 latency per rate."""
    import numpy as np
    import torch
    from paper_1808_09571_gb300 import geo3d, serve
    ctx = geo3d.Context(0, traversal=args.traversal)
    store = serve.build_store(ctx, args.store)
    nm = len(store.handles)
    rates = [float(x) for x in rates_arg.split(",")]
    rng = np.random.default_rng(1812)
    # warm-up: a short stream at the lowest rate
    wa = serve.poisson_arrivals(rates[0], max(50, int(rates[0] * 0.2)), rng)
    serve.serve(ctx, store, wa, *serve.random_requests(nm, len(wa), rng))
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    st0 = ctx.stats()
    per = []
    total_q, total_s = 0, 0.0
    for rate in rates:
        n = max(1, int(rate * args.serve_seconds))
        arr = serve.poisson_arrivals(rate, n, rng)
        a, b, op = serve.random_requests(nm, n, rng)
        r = serve.serve(ctx, store, arr, a, b, op, max_round=args.serve_max_round)
        assert (r.status == 0).all(), np.unique(r.status)
        per.append({"offered_req_s": rate, "requests": n, "throughput_req_s": r.throughput,
                    "p50_ms": float(np.percentile(r.latency_ms, 50)),
                    "p99_ms": float(np.percentile(r.latency_ms, 99)),
                    "rounds": r.rounds, "mean_round_size": r.mean_round_size,
                    "intersecting": int(r.hit[op == 1].sum())})
        print(json.dumps(per[-1]), file=sys.stderr, flush=True)
        total_q += n
        total_s += r.elapsed_s
    clocks = sampler.stop()
    st1 = ctx.stats()
    top = per[-1]
    out = {"metric": METRIC, "value": top["throughput_req_s"], "unit": UNIT, "n_gpus": 1,
           "steps": len(rates), "warmup": 1, "ms_per_step": 1000.0 * total_s / len(rates),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 (FP64/exact on certified candidates)", "data": "synthetic",
           "config": {"workload": f"served_stream_store_{nm}", "store_meshes": nm,
                      "store_faces": int(store.faces.sum()), "store_bytes_est": int(store.bytes_est),
                      "store_budget": int(store.budget), "refused_meshes": int(store.refused),
                      "store_build_s": round(store.build_s, 2),
                      "step": "one offered rate: Poisson arrivals for the arrival window, served to completion",
                      "value_is": f"throughput at the highest offered rate ({rates[-1]:.0f} req/s)"},
           "rates": per, "node_pairs": int(st1["node_pairs"] - st0["node_pairs"]),
           "clocks": clocks, "gpu_launches": int(st1["launches"] - st0["launches"]),
           "roofline": None, "cpu_baseline": None,
           "e2e": {"value": total_q / total_s, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                   "note": "requests arrive as host arrays; results stay on the device"}}
    ctx.close()
    return out


def run_mlp(args):
    """The proposal network's forward pass (1536 -> 256 -> 256 -> 256 ->
    4096, BF16 operands, FP32 accumulation on the tcgen05 tensor cores) on
    --rows rows of random features: --warmup untimed and --steps timed
    passes (CUDA events); roofline against the measured BF16 peak."""
    import torch
    from paper_1808_09571_gb300 import geo3d, learn
    dev = torch.device("cuda:0")
    ctx = geo3d.Context(0)
    mlp = geo3d.MLP(ctx, learn.he_init(1))
    g = torch.Generator(device=dev)
    g.manual_seed(1808)
    X = torch.randn(args.rows, 1536, device=dev, generator=g)
    for _ in range(args.warmup):
        mlp.forward(X)
    torch.cuda.synchronize()
    ctx.profile_begin("")
    ts = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mlp.forward(X)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    prof = ctx.profile_end()
    ms = sorted(ts)[len(ts) // 2]
    flops = 2.0 * args.rows * (1536 * 256 + 256 * 256 * 2 + 256 * 4096)
    gl, gms, _ = prof.get("k_gemm_tc", (0, 0.0, 0.0))
    peaks = measured_peaks() or {}
    peak = peaks.get("bf16_tflops", 1900.0)
    ach = flops / (gms / max(1, args.steps) / 1000.0) / 1e12 if gms > 0 else 0.0
    out = {"metric": "proposal forward rows/s", "value": args.rows / (ms / 1000.0), "unit": "rows/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16 operands, fp32 accumulate", "data": "synthetic",
           "config": {"workload": f"mlp_forward_{args.rows}_rows", "layers": "1536-256-256-256-4096"},
           "roofline": {"bound": "tensor", "kernel": "k_gemm_tc", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                        "frac": ach / peak, "traffic": None,
                        "peak_note": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json bf16_tflops)",
                        "flops_per_step": flops},
           "kernels": {k: {"launches": v[0], "ms_per_step": round(v[1] / max(1, args.steps), 4)}
                       for k, v in prof.items()},
           "gpu_launches": int(sum(v[0] for v in prof.values()))}
    print(json.dumps(out), flush=True)
    mlp.close()
    ctx.close()


def run_learned(args):
    out = learned_bench(args)
    out.pop("_params")
    print(json.dumps(out), flush=True)


def learned_bench(args):
    """The learned proposal (config 4): the network is trained on the GPU by
    the library's kernels on pairs labelled by the engine's own witnesses,
    then held-out pairs of 100k-face meshes run, in chunks of at most
    --eval-chunk pairs (each chunk one batch), without a proposal, with the
    trained network, and with the true witness clusters as hints (the
    ceiling of any proposal); a sample of them also runs as single calls
    without a proposal (the plain form).  Reports hit rates, the seeded
    bound's excess over the distance, work counters and pairs/s."""
    import numpy as np
    import torch
    from paper_1808_09571_gb300 import geo3d, learn
    dev = torch.device("cuda:0")
    ctx = geo3d.Context(0, isect_first=2, frontier_capacity=args.frontier_capacity)
    from paper_1808_09571_gb300 import synth
    t0 = time.perf_counter()
    X, Y = [], []
    bank, cache = synth.TemplateBank(5000), {}  # the training shapes, shared by all chunks
    for c0 in range(0, args.train_pairs, 1024):  # chunks keep the device memory bounded
        n = min(1024, args.train_pairs - c0)
        meshes, queries = learn.make_pairs_device(n, seed=5000 + c0, t_min=args.train_tmin, t_max=args.train_tmax,
                                                  variants=args.train_variants, device=dev, bank=bank, cache=cache)
        hs = learn.load(ctx, meshes)
        lab, _ = learn.labels_of(ctx, hs, queries)
        keep = np.nonzero(lab >= 0)[0]
        X.append(ctx.pair_features([(hs[queries[i][0]], hs[queries[i][1]]) for i in keep]).clone())
        Y.append(torch.from_numpy(lab[keep].astype(np.int32)).to(dev))
        ctx.mesh_free_many(hs)
        del meshes
    del cache
    X, Y = torch.cat(X), torch.cat(Y)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    mlp = geo3d.MLP(ctx, learn.he_init(1))
    t1 = time.perf_counter()
    curve = learn.train(mlp, X, Y, steps=args.train_steps, batch=512, lr=1e-3, log_every=max(1, args.train_steps // 6))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    del X, Y

    proposal_kernels = ("k_pair_features", "k_to_bf16", "k_gemm_tc", "k_gemm_bf16", "k_topk", "k_set_proposal")
    names = ("none", "trained", "true_clusters")
    acc = {k: {"ms": 0.0, "node_pairs": 0, "tri_tests": 0, "candidates": 0, "seed_excess_sum": 0.0, "seed_q": 0,
               "kernels": {}} for k in names}
    hits = {"top1": 0.0, "top4": 0.0, "top16": 0.0}
    n_eval = n_lab = 0
    single = {"queries": 0, "ms": 0.0}

    def timed(run, key, reps=5):
        run()
        torch.cuda.synchronize()
        ctx.stats_reset()
        ts = []
        ctx.profile_begin("")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = run()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        prof = ctx.profile_end()
        st = ctx.stats()
        a = acc[key]
        a["ms"] += sorted(ts)[reps // 2]
        for c in ("node_pairs", "tri_tests", "candidates"):
            a[c] += st[c] // reps
        a["seed_excess_sum"] += st["seed_excess_ppm"] / 1e6 / reps
        a["seed_q"] += st["seed_queries"] // reps
        for k, v in prof.items():
            a["kernels"][k] = a["kernels"].get(k, 0.0) + v[1] / reps
        return r

    ebank, ecache = synth.TemplateBank(99991), {}  # held-out shapes (another seed than the training ones)
    for c0 in range(0, args.eval_pairs, args.eval_chunk):
        n = min(args.eval_chunk, args.eval_pairs - c0)
        meshes, queries = learn.make_pairs_device(n, seed=99991 + c0, t_min=100000, t_max=100000,
                                                  variants=args.train_variants, device=dev, bank=ebank,
                                                  cache=ecache)
        hs = learn.load(ctx, meshes)
        lab, _ = learn.labels_of(ctx, hs, queries)
        keep = np.nonzero(lab >= 0)[0]
        Xe = ctx.pair_features([(hs[queries[i][0]], hs[queries[i][1]]) for i in keep])
        r = learn.hit_rates(mlp, Xe, torch.from_numpy(lab[keep].astype(np.int32)).to(dev))
        for k in hits:
            hits[k] += r[k] * len(keep)
        n_lab += len(keep)
        del Xe
        qs = [(hs[a], hs[b], 0) for (a, b, _) in queries]
        ctx.set_proposal(None)
        r0 = timed(lambda: ctx.batch(qs), "none")
        ctx.set_proposal(mlp)
        r1 = timed(lambda: ctx.batch(qs), "trained")
        ctx.set_proposal(None)
        r2 = timed(lambda: ctx.batch_hint(qs, lab), "true_clusters")
        for rr in (r1, r2):
            assert np.array_equal(rr[0], r0[0]) and (rr[2] == 0).all()
        if c0 == 0:  # the plain form: one call per query, no proposal
            m = min(200, len(qs))
            for a_, b_, _ in qs[:5]:
                ctx.distance(a_, b_)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for a_, b_, _ in qs[:m]:
                ctx.distance(a_, b_)
            e1.record()
            torch.cuda.synchronize()
            single = {"queries": m, "ms": e0.elapsed_time(e1)}
        n_eval += n
        ctx.mesh_free_many(hs)
        del meshes, qs

    res = {}
    for k in names:
        a = acc[k]
        kms = sum(a["kernels"].values())
        pk = {kk: round(a["kernels"][kk], 4) for kk in proposal_kernels if kk in a["kernels"]}
        res[k] = {"pairs_per_s": n_eval / (a["ms"] / 1000.0), "ms": a["ms"], "node_pairs": a["node_pairs"],
                  "tri_tests": a["tri_tests"], "candidates": a["candidates"],
                  "seed_excess": a["seed_excess_sum"] / max(1, a["seed_q"]),
                  "proposal_kernels_ms": pk, "kernel_ms": round(kms, 4),
                  "gemm_share": ((pk.get("k_gemm_tc", 0.0) + pk.get("k_gemm_bf16", 0.0)) / kms) if kms > 0 else 0.0,
                  "top_kernels_ms": {kk: round(v, 4) for kk, v in
                                     sorted(a["kernels"].items(), key=lambda kv: -kv[1])[:8]}}
    plain = single["queries"] / (single["ms"] / 1000.0) if single["ms"] > 0 else None
    out = {"metric": METRIC, "value": res["trained"]["pairs_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 5,
           "warmup": 1, "ms_per_step": res["trained"]["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (FP64/exact on certified candidates); network bf16 / fp32 accumulate",
           "data": "synthetic",
           "config": {"workload": f"learned_proposal_eval_{n_eval}x100k",
                      "train_pairs": int(args.train_pairs),
                      "train_faces": f"log-uniform [{args.train_tmin}, {args.train_tmax}]",
                      "eval_pairs": n_eval, "eval_chunk": args.eval_chunk, "eval_faces": 100000,
                      "train_steps": args.train_steps, "train_variants": args.train_variants,
                      "frontier_capacity": ctx.config()["frontier_capacity"],
                      "data_s": round(data_s, 1), "train_s": round(train_s, 2),
                      "value_is": "pairs/s of the held-out pairs, batched, with the trained proposal"},
           "loss_curve": curve, "hit_rates": {k: v / max(1, n_lab) for k, v in hits.items()}, "runs": res,
           "plain_single_calls": {"queries": single["queries"], "ms": single["ms"], "pairs_per_s": plain},
           "gain_vs_plain": res["trained"]["pairs_per_s"] / res["none"]["pairs_per_s"],
           "ceiling_vs_plain": res["true_clusters"]["pairs_per_s"] / res["none"]["pairs_per_s"],
           "gain_vs_single_calls": (res["trained"]["pairs_per_s"] / plain) if plain else None,
           "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None,
           "_params": mlp.get_params()}
    ctx.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "pairs":
        run_pairs(args)
        return
    if args.workload == "segments":
        run_segments(args)
        return
    if args.workload == "volume":
        run_volume(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "learned":
        run_learned(args)
        return
    if args.workload == "mlp":
        run_mlp(args)
        return
    from paper_1808_09571_gb300 import replicas
    ws, rank, local = replicas.env()
    import torch
    if ws > 1:
        torch.cuda.set_device(local)
    dist = replicas.init("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ore, tI, tubes, info, np = make_workload(args.places)
    from paper_1808_09571_gb300 import geo3d
    ctx = geo3d.Context(local, leaf_size=args.leaf_size, traversal=args.traversal, morton_bits=args.morton_bits,
                        isect_first=args.isect_first)
    stream = torch.cuda.current_stream(dev)

    # device-resident inputs
    oreV = torch.from_numpy(ore.V).to(dev)
    oreI = torch.from_numpy(ore.I.view(np.int32)).to(dev)
    tI_d = torch.from_numpy(tI.view(np.int32)).to(dev)
    tV = [torch.from_numpy(v).to(dev) for v in tubes]
    nq = 2 * len(tubes)
    d_dist = torch.empty(nq, dtype=torch.float64, device=dev)
    d_hit = torch.empty(nq, dtype=torch.uint8, device=dev)
    d_stat = torch.empty(nq, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    def run_step(Vore, Iore, Vt, It, dist_out, hit_out, stat_out):
        ms = ctx.mesh_load_many([(Vore, Iore)] + [(v, It) for v in Vt], copy_fp64_master=False)
        ctx.mesh_build_bvh_many(ms)
        O, T = ms[0], ms[1:]
        qs = [(t, O, 0) for t in T] + [(t, O, 1) for t in T]
        ctx.batch(qs, dist_out=dist_out, hit_out=hit_out, status_out=stat_out, sync=False)
        ctx.mesh_free_many_async(T + [O], stream=stream)

    def step():
        run_step(oreV, oreI, tV, tI_d, d_dist, d_hit, d_stat)

    tuned = None
    if not args.no_autotune:  # untimed, before warm-up: the step's own 128 queries
        ms_ = ctx.mesh_load_many([(oreV, oreI)] + [(v, tI_d) for v in tV], copy_fp64_master=False)
        ctx.mesh_build_bvh_many(ms_)
        t0 = time.perf_counter()
        tuned = ctx.autotune([(t, ms_[0], 0) for t in ms_[1:]] + [(t, ms_[0], 1) for t in ms_[1:]],
                             tune_leaf_size=True, reps=3, count_build=True)
        tuned = {"chosen": {k: tuned[k] for k in ("leaf_size", "warps_per_cta", "ctas_per_sm", "stack_depth",
                                                   "isect_first", "morton_bits", "traversal", "dives")},
                 "tuning_s": round(time.perf_counter() - t0, 2)}
        ctx.mesh_free_many(ms_)

    for _ in range(args.warmup):
        step()
    ctx.sync()
    replicas.barrier(dist)
    torch.cuda.synchronize()
    ctx.stats_reset()
    st0 = ctx.stats()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ctx.profile_begin("")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    replicas.barrier(dist)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier(dist)
    prof = ctx.profile_end()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ctx.sync()
    st1 = ctx.stats()
    status = d_stat.cpu().numpy()
    if (status != 0).any():
        raise RuntimeError(f"query errors: {np.unique(status)}")
    dist_timed, hit_timed = d_dist.cpu().numpy(), d_hit.cpu().numpy()  # results of the last timed step
    ms = replicas.max_over_ranks(ms, dist, dev)
    value = replicas.job_rate(nq * args.steps, ws, ms)

    # ---- roofline of the dominant kernel ------------------------------------
    peaks = measured_peaks() or {}
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dname, (dl, dms, _) = dom
    tri_tests = st1["tri_tests"] - st0["tri_tests"]
    prefilter = st1["tri_prefilter"] - st0["tri_prefilter"]
    nodes = st1["node_pairs"] - st0["node_pairs"]
    n_faces = ore.nt + len(tubes) * len(tI)
    roof = None
    if dname in ("k_traverse", "k_frontier"):
        # FP32 work from the device counters, and the algorithmic bytes the
        # traversal reads: every distinct internal node (64 B: both child
        # boxes) and every face of the distinct leaves tested (48 B) of each
        # query, counted by one untimed batch with count_visits on the same
        # meshes and queries
        flops = tri_tests * FLOP_FULL_TEST + prefilter * FLOP_PREFILTER + nodes * FLOP_NODE
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        fpeak = sms * 128 * 2 * (peaks.get("sm_max_mhz", 2070.0) * 1e6) / 1e12
        fach = flops / dl / (dms / dl / 1000.0) / 1e12
        ms_c = ctx.mesh_load_many([(oreV, oreI)] + [(v, tI_d) for v in tV], copy_fp64_master=False)
        ctx.mesh_build_bvh_many(ms_c)
        ctx.set_config(count_visits=1)
        ctx.stats_reset()
        ctx.batch([(t, ms_c[0], 0) for t in ms_c[1:]] + [(t, ms_c[0], 1) for t in ms_c[1:]])
        stc = ctx.stats()
        ctx.set_config(count_visits=0)
        ctx.mesh_free_many(ms_c)
        launches_per_step = dl / args.steps
        alg = (48.0 * stc["distinct_faces"] + 64.0 * stc["distinct_nodes"]) / launches_per_step
        hbm = peaks.get("hbm_gbs", 6800.0)
        ach = alg / (dms / dl / 1000.0) / 1e9
        # the DRAM counters were taken before k_frontier's leaf batches were
        # dealt by warp index first (the same leaf pairs and faces are read,
        # in another order): no current capture, so traffic is reported as
        # unknown and the earlier figure as context only
        traffic = None
        earlier = None
        if dname == "k_frontier":
            earlier = FRONTIER_DRAM_PER_LAUNCH_64 if len(tubes) == 64 else FRONTIER_DRAM_PER_ALG_BYTE * alg
        roof = {"bound": "hbm", "kernel": dname, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "traffic_before_last_change": earlier, "algorithmic_bytes_per_launch": alg,
                "distinct_faces_per_step": stc["distinct_faces"], "distinct_nodes_per_step": stc["distinct_nodes"],
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "traffic_note": ("null: the kernel changed after its last ncu capture; traffic_before_last_change "
                                 "= dram bytes read + written per launch in that capture (one pass, this step's "
                                 "two launches: 125.2 MB, 96.4 MB), below the algorithmic bytes, which count the "
                                 "shared ore body once per query" if len(tubes) == 64 else
                                 "null: the kernel changed after its last ncu capture; traffic_before_last_change "
                                 "= the 8-placement capture's DRAM bytes per algorithmic byte (1.19) times this "
                                 "launch's algorithmic bytes"),
                "alu": {"achieved": fach, "peak": fpeak, "unit": "TFLOP/s", "frac": fach / fpeak,
                        "peak_note": f"FP32 non-tensor: {sms} SMs x 128 lanes x 2 x sm_max "
                                     f"{peaks.get('sm_max_mhz', 2070.0)} MHz"}}
    else:
        bpe = build_bytes_per_face(ore, tubes, tI).get(dname)
        if bpe is not None:
            launch_bytes = bpe * n_faces  # every launch of these kernels covers all faces of the step
            ach = launch_bytes / (dms / dl / 1000.0) / 1e9
            peak = peaks.get("hbm_gbs", 6800.0)
            roof = {"bound": "hbm", "kernel": dname, "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "traffic": None,
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    # the HBM fraction of every build kernel as well
    per_face = build_bytes_per_face(ore, tubes, tI)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_kernels = {}
    for k, bpf in per_face.items():
        if k in prof:
            kl, kms, _ = prof[k]
            a_ = bpf * n_faces / (kms / kl / 1000.0) / 1e9
            hbm_kernels[k] = {"bytes_per_face": bpf, "achieved_gbs": round(a_, 1), "frac": round(a_ / hbm_peak, 3),
                              "ms_per_launch": round(kms / kl, 4)}
    if roof is not None:
        roof["build_kernels_hbm"] = hbm_kernels
    kern_table = {k: {"launches": v[0], "total_ms": round(v[1], 3), "share": round(v[1] / ms, 4)}
                  for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # ---- end to end from pinned host buffers ----------------------------------
    # End to end through the C ABI with host buffers: every step passes the
    # pinned host vertex / index arrays of its 65 meshes straight to
    # g3d_mesh_load_many, which copies them to the device in stream order
    # and validates them (the 64 placements share one index array, which
    # crosses once per call); results come back to pinned host memory
    # through g3d_batch.  Loads run on a second stream: the load of step k+1
    # (host copies + ingest) overlaps the build and queries of step k.
    e2e = None
    if not args.no_e2e:
        hV = torch.from_numpy(ore.V).pin_memory()
        hI = torch.from_numpy(ore.I.view(np.int32)).pin_memory()
        htI = torch.from_numpy(tI.view(np.int32)).pin_memory()
        htV = [torch.from_numpy(v).pin_memory() for v in tubes]
        h_dist = torch.empty(nq, dtype=torch.float64).pin_memory()
        h_hit = torch.empty(nq, dtype=torch.uint8).pin_memory()
        h_stat = torch.empty(nq, dtype=torch.int32).pin_memory()
        load_s = torch.cuda.Stream(dev)
        host_meshes = [(hV, hI)] + [(v, htI) for v in htV]

        def load_host():
            return ctx.mesh_load_many(host_meshes, copy_fp64_master=False, stream=load_s)

        def compute(ms_):
            ctx.mesh_build_bvh_many(ms_, stream=stream)
            O, T = ms_[0], ms_[1:]
            qs_ = [(t, O, 0) for t in T] + [(t, O, 1) for t in T]
            ctx.batch(qs_, dist_out=h_dist, hit_out=h_hit, status_out=h_stat, stream=stream, sync=False)
            ctx.mesh_free_many_async(ms_, stream=stream)

        def run_e2e(n):
            nxt = load_host()
            for k in range(n):
                cur = nxt
                compute(cur)
                if k + 1 < n:
                    nxt = load_host()  # returns when the copies and checks are done; step k runs meanwhile

        run_e2e(2)
        torch.cuda.synchronize()
        replicas.barrier(dist)
        t0 = time.perf_counter()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        run_e2e(args.steps)
        f1.record(stream)
        torch.cuda.synchronize()
        ems = max(f0.elapsed_time(f1), 1000 * (time.perf_counter() - t0))
        ems = replicas.max_over_ranks(ems, dist, dev)
        assert (h_stat.numpy() == 0).all()
        assert np.array_equal(h_dist.numpy(), d_dist.cpu().numpy(), equal_nan=True)
        # the 64 placements pass one host index array: the library copies it once per call
        h2d = ore.V.nbytes + ore.I.nbytes + sum(v.nbytes for v in tubes) + tI.nbytes
        e2e = {"value": replicas.job_rate(nq * args.steps, ws, ems), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(nq * (8 + 1 + 4)),
               "path": "pinned host pointers into g3d_mesh_load_many (library copies, stream-ordered; a host array "
                       "passed for several meshes crosses once); g3d_batch writes pinned host results",
               "pipeline": "load of step k+1 on a second stream overlaps build and queries of step k"}

    # ---- plain (unbatched) form on prebuilt BVHs: per-query latency -----------
    plain = None
    if not args.no_plain and rank == 0:
        O = ctx.load_and_build(oreV, oreI, copy_fp64_master=False)
        T = [ctx.load_and_build(v, tI_d, copy_fp64_master=False) for v in tV]
        one = torch.empty(1, dtype=torch.float64, device=dev)
        oneh = torch.empty(1, dtype=torch.uint8, device=dev)
        lat = []
        for rep in range(2):
            for k, t in enumerate(T):
                for op in (0, 1):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    if op == 0:
                        ctx.distance(t, O, out=one, sync=False)
                    else:
                        ctx.intersects(t, O, out=oneh, sync=False)
                    b.record(stream)
                    b.synchronize()
                    if rep == 1:
                        lat.append(a.elapsed_time(b))
        ctx.sync()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.batch([(t, O, 0) for t in T] + [(t, O, 1) for t in T], dist_out=d_dist, hit_out=d_hit,
                  status_out=d_stat, sync=False)
        b.record(stream)
        b.synchronize()
        lat.sort()
        plain = {"pairs_per_s_unbatched": len(lat) / (sum(lat) / 1000.0),
                 "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                 "batched_queries_only_ms": a.elapsed_time(b),
                 "pairs_per_s_batched_queries_only": nq / (a.elapsed_time(b) / 1000.0)}
        for m in T + [O]:
            ctx.mesh_free(m)

    cpu = cpu_all = None
    parity_checked = 0
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu, checked = cpu_baseline(ore, tI, tubes, info, np)
        parity_checked = check_sampled_parity(checked, dist_timed, hit_timed, len(tubes))
        cpu_all = cpu_baseline_all_cores(ore, tI, tubes, np)

    secs = ms / 1000.0
    in_gb = (ore.V.nbytes + ore.I.nbytes + sum(v.nbytes for v in tubes) + len(tubes) * tI.nbytes) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (FP64/exact on certified candidates)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "tube_faces": int(len(tI)), "orebody_faces": int(ore.nt),
                   "placements": len(tubes), "queries_per_step": nq,
                   "step": f"ingest of {len(tubes) + 1} meshes + one batched BVH build + one batched launch of the "
                           f"{nq} queries",
                   "l2": f"inputs {in_gb:.1f} GB per step > 129 MB L2, no flush needed", "autotune": tuned},
        "tri_pair_tests_per_s": tri_tests / secs, "tri_pair_prefilter_per_s": prefilter / secs,
        "node_pairs_per_s": nodes / secs,
        "brute_force_equivalent_tri_pairs_per_s": {
            "value": float(nq) * ore.nt * len(tI) * args.steps / secs,
            "note": "all nA x nB face pairs of every query per second of the step: the dense work the "
                    "branch-and-bound avoids, not work done"},
        "roofline": roof, "kernels": kern_table, "clocks": clocks,
        "gpu_launches": int(st1["launches"] - st0["launches"]),
        "e2e": e2e, "plain": plain, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
        "parity_checked": parity_checked,
    }
    ctx.close()
    if rank == 0 and ws == 1 and not args.no_extras:
        # the other configurations, measured in the same run (untimed by the
        # headline's clock): the small case, the independent pairs at their
        # stated size, and the learned proposal against the plain form
        torch.cuda.empty_cache()
        out["small_icosphere"] = small_bench()
        torch.cuda.empty_cache()
        # the served stream first: its store of 10,000 meshes (about 104 GB)
        # is admitted against the free device memory
        sb = serve_bench(args, "2000,10000,50000")
        out["served_stream"] = {k: sb[k] for k in ("value", "unit", "config", "rates", "gpu_launches")}
        torch.cuda.empty_cache()
        lb = learned_bench(args)
        params = lb.pop("_params")
        out["learned_proposal"] = {k: lb[k] for k in ("value", "unit", "config", "hit_rates", "runs", "gain_vs_plain",
                                                      "ceiling_vs_plain", "plain_single_calls",
                                                      "gain_vs_single_calls")}
        torch.cuda.empty_cache()
        pb = pairs_bench(args, args.extras_pairs, steps=5, warmup=3, proposal_params=params)
        out["independent_pairs"] = {k: pb[k] for k in ("value", "unit", "ms_per_step", "config", "batched_queries_only",
                                                       "batched_queries_learned", "graph_replay", "plain_single_calls",
                                                       "gpu_launches")}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
