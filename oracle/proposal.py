"""Plain reference of the learned proposal's inputs and output selection
(test infrastructure only; nothing in the product imports it).

The proposal network reads, for a pair of meshes, per-cluster statistics of
both meshes in a frame common to the pair, and its output is reduced to the
k highest-scoring cluster pairs.  The paper has no learned component; these
definitions are the engine's own and are written here as plainly as they are
stated:

- face order: faces sorted by the Morton key of their centroid, ties by face
  index (a stable sort).  The key quantises the centroid to 2^bits - 1 cells
  per axis over the vertex box of the float32 coordinates and interleaves
  the cell bits with x highest.  The quantisation decides integers, so it is
  taken in float32 exactly as the build takes it.
- clusters: 64 per mesh; cluster c holds the faces at sorted positions
  [ceil(c nt / 64), ceil((c + 1) nt / 64)).
- cluster statistics: the box of the cluster's vertices, the mean of its
  face centroids (a + b + c) / 3, and its area-weighted normal: the sum over
  faces of (b - a) x (c - a) / 2 divided by the sum of the face areas
  |(b - a) x (c - a)| / 2 (zero when the area is zero).
- pair features: the joint box of both meshes' non-empty clusters gives a
  centre C and a scale s (half its diagonal; 1 when that is zero); each
  cluster contributes (lo - C)/s, (hi - C)/s, (centroid - C)/s and its mean
  normal, 12 numbers, mesh A's 64 clusters then mesh B's; empty clusters
  contribute zeros.
- selection: the k largest logits of a row, ties to the lowest index.

Everything except the Morton quantisation is computed in float64.
"""
from __future__ import annotations

import numpy as np

CLUSTERS = 64
FEAT_PER_CLUSTER = 12


def _spread(v: np.ndarray, bits: int) -> np.ndarray:
    """Bit b of v moved to bit 3 b."""
    v = v.astype(np.uint64)
    out = np.zeros_like(v)
    for b in range(bits):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def morton_order(V, I, bits: int) -> np.ndarray:
    """Face indices in Morton order of their centroids (stable)."""
    V32 = np.asarray(V, np.float64).astype(np.float32)  # the stored coordinates (round to nearest)
    I = np.asarray(I, np.int64).reshape(-1, 3)
    lo, hi = V32.min(0), V32.max(0)
    cells = np.float32((1 << bits) - 1)
    ext = (hi - lo).astype(np.float32)
    scale = np.where(ext > 0, cells / np.where(ext > 0, ext, np.float32(1)), np.float32(0)).astype(np.float32)
    a, b, c = V32[I[:, 0]], V32[I[:, 1]], V32[I[:, 2]]
    cen = ((a + b) + c) * np.float32(1.0 / 3.0)
    q = np.minimum(np.maximum((cen - lo) * scale, np.float32(0)), cells).astype(np.uint32)
    key = (_spread(q[:, 0], bits) << np.uint64(2)) | (_spread(q[:, 1], bits) << np.uint64(1)) | _spread(q[:, 2], bits)
    return np.lexsort((np.arange(len(I)), key))


def cluster_ranges(nt: int):
    """[first, last) sorted positions of each of the 64 clusters."""
    return [(-(-c * nt // CLUSTERS), -(-(c + 1) * nt // CLUSTERS)) for c in range(CLUSTERS)]


def cluster_stats(V, I, order):
    """Per cluster: dict with lo, hi, centroid, normal_sum, area, count
    (float64; lo/hi of the float32 coordinates, empty clusters have
    count 0)."""
    V64 = np.asarray(V, np.float64).astype(np.float32).astype(np.float64)
    I = np.asarray(I, np.int64).reshape(-1, 3)
    F = V64[I[np.asarray(order)]]  # [nt, 3 vertices, 3]
    out = []
    for f0, f1 in cluster_ranges(len(I)):
        G = F[f0:f1]
        if len(G) == 0:
            out.append({"count": 0})
            continue
        a, b, c = G[:, 0], G[:, 1], G[:, 2]
        n = np.cross(b - a, c - a)
        out.append({"lo": G.reshape(-1, 3).min(0), "hi": G.reshape(-1, 3).max(0),
                    "centroid": ((a + b + c) / 3.0).mean(0), "normal_sum": 0.5 * n.sum(0),
                    "area": 0.5 * np.sqrt((n * n).sum(1)).sum(), "count": len(G)})
    return out


def pair_features(stats_a, stats_b) -> np.ndarray:
    """The 2 x 64 x 12 features of a mesh pair from both meshes' cluster
    statistics."""
    full = [s for s in stats_a + stats_b if s["count"] > 0]
    lo = np.min([s["lo"] for s in full], axis=0)
    hi = np.max([s["hi"] for s in full], axis=0)
    C = 0.5 * (lo + hi)
    s = 0.5 * float(np.sqrt(((hi - lo) ** 2).sum()))
    inv = 1.0 / s if s > 0 else 1.0
    X = np.zeros((2 * CLUSTERS, FEAT_PER_CLUSTER))
    for k, st in enumerate(stats_a + stats_b):
        if st["count"] == 0:
            continue
        X[k, 0:3] = (st["lo"] - C) * inv
        X[k, 3:6] = (st["hi"] - C) * inv
        X[k, 6:9] = (st["centroid"] - C) * inv
        X[k, 9:12] = st["normal_sum"] / st["area"] if st["area"] > 0 else 0.0
    return X.reshape(-1)


def mesh_pair_features(VA, IA, VB, IB, bits: int) -> np.ndarray:
    sa = cluster_stats(VA, IA, morton_order(VA, IA, bits))
    sb = cluster_stats(VB, IB, morton_order(VB, IB, bits))
    return pair_features(sa, sb)


def topk(logits, k: int) -> np.ndarray:
    """Indices of the k largest values of each row, largest first, ties to
    the lowest index."""
    Z = np.atleast_2d(np.asarray(logits, np.float64))
    out = np.zeros((len(Z), k), np.int64)
    for r, row in enumerate(Z):
        ranked = sorted(range(len(row)), key=lambda j: (-row[j], j))
        out[r] = ranked[:k]
    return out
