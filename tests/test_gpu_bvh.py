"""The BVH build kernels (ingest, Morton codes, segmented radix sort, gather,
radix tree, refit) checked through the exported tree against the build's
rules recomputed on the host:

- the face order is a stable sort of the Morton keys, which the host
  recomputes with the same float32 operations (vertex box of the float32
  coordinates, centroid (a + b + c) * (1/3), cell = trunc((c - lo) * cells /
  extent) clamped, x bits highest) -- an independent sort (numpy lexsort);
- face ids are a permutation; leaf k holds faces [k L, k L + L) in that order
  and its box is exactly their min / max;
- every internal node's child boxes are exactly the leaf boxes or the unions
  of the children's boxes; every leaf is reached once from the root and the
  leaf counts below each child add up."""
import numpy as np
import pytest

from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu


def spread10(v):
    v = v.astype(np.uint64) & 0x3FF
    out = np.zeros_like(v)
    for b in range(10):
        out |= ((v >> b) & 1) << (3 * b)
    return out


def host_order(V, I, bits):
    V32 = np.asarray(V, np.float64).astype(np.float32)  # round to nearest, as the ingest does
    lo, hi = V32.min(0), V32.max(0)
    cells = np.float32((1 << bits) - 1)
    e = (hi - lo).astype(np.float32)
    sc = np.where(e > 0, cells / np.where(e > 0, e, np.float32(1)), np.float32(0)).astype(np.float32)
    a, b, c = V32[I[:, 0]], V32[I[:, 1]], V32[I[:, 2]]
    cen = ((a + b) + c) * np.float32(1.0 / 3.0)
    q = np.minimum(np.maximum((cen - lo) * sc, np.float32(0)), cells).astype(np.uint32)
    key = (spread10(q[:, 0]) << 2) | (spread10(q[:, 1]) << 1) | spread10(q[:, 2])
    return np.lexsort((np.arange(len(I)), key)), V32


def check_tree(T, V32, I, L):
    nt = len(I)
    ids = T["face_ids"]
    nleaf = len(T["leaf_lo"])
    assert nleaf == (nt + L - 1) // L
    assert np.array_equal(np.sort(ids), np.arange(nt))
    F = V32[I[ids]]  # [nt, 3, 3] in BVH order
    for k in range(nleaf):
        f = F[k * L:(k + 1) * L].reshape(-1, 3)
        assert T["leaf_first"][k] == k * L and T["leaf_count"][k] == min(L, nt - k * L)
        assert np.array_equal(T["leaf_lo"][k], f.min(0)) and np.array_equal(T["leaf_hi"][k], f.max(0))
    if nleaf == 1:
        return
    seen_leaf = np.zeros(nleaf, int)
    seen_node = np.zeros(nleaf - 1, int)

    def box_of(ref):
        if ref < 0:
            return T["leaf_lo"][~ref], T["leaf_hi"][~ref], 1
        lo = np.minimum(T["node_lo"][ref, 0], T["node_lo"][ref, 1])
        hi = np.maximum(T["node_hi"][ref, 0], T["node_hi"][ref, 1])
        return lo, hi, int(T["node_below"][ref].sum())

    stack = [0]
    seen_node[0] = 1
    while stack:
        n = stack.pop()
        for c in range(2):
            ref = int(T["node_child"][n, c])
            lo, hi, below = box_of(ref)
            assert np.array_equal(T["node_lo"][n, c], lo) and np.array_equal(T["node_hi"][n, c], hi), (n, c)
            assert T["node_below"][n, c] == below, (n, c)
            if ref < 0:
                seen_leaf[~ref] += 1
            else:
                seen_node[ref] += 1
                stack.append(ref)
    assert np.all(seen_leaf == 1) and np.all(seen_node == 1)


def cases():
    rng = np.random.default_rng(17)
    soup = synth.tiny_random_mesh(3000, rng, spread=2.0, size=0.2, dtype=np.float32)
    ore = synth.small_ore_body()
    tube, _ = synth.drill_hole(700, seed=3)
    ico, _ = synth.small_pairs()["A"]
    return {"soup_random_order": (soup.V, soup.I), "ore_500": (ore.V, ore.I),
            "tube_22k": (tube.V.astype(np.float32), tube.I), "icosphere_fp64": (ico.V, ico.I)}


@pytest.mark.parametrize("L,bits", [(16, 10), (8, 8), (4, 10), (2, 9)])
def test_bvh_against_host_rules(g3d, L, bits):
    ctx = g3d.Context(0, leaf_size=L, morton_bits=bits)
    for name, (V, I) in cases().items():
        m = ctx.load_and_build(V, I)
        T = ctx.mesh_export(m)
        order, V32 = host_order(V, I, bits)
        assert np.array_equal(T["face_ids"], order), name
        check_tree(T, V32, I, L)
        ctx.mesh_free(m)
    ctx.close()
