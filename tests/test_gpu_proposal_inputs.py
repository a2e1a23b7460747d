"""The learned proposal's inputs and selection on the GPU against the
proposal oracle (oracle/proposal.py), through the C ABI.

- g3d_pair_features (the cluster statistics of both meshes in Morton order,
  then the 1,536 joint-frame features) element by element.  The GPU sums in
  float32 (per thread, then a warp and block tree): the mean of n terms
  carries an absolute error of about (n / 128 + 9) units of 2^-24 times the
  largest term, here (clusters of <= 1,000 faces, coordinates within a few
  units of the pair's box) below 1e-5 of the frame scale; box corners are
  exact before the frame transform (a few units of 2^-24).  Bar:
  |gpu - oracle| <= 2e-5 + 1e-5 |oracle|.
- g3d_proposal_topk: bit-exact indices (ties to the lowest index) on
  integer-valued logits full of ties.
"""
import numpy as np
import pytest

from oracle import proposal as P
from paper_1808_09571_gb300 import synth

pytestmark = pytest.mark.gpu


def _meshes():
    rng = np.random.default_rng(61)
    out = []
    for nt in (1, 10, 63, 64, 65, 500, 3001):
        M = synth.tiny_random_mesh(nt, rng, spread=1.5, size=0.3)
        out.append((M.V.astype(np.float32), M.I))
    V, I = synth.jittered_uv_sphere(20000, 1.0, rng)
    out.append((V.astype(np.float32), I))
    V, I = synth.small_tube(12000, rng)
    out.append((V.astype(np.float32), I))
    V, I = synth.box_mesh(2.0, 1.0, 0.5)
    out.append((V, I))  # float64 input: features of its float32 rounding
    return out


@pytest.mark.parametrize("bits", [8, 10])
def test_pair_features_match_oracle(g3d, bits):
    ctx = g3d.Context(0, morton_bits=bits, time_limit_ms=10000)
    ms = _meshes()
    hs = ctx.mesh_load_many(ms, copy_fp64_master=False)
    ctx.mesh_build_bvh_many(hs)
    pairs = [(i, j) for i in range(len(ms)) for j in range(len(ms)) if (i + 2 * j) % 3 == 0]
    X = ctx.pair_features([(hs[i], hs[j]) for i, j in pairs]).cpu().numpy().astype(np.float64)
    for r, (i, j) in enumerate(pairs):
        want = P.mesh_pair_features(ms[i][0], ms[i][1], ms[j][0], ms[j][1], bits)
        err = np.abs(X[r] - want)
        bad = err > 2e-5 + 1e-5 * np.abs(want)
        assert not bad.any(), (i, j, np.nonzero(bad)[0][:8], X[r][bad][:4], want[bad][:4])
        # empty clusters are exactly zero on both sides
        assert np.array_equal(X[r] == 0, want == 0) or not ((want == 0) & (X[r] != 0)).any()
    ctx.close()


@pytest.mark.parametrize("k", [1, 4, 8])
def test_topk_matches_oracle(g3d, k):
    import torch
    ctx = g3d.Context(0)
    rng = np.random.default_rng(100 + k)
    Z = rng.integers(-30, 30, size=(50, 4096)).astype(np.float32)
    Z[3] = 7.0  # one row entirely tied
    Z[4, 4095] = 1000.0  # the winner in the last position
    got = ctx.proposal_topk(torch.from_numpy(Z).cuda(), k).cpu().numpy()
    np.testing.assert_array_equal(got, P.topk(Z, k))
    assert list(got[3]) == list(range(k))
    assert got[4, 0] == 4095
    ctx.close()
