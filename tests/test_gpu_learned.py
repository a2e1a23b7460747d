"""The learned proposal through the C ABI: GEMM / gradient / optimizer parity
with the FP64 oracle, exactness of results whatever the network predicts,
and what the trained network gains."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


def bf16(x):
    """Round float32 values to bfloat16 (nearest even), as float64."""
    a = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    a = ((a + (((a >> 16) & 1) + 0x7FFF)) >> 16) << 16
    return a.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def ctx(g3d):
    c = g3d.Context(0, time_limit_ms=10000)
    yield c
    c.close()


@pytest.mark.parametrize("rows", [1, 37, 128, 300, 1029])
def test_forward_matches_bf16_oracle(ctx, g3d, rows):
    """The forward pass (tcgen05 GEMMs: 128-row tiles, so 1, 37 and 300
    rows end in a partial tile, 1,029 spans 9 tiles) against the oracle."""
    import torch
    rng = np.random.default_rng(3 + rows)
    p = M.init_params(7)
    p[-4096:] = rng.normal(0, 0.1, 4096)
    mlp = g3d.MLP(ctx, p)
    X = rng.normal(0, 1, (rows, 1536)).astype(np.float32)
    z = mlp.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    # oracle with every GEMM operand rounded to bfloat16, FP32-exact bias
    h = X.astype(np.float64)
    for li, (W, b) in enumerate(M.unpack(p.astype(np.float64))):
        h = bf16(h) @ bf16(W) + b
        if li < 3:
            h = np.maximum(h, 0.0)
    err = np.abs(z - h)
    assert err.max() <= 1e-2 * np.abs(h).max(), err.max()
    assert err.mean() <= 1e-3 * np.abs(h).mean(), err.mean()
    mlp.close()


def test_gradients_match_oracle(ctx, g3d):
    """Against the oracle with bfloat16-rounded matrix operands (the GPU's
    arithmetic): tight.  Against the exact FP64 oracle: the bfloat16 error
    of a 4-layer backward, stated per tensor."""
    import torch
    rng = np.random.default_rng(4)
    p = M.init_params(8)
    mlp = g3d.MLP(ctx, p)
    X = rng.normal(0, 1, (64, 1536)).astype(np.float32)
    lab = rng.integers(0, 4096, 64).astype(np.int32)
    g, loss = mlp.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(lab).cuda())
    loss_e, g_e = M.loss_and_grad(p, X, lab, rnd=bf16)
    loss_ref, g_ref = M.loss_and_grad(p, X, lab)
    assert abs(loss - loss_e) <= 1e-3 * loss_e
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    k = 0
    for i, o in M.DIMS:
        for size in (i * o, o):
            a = g[k:k + size].astype(np.float64)
            e, b = g_e[k:k + size], g_ref[k:k + size]
            k += size

            def cos_rel(u, v):
                return (float(u @ v / (np.linalg.norm(u) * np.linalg.norm(v) + 1e-300)),
                        float(np.linalg.norm(u - v) / (np.linalg.norm(v) + 1e-300)))
            ce, re = cos_rel(a, e)
            cr, rr = cos_rel(a, b)
            assert ce >= 0.9995 and re <= 0.03, ("emulated", i, o, size, ce, re)
            assert cr >= 0.99 and rr <= 0.15, ("fp64", i, o, size, cr, rr)
    mlp.close()


def test_adam_step_matches_numpy(ctx, g3d):
    import torch
    rng = np.random.default_rng(5)
    p = M.init_params(9)
    mlp = g3d.MLP(ctx, p)
    X = torch.from_numpy(rng.normal(0, 1, (32, 1536)).astype(np.float32)).cuda()
    lab = torch.from_numpy(rng.integers(0, 4096, 32).astype(np.int32)).cuda()
    g, _ = mlp.gradients(X, lab)
    mlp.train_step(X, lab, 1e-3)
    q = mlp.get_params()
    m = 0.1 * g.astype(np.float64)
    v = 0.001 * g.astype(np.float64) ** 2
    expect = p - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    np.testing.assert_allclose(q, expect, rtol=1e-4, atol=1e-6)
    mlp.close()


@pytest.fixture(scope="module")
def trained(ctx, g3d):
    """A proposal trained on 768 method-labelled pairs."""
    import torch
    from paper_1808_09571_gb300 import learn
    meshes, queries, _ = learn.make_pairs(768, seed=11, t_min=2000, t_max=16000)
    hs = learn.load(ctx, meshes)
    lab, _ = learn.labels_of(ctx, hs, queries)
    keep = np.nonzero(lab >= 0)[0]
    X = ctx.pair_features([(hs[queries[i][0]], hs[queries[i][1]]) for i in keep])
    Y = torch.from_numpy(lab[keep].astype(np.int32)).cuda()
    mlp = g3d.MLP(ctx, learn.he_init(1))
    curve = learn.train(mlp, X, Y, steps=400, batch=256, lr=1e-3, log_every=100)
    ctx.mesh_free_many(hs)
    yield mlp, curve
    mlp.close()


def test_training_lowers_the_loss(trained):
    mlp, curve = trained
    assert curve[-1][1] < 0.7 * curve[0][1], curve


def test_proposal_never_changes_results(ctx, g3d, trained):
    from paper_1808_09571_gb300 import learn
    mlp, _ = trained
    meshes, queries, _ = learn.make_pairs(96, seed=12, t_min=1000, t_max=20000)
    hs = learn.load(ctx, meshes)
    qs = [(hs[a], hs[b], 0) for (a, b, _) in queries] + [(hs[a], hs[b], 1) for (a, b, _) in queries[:20]]
    ctx.set_proposal(None)
    d0, h0, s0 = ctx.batch(qs)
    rnd = g3d.MLP(ctx, learn.he_init(99))
    gate0 = ctx.config()["proposal_min_faces"]
    # every query proposed for, those of two meshes of >= 8,192 faces, none
    for gate in (1, 8192, 1 << 30):
        ctx.set_config(proposal_min_faces=gate)
        for prop in (rnd, mlp):
            ctx.set_proposal(prop)
            d1, h1, s1 = ctx.batch(qs)
            assert (s1 == 0).all()
            np.testing.assert_array_equal(d1, d0)
            np.testing.assert_array_equal(h1, h0)
    ctx.set_proposal(None)
    ctx.set_config(proposal_min_faces=gate0)
    rnd.close()
    ctx.mesh_free_many(hs)


def test_trained_proposal_gain(ctx, g3d, trained):
    """Held-out pairs: the trained network ranks the true cluster pair far
    above chance, and the bound its proposal seeds is tighter than the one
    an untrained network's proposal seeds (proposal dives only add
    candidates, so neither is looser than no proposal)."""
    from paper_1808_09571_gb300 import learn
    mlp, _ = trained
    # both meshes of every pair above the size from which the network
    # proposes (8,192 faces)
    meshes, queries, _ = learn.make_pairs(192, seed=13, t_min=8192, t_max=16000)
    hs = learn.load(ctx, meshes)
    lab, _ = learn.labels_of(ctx, hs, queries)
    keep = np.nonzero(lab >= 0)[0]
    import torch
    X = ctx.pair_features([(hs[queries[i][0]], hs[queries[i][1]]) for i in keep])
    rates = learn.hit_rates(mlp, X, torch.from_numpy(lab[keep].astype(np.int32)).cuda())
    assert rates["top16"] > 10 * 16 / 4096, rates
    qs = [(hs[a], hs[b], 0) for (a, b, _) in queries]
    rnd = g3d.MLP(ctx, learn.he_init(98))
    work = {}
    for name, prop in (("none", None), ("untrained", rnd), ("trained", mlp)):
        ctx.set_proposal(prop)
        ctx.batch(qs)
        ctx.stats_reset()
        ctx.batch(qs)
        st = ctx.stats()
        work[name] = {k: st[k] for k in ("node_pairs", "tri_tests", "candidates")}
        # mean excess of the seeded bound over the distance (deterministic:
        # the bound after the dives does not depend on warp timing)
        work[name]["seed_excess"] = st["seed_excess_ppm"] / 1e6 / max(1, st["seed_queries"])
    ctx.set_proposal(None)
    print("hit rates", rates, "work", work)
    assert work["trained"]["seed_excess"] < work["untrained"]["seed_excess"], work
    assert work["untrained"]["seed_excess"] <= work["none"]["seed_excess"], work
    rnd.close()
    ctx.mesh_free_many(hs)


def test_checkpoint_round_trip(ctx, g3d, tmp_path):
    rng = np.random.default_rng(6)
    p = M.init_params(10)
    p[-4096:] = rng.normal(0, 0.1, 4096)
    a = g3d.MLP(ctx, p)
    a.save(str(tmp_path / "net.g3dmlp"))
    b = g3d.MLP(ctx)
    b.load(str(tmp_path / "net.g3dmlp"))
    np.testing.assert_array_equal(b.get_params(), a.get_params())
    (tmp_path / "short.g3dmlp").write_bytes((tmp_path / "net.g3dmlp").read_bytes()[:1000])
    with pytest.raises(g3d.G3DError):
        b.load(str(tmp_path / "short.g3dmlp"))
    (tmp_path / "other.g3dmlp").write_bytes(b"NOTAMLP!" + bytes(16))
    with pytest.raises(g3d.G3DError):
        b.load(str(tmp_path / "other.g3dmlp"))
    with pytest.raises(g3d.G3DError):
        b.load(str(tmp_path / "missing.g3dmlp"))
    a.close()
    b.close()


def test_training_loop_on_the_device(ctx, g3d):
    """g3d_mlp_train: minibatches drawn on the device; the loss drops on a
    small labelled set and the same seed repeats the run exactly."""
    import torch
    rng = np.random.default_rng(12)
    X = torch.from_numpy(rng.normal(0, 1, (300, 1536)).astype(np.float32)).cuda()
    Y = torch.from_numpy(rng.integers(0, 4096, 300).astype(np.int32)).cuda()
    from paper_1808_09571_gb300 import learn
    runs = []
    for _ in range(2):
        m = g3d.MLP(ctx, learn.he_init(3))
        first = m.train(X, Y, steps=1, batch=64, lr=1e-3, seed=7)
        last = m.train(X, Y, steps=300, batch=64, lr=1e-3, seed=8)
        runs.append(m.get_params())
        m.close()
    assert last < 0.5 * first, (first, last)
    np.testing.assert_array_equal(runs[0], runs[1])


def test_checkpoint_resumes_training_exactly(ctx, g3d, tmp_path):
    """A checkpoint carries Adam's state: stopping, saving, loading into a
    new network and continuing gives the parameters of the uninterrupted run."""
    import torch
    from paper_1808_09571_gb300 import learn
    rng = np.random.default_rng(13)
    X = torch.from_numpy(rng.normal(0, 1, (200, 1536)).astype(np.float32)).cuda()
    Y = torch.from_numpy(rng.integers(0, 4096, 200).astype(np.int32)).cuda()
    a = g3d.MLP(ctx, learn.he_init(4))
    a.train(X, Y, steps=50, batch=32, seed=1)
    a.train(X, Y, steps=50, batch=32, seed=2)
    b = g3d.MLP(ctx, learn.he_init(4))
    b.train(X, Y, steps=50, batch=32, seed=1)
    b.save(str(tmp_path / "mid.g3dmlp"))
    c = g3d.MLP(ctx)
    c.load(str(tmp_path / "mid.g3dmlp"))
    c.train(X, Y, steps=50, batch=32, seed=2)
    np.testing.assert_array_equal(c.get_params(), a.get_params())
    for m in (a, b, c):
        m.close()
