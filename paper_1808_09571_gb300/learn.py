"""Training and evaluation of the learned proposal (host orchestration).

The network, its features, loss, gradients and optimizer all run in the CUDA
library (g3d_pair_features, g3d_mlp_*); this module only generates training
pairs, labels them with the engine's own distance results (the cluster pair
holding the minimising face pair, from g3d_batch_ex), drives the training
loop and saves / restores checkpoints.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import geo3d, synth

CLUSTERS = 64


def he_init(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in [(1536, 256), (256, 256), (256, 256), (256, 4096)]:
        parts.append(rng.normal(0.0, np.sqrt(2.0 / i), size=i * o))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def make_pairs(n_pairs: int, seed: int, t_min: int, t_max: int, variants: int = 4):
    """Separated pairs of jittered spheres / tubes with face counts
    log-uniform in [t_min, t_max] (distance queries only), `variants`
    template shapes per kind and size bucket."""
    meshes, queries, info = synth.batch_workload(n_pairs, seed=seed, t_min=t_min, t_max=t_max, p_intersect=0.0,
                                                 gap_range=(1e-3, 0.5), variants=variants)
    return meshes, [(a, b, 0) for (a, b, _) in queries], info


def make_pairs_device(n_pairs: int, seed: int, t_min: int, t_max: int, variants: int = 4, device="cuda:0",
                      bank=None, cache=None):
    """The pairs of make_pairs (separated jittered spheres / tubes, face
    counts log-uniform in [t_min, t_max], gap log-uniform in [1e-3, 0.5]
    along a random direction, extreme vertices aligned), placed on the
    device: the template shapes are made on the host once per (kind, size
    bucket, variant), the per-pair rotations, offsets and extreme-vertex
    searches run as batched tensor operations over all instances of a
    template.  Draws the same per-pair parameters as make_pairs but rounds
    in a different order, so the float32 vertices are not bit-identical to
    it.  `bank` (a synth.TemplateBank) and `cache` (a dict of device copies
    of its templates) may be shared by several calls, so that a large
    training set draws on one set of shapes made once.  Returns (meshes
    [(V float32 [nv, 3] device, I int32 [nt, 3] device)], queries
    [(ia, ib, 0)])."""
    import math

    import torch
    rng = np.random.default_rng(seed)
    bank = bank if bank is not None else synth.TemplateBank(seed)
    cache = cache if cache is not None else {}
    lo, hi = math.log(t_min), math.log(t_max)
    glo, ghi = math.log(1e-3), math.log(0.5)
    keys, tdev = {}, []
    pa, pb, RA, RB, U, G = [], [], [], [], [], []
    for _ in range(n_pairs):
        tk = []
        for _ in range(2):
            kind = "sphere" if rng.random() < 0.5 else "tube"
            T = int(round(math.exp(rng.uniform(lo, hi))))
            V0, I0 = bank.get(kind, T, int(rng.integers(0, variants)))
            k = I0.ctypes.data
            if k not in keys:
                if k not in cache:
                    cache[k] = (torch.from_numpy(V0).to(device),
                                torch.from_numpy(np.ascontiguousarray(I0).view(np.int32)).to(device))
                keys[k] = len(tdev)
                tdev.append(cache[k])
            tk.append(keys[k])
        pa.append(tk[0])
        pb.append(tk[1])
        RA.append(synth.random_rotation(rng))
        RB.append(synth.random_rotation(rng))
        U.append(synth.random_unit(rng))
        G.append(math.exp(rng.uniform(glo, ghi)))
    RA = torch.from_numpy(np.stack(RA)).to(device)
    RB = torch.from_numpy(np.stack(RB)).to(device)
    U = torch.from_numpy(np.stack(U)).to(device)
    G = torch.from_numpy(np.asarray(G)).to(device)
    pa_t, pb_t = np.asarray(pa), np.asarray(pb)
    VA = [None] * n_pairs
    Q = torch.empty((n_pairs, 3), dtype=torch.float64, device=device)
    for t in np.unique(pa_t):  # side A: rotate, round, extreme vertex along u
        idx = np.nonzero(pa_t == t)[0]
        it = torch.from_numpy(idx).to(device)
        X = torch.matmul(tdev[t][0][None], RA[it].transpose(1, 2)).float()  # [k, nv, 3]
        Xd = X.double()
        j = torch.argmax(torch.einsum("knc,kc->kn", Xd, U[it]), dim=1)
        Q[it] = Xd[torch.arange(len(idx), device=device), j]
        for r, i in enumerate(idx):
            VA[i] = X[r]
    VB = [None] * n_pairs
    for t in np.unique(pb_t):  # side B: rotate, place at the gap beyond A's extreme vertex
        idx = np.nonzero(pb_t == t)[0]
        it = torch.from_numpy(idx).to(device)
        X = torch.matmul(tdev[t][0][None], RB[it].transpose(1, 2))
        j = torch.argmin(torch.einsum("knc,kc->kn", X, U[it]), dim=1)
        P = X[torch.arange(len(idx), device=device), j]
        off = Q[it] + G[it, None] * U[it] - P
        X = (X + off[:, None, :]).float()
        for r, i in enumerate(idx):
            VB[i] = X[r]
    meshes, queries = [], []
    for i in range(n_pairs):
        meshes += [(VA[i], tdev[pa[i]][1]), (VB[i], tdev[pb[i]][1])]
        queries.append((2 * i, 2 * i + 1, 0))
    return meshes, queries


def load(ctx: "geo3d.Context", meshes, device="cuda:0"):
    """Load and build meshes given as host arrays (copied to the device, an
    index array shared by several meshes once) or as device tensors."""
    import torch
    if meshes and isinstance(meshes[0][0], torch.Tensor):
        hs = ctx.mesh_load_many(list(meshes), copy_fp64_master=False)
        for c0 in range(0, len(hs), 60000):
            ctx.mesh_build_bvh_many(hs[c0:c0 + 60000])
        return hs
    uniq, dV, dI = {}, [], []
    for V, I in meshes:
        k = I.ctypes.data
        if k not in uniq:
            uniq[k] = torch.from_numpy(I.view(np.int32)).to(device)
        dI.append(uniq[k])
        dV.append(torch.from_numpy(V).to(device))
    hs = ctx.mesh_load_many(list(zip(dV, dI)), copy_fp64_master=False)
    for c0 in range(0, len(hs), 60000):
        ctx.mesh_build_bvh_many(hs[c0:c0 + 60000])
    return hs


def labels_of(ctx: "geo3d.Context", hs, queries):
    """Label = cA * 64 + cB, the clusters holding the face pair attaining each
    distance (computed by the library with the witness); -1 when the pair
    intersects or has no witness."""
    qs = [(hs[a], hs[b], 0) for (a, b, _) in queries]
    d, w, s, cl = ctx.batch_witness(qs)
    lab = np.where((s == 0) & (w >= 0), cl, -1).astype(np.int64)
    return lab, d


def train(mlp: "geo3d.MLP", X, labels, steps: int, batch: int = 256, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Minibatch Adam on (X [n x 1536] device tensor, labels [n] device int32).
    Returns the loss of every logged step."""
    import torch
    n = X.shape[0]
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    curve = []
    for t in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g, device=X.device)
        mlp.train_step(X[idx].contiguous(), labels[idx].contiguous(), lr, loss_out=loss)
        if log_every and (t % log_every == 0 or t == steps - 1):
            curve.append((t, float(loss.item())))
    return curve


def hit_rates(mlp: "geo3d.MLP", X, labels, ks=(1, 4, 16)):
    """Fraction of rows whose label is among the top-k logits."""
    import torch
    z = mlp.forward(X)
    out = {}
    lab = labels.long()
    for k in ks:
        top = torch.topk(z, k, dim=1).indices
        out[f"top{k}"] = float((top == lab[:, None]).any(dim=1).float().mean().item())
    return out


def save_checkpoint(path: str, mlp: "geo3d.MLP", meta: dict):
    """The library's checkpoint file (g3d_mlp_save) + a JSON description."""
    mlp.save(path + ".g3dmlp")
    with open(path + ".json", "w") as f:
        json.dump({"num_params": int(mlp.n), "dtype": "float32", **meta}, f)


def load_checkpoint(path: str, mlp: "geo3d.MLP") -> dict:
    meta = json.load(open(path + ".json"))
    mlp.load(path + ".g3dmlp")
    return meta
