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


def load(ctx: "geo3d.Context", meshes, device="cuda:0"):
    import torch
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
