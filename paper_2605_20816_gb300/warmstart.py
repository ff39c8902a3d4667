"""Training data and training loop of the learned warm start.

Every diagram is drawn with the seeded generator (synth.poly_params),
rasterised with pd_assign, compacted to its non-empty grains; the inputs are
pd_mlp_features of the labels and the targets pd_mlp_targets of the
generating parameters.  Training runs pd_mlp_train_step (the library's own
forward, backward and Adam kernels) on shuffled minibatches.  Only the
plumbing (concatenation, shuffling) happens in torch here.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pd, synth


def diagram(seed: int, shape, N: int, d: int = 4):
    """(grid, labels CUDA int32, N_eff, theta CUDA float64) of one seeded
    degree-d polynomial diagram."""
    dim = len(shape)
    K = pd.pd_K(dim, d)
    y, z = synth.poly_params(seed, N, dim, K)
    th = pd.pd_theta_from_apd(dim, d, y, np.zeros(N)).numpy()
    th[:, dim + 1:] = z[:, dim + 1:]
    grid = pd.Grid(shape)
    lab, _, _ = pd.pd_assign(grid, N, d, torch.from_numpy(th).cuda())
    lab, n_eff, used = synth.compact(lab.cpu().numpy())
    return grid, torch.from_numpy(lab.astype(np.int32)).cuda(), n_eff, torch.from_numpy(
        np.ascontiguousarray(th[used])).cuda()


def dataset(n_diagrams: int, seed0: int = 5_000_000, side: int = 256, grains=(50, 400), d: int = 4):
    """Inputs [G, 135] and targets [G, K] over all grains of n_diagrams maps."""
    rng = synth.rng(seed0)
    Ns = rng.integers(grains[0], grains[1] + 1, size=n_diagrams)
    X, T = [], []
    for q in range(n_diagrams):
        grid, lab, n, th = diagram(seed0 + 1 + q, (side, side), int(Ns[q]), d)
        X.append(pd.pd_mlp_features(grid, lab, n))
        T.append(pd.pd_mlp_targets(th))
    return torch.cat(X), torch.cat(T)


def train(net: pd.MLP, X, T, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
    """Adam on shuffled minibatches; returns the per-epoch mean losses."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    n = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot, cnt = 0.0, 0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            if idx.numel() < 2:
                continue
            loss = net.train_step(X.index_select(0, idx).contiguous(), T.index_select(0, idx).contiguous(), lr)
            tot += float(loss.item()) * idx.numel()
            cnt += idx.numel()
        losses.append(tot / max(cnt, 1))
    return losses
