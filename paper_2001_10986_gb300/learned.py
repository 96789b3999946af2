"""Orchestration of the learned warm start: logging (features, target) pairs
from plain runs and training the network on them. Every computation runs in
the library's kernels (features, targets, forward, backward, Adam); this
module only loops over half-sweeps and batches, with torch holding the device
memory."""
from __future__ import annotations

import numpy as np

from . import dd, synthetic as syn


def log_pairs(mu, nu, b, levels, schedule, *, min_level=0, stream=None, **opts):
    """Run the schedule with the plain warm start and return the training pairs
    (features n×1089, targets n×64, CUDA tensors) of every half-sweep at a
    level ≥ min_level."""
    import torch
    g = dd.DD(mu, nu, b, levels, schedule, stream=stream, **opts)
    feats, tgts = [], []
    try:
        total = sum(s for _, s, _ in schedule)
        for _ in range(total):
            g.sweep(1)
            if g.info()[0] >= min_level:
                # pairs of the sweep's last (B) half-sweep
                f, t = g.training_pairs()
                feats.append(f)
                tgts.append(t)
    finally:
        g.close()
    return torch.cat(feats), torch.cat(tgts)


def train(pairs, *, epochs=30, batch=512, lr=1e-3, seed=0, init_seed=1, log=None):
    """Adam on the mean squared error over shuffled batches; returns the MLP."""
    import torch
    X, T = pairs
    net = dd.MLP(syn.mlp_init(init_seed))
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    n = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).to(X.device)
        tot = 0.0
        for k in range(0, n, batch):
            idx = perm[k:k + batch]
            tot += net.train_step(X[idx], T[idx], lr) * idx.numel()
        if log is not None:
            log(ep, tot / n)
    return net
