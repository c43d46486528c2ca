"""The learned scheduler's training loop: round logs of the plain schedule in, parameters out.

Every step runs in the library's kernels: a plain dt_insert with DT_FLAG_LOG records, per point,
the cavity size of its insertion and whether it lost a conflict first; dt_get_features computes
the point's features; dt_mlp_train fits the network with Adam on the GPU. This module only
strings those calls together.
"""
from __future__ import annotations

import numpy as np

from . import DT_FLAG_LOG, Triangulation, _torch, init_params, mlp_train


def collect(clouds, seed: int = 0):
    """Labelled feature rows (CUDA float32 x [m, 8], y [m, 2]) from plain logged inserts of the
    given clouds (host float64 arrays [n, 3])."""
    torch = _torch()
    xs, ys = [], []
    for xyz in clouds:
        pts = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float64)).cuda()
        with Triangulation(seed=seed, flags=DT_FLAG_LOG) as t:
            t.insert(pts)
            x, y, valid = t.features(len(xyz))
        keep = valid.bool()
        xs.append(x[keep])
        ys.append(y[keep])
    return torch.cat(xs), torch.cat(ys)


def train(x, y, steps: int = 3000, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Fits the network on (x, y) with the GPU kernels; returns (params numpy float32 [1410],
    per-step minibatch losses)."""
    torch = _torch()
    params = torch.from_numpy(init_params(seed)).cuda()
    losses = mlp_train(params, x, y, steps, batch, lr, seed)
    return params.cpu().numpy(), losses


def train_scheduler(clouds, steps: int = 3000, seed: int = 0):
    """Round logs of the plain schedule on `clouds`, then training: the scheduler's parameters."""
    x, y = collect(clouds, seed)
    params, losses = train(x, y, steps=steps, seed=seed)
    return params, losses
