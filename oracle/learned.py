"""Oracle of the learned scheduler's arithmetic (TEST INFRASTRUCTURE ONLY: used by the tests and
the benchmark's CPU legs, never by the product path).

Plain float64 numpy, written from the definitions, sharing no code with the CUDA kernels:
  * the network 8 -> 32 -> 32 -> 2 with ReLU hidden layers (parameter layout W1[8][32], b1[32],
    W2[32][32], b2[32], W3[32][2], b3[2], W[i][j] = input i -> output j);
  * its loss per sample, (o0 - y0)^2 + softplus(o1) - y1 * o1, averaged, and the gradient of
    that mean by backpropagation written out layer by layer;
  * the eight per-point features of the scheduler from a point set in insertion order;
  * training: Adam with bias correction (Kingma and Ba, "Adam: a method for stochastic
    optimization", ICLR 2015, Algorithm 1; beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on
    minibatches drawn with replacement by a counter-based SplitMix64 hash (Steele, Lea and
    Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
The paper has no learned component; these definitions are the repository's own (the scheduler
only reorders insertions, so the tetrahedra never depend on them).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 8, 32, 2
SHAPES = [(N_IN, N_H), (N_H,), (N_H, N_H), (N_H,), (N_H, N_OUT), (N_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(params):
    p = np.asarray(params, dtype=np.float64).ravel()
    assert p.size == N_PARAMS
    out, k = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(p[k:k + n].reshape(s))
        k += n
    return out


def forward(params, x):
    """Outputs [n, 2] and the hidden activations (pre- and post-ReLU) of rows x [n, 8]."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    out = h2 @ W3 + b3
    return out, (z1, h1, z2, h2)


def softplus(z):
    return np.logaddexp(0.0, z)


def loss(params, x, y):
    out, _ = forward(params, x)
    y = np.asarray(y, dtype=np.float64)
    per = (out[:, 0] - y[:, 0]) ** 2 + softplus(out[:, 1]) - y[:, 1] * out[:, 1]
    return float(per.mean())


def loss_grad(params, x, y):
    """(mean loss, gradient [1410]) by backpropagation."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[0]
    out, (z1, h1, z2, h2) = forward(params, x)
    per = (out[:, 0] - y[:, 0]) ** 2 + softplus(out[:, 1]) - y[:, 1] * out[:, 1]
    # d(mean loss)/d(out)
    d_out = np.empty_like(out)
    d_out[:, 0] = 2.0 * (out[:, 0] - y[:, 0]) / n
    d_out[:, 1] = (1.0 / (1.0 + np.exp(-out[:, 1])) - y[:, 1]) / n
    gW3 = h2.T @ d_out
    gb3 = d_out.sum(axis=0)
    d_h2 = d_out @ W3.T
    d_z2 = d_h2 * (z2 > 0)
    gW2 = h1.T @ d_z2
    gb2 = d_z2.sum(axis=0)
    d_h1 = d_z2 @ W2.T
    d_z1 = d_h1 * (z1 > 0)
    gW1 = x.T @ d_z1
    gb1 = d_z1.sum(axis=0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return float(per.mean()), g


def grid_bits(n):
    """Feature grid: about four points per cell, 1..8 bits per axis."""
    g = 1
    while g < 8 and (1 << (3 * (g + 1))) * 4 <= n:
        g += 1
    return g


def features(xyz_sorted, keys_sorted, rounds_sorted, dup_sorted, bbox):
    """The scheduler's features of points given in insertion order.

    For a point in cell c of a 2^g-per-axis grid over the box (c = floor((x - lo) * 2^g / ext),
    clamped), with n_c the number of non-duplicate points in c and the 6 face neighbours that
    exist inside the grid:
      0: log2(1 + n_c) / 8          1: log2(1 + mean of the neighbours) / 8
      2: (log2(1 + max) - log2(1 + min)) / 8 over the neighbours
      3: (n_c - mean) / (1 + n_c + mean)
      4: bits 57..62 of the Moore key / 64     5: bits 51..56 / 64
      6: BRIO round / 8              7: 2 min over axes of min(u, 1 - u), u = (x - lo) / ext
    """
    P = np.asarray(xyz_sorted, dtype=np.float64)
    n = P.shape[0]
    g = grid_bits(n)
    G = 1 << g
    lo = np.asarray(bbox[:3], dtype=np.float64)
    ext = np.asarray(bbox[3:], dtype=np.float64) - lo
    scale = np.where(ext > 0, G / np.where(ext > 0, ext, 1.0), 0.0)
    q = np.clip(np.floor((P - lo) * scale), 0, G - 1).astype(np.int64)
    u = np.where(ext > 0, (P - lo) / np.where(ext > 0, ext, 1.0), 0.5)
    u = np.clip(u, 0.0, 1.0)
    count = np.zeros((G, G, G), dtype=np.int64)  # [z][y][x]
    keep = ~np.asarray(dup_sorted, dtype=bool)
    np.add.at(count, (q[keep, 2], q[keep, 1], q[keep, 0]), 1)
    out = np.zeros((n, 8), dtype=np.float64)
    for s in range(n):
        cx, cy, cz = q[s]
        nc = count[cz, cy, cx]
        nb = []
        for d in range(3):
            for e in (-1, 1):
                r = [cx, cy, cz]
                r[d] += e
                if 0 <= r[d] < G:
                    nb.append(count[r[2], r[1], r[0]])
        mean = float(np.mean(nb)) if nb else float(nc)
        mx = max(nb) if nb else nc
        mn = min(nb) if nb else nc
        key = int(keys_sorted[s])
        out[s] = [np.log2(1 + nc) / 8, np.log2(1 + mean) / 8, (np.log2(1 + mx) - np.log2(1 + mn)) / 8,
                  (nc - mean) / (1 + nc + mean), ((key >> 57) & 63) / 64, ((key >> 51) & 63) / 64,
                  int(rounds_sorted[s]) / 8, 2 * min(min(u[s, k], 1 - u[s, k]) for k in range(3))]
    return out


# ------------------------------------------------------------------ training
_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15  # SplitMix64's increment
_STEP_SALT = 0x51ED2701        # per-step seed offset of the minibatch draw


def splitmix64_mix(z: int) -> int:
    """SplitMix64's output function (Steele, Lea, Flood 2014) on one 64-bit integer."""
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def draw_indices(n: int, batch: int, seed: int) -> np.ndarray:
    """Minibatch of `batch` sample indices in [0, n), with replacement: index k is
    mix(seed + (k + 1) * golden) mod n, i.e. output k of a SplitMix64 stream started at seed."""
    return np.array([splitmix64_mix(seed + (k + 1) * _GOLDEN) % n for k in range(batch)], dtype=np.int64)


def adam_step(params, grad, m, v, lr: float, t: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update at step t >= 1 (Kingma and Ba 2015, Algorithm 1):
    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
    p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  Returns (p, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    p = np.asarray(params, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return p, m, v


def train(params, x, y, steps: int, batch: int, lr: float, seed: int):
    """`steps` Adam steps from zero moments; step t (0-based) draws its minibatch with seed
    seed + (t + 1) * 0x51ED2701 (mod 2^64) and takes the gradient of the minibatch's mean loss.
    Returns (params, per-step minibatch losses)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = np.asarray(params, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for t in range(steps):
        idx = draw_indices(len(x), batch, (seed + (t + 1) * _STEP_SALT) & _MASK64)
        L, g = loss_grad(p, x[idx], y[idx])
        losses.append(L)
        p, m, v = adam_step(p, g, m, v, lr, t + 1)
    return p, np.array(losses)
