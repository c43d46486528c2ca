"""Pins of the learned scheduler's oracle (oracle/learned.py) against what does not depend on it:
central finite differences, closed forms of special parameter settings, and features worked out
by hand on a small point set."""
import numpy as np
import pytest

from oracle import learned as L


def random_problem(seed, n=40):
    rng = np.random.default_rng(seed)
    params = rng.normal(0, 0.4, L.N_PARAMS)
    x = rng.random((n, 8))
    y = np.c_[rng.random(n) * 5, (rng.random(n) < 0.3).astype(float)]
    return params, x, y


def test_parameter_count_matches_the_layout():
    assert L.N_PARAMS == 8 * 32 + 32 + 32 * 32 + 32 + 32 * 2 + 2 == 1410


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_equals_central_differences(seed):
    params, x, y = random_problem(seed)
    _, g = L.loss_grad(params, x, y)
    h = 1e-6
    rng = np.random.default_rng(100 + seed)
    for k in rng.choice(L.N_PARAMS, 60, replace=False):
        e = np.zeros(L.N_PARAMS)
        e[k] = h
        fd = (L.loss(params + e, x, y) - L.loss(params - e, x, y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_zero_last_layer_closed_form():
    """With W3 = 0 the outputs are b3 for every sample: the loss and the b3 gradient have closed
    forms and nothing flows back into the hidden layers."""
    params, x, y = random_problem(5)
    W1, b1, W2, b2, W3, b3 = L.unpack(params)
    p = params.copy()
    off3 = 8 * 32 + 32 + 32 * 32 + 32
    p[off3:off3 + 64] = 0.0
    b30, b31 = p[-2], p[-1]
    expect = np.mean((b30 - y[:, 0]) ** 2 + np.log1p(np.exp(b31)) - y[:, 1] * b31)
    val, g = L.loss_grad(p, x, y)
    assert abs(val - expect) < 1e-12
    assert abs(g[-2] - np.mean(2 * (b30 - y[:, 0]))) < 1e-12
    assert abs(g[-1] - np.mean(1 / (1 + np.exp(-b31)) - y[:, 1])) < 1e-12
    assert np.all(g[:off3] == 0.0)


def test_forward_of_a_hand_wired_network():
    """Only the path x0 -> h1[0] -> h2[0] -> out0 carries weight: out0 = 2 relu(x0) + 0.5."""
    p = np.zeros(L.N_PARAMS)
    p[0 * 32 + 0] = 1.0                       # W1[0][0]
    off2 = 8 * 32 + 32
    p[off2 + 0 * 32 + 0] = 1.0                # W2[0][0]
    off3 = off2 + 32 * 32 + 32
    p[off3 + 0 * 2 + 0] = 2.0                 # W3[0][0]
    p[-2] = 0.5
    x = np.zeros((3, 8))
    x[:, 0] = [1.5, -2.0, 0.25]
    out, _ = L.forward(p, x)
    assert np.allclose(out[:, 0], [3.5, 0.5, 1.0]) and np.allclose(out[:, 1], 0.0)


def test_features_worked_by_hand():
    """The 8 cube corners and the centre: a 2 x 2 x 2 grid (nine points), the centre shares the
    top cell with corner (1, 1, 1)."""
    corners = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=float)
    pts = np.vstack([corners, [[0.5, 0.5, 0.5]]])
    keys = np.array([(5 << 57) | (7 << 51)] * 9, dtype=np.uint64)
    rounds = np.array([0] * 8 + [3])
    dup = np.zeros(9, dtype=bool)
    f = L.features(pts, keys, rounds, dup, [0, 0, 0, 1, 1, 1])
    # corner (0,0,0): alone in its cell, three neighbours with one point each
    assert np.allclose(f[0], [1 / 8, 1 / 8, 0, 0, 5 / 64, 7 / 64, 0, 0])
    # corner (1,1,1): cell (1,1,1) holds it and the centre; neighbours (0,1,1), (1,0,1), (1,1,0)
    assert np.allclose(f[7], [np.log2(3) / 8, 1 / 8, 0, 0.25, 5 / 64, 7 / 64, 0, 0])
    # the centre: same cell, in the middle of the box
    assert np.allclose(f[8], [np.log2(3) / 8, 1 / 8, 0, 0.25, 5 / 64, 7 / 64, 3 / 8, 1.0])
    # corner (1,0,0): cell (1,0,0), neighbours (0,0,0), (1,1,0), (1,0,1): counts 1, 1, 1
    assert np.allclose(f[1][:4], [1 / 8, 1 / 8, 0, 0])
    # a duplicate is not counted
    f2 = L.features(pts, keys, rounds, np.array([False] * 8 + [True]), [0, 0, 0, 1, 1, 1])
    assert np.allclose(f2[7][:4], [1 / 8, 1 / 8, 0, 0])


def test_grid_bits_about_four_points_per_cell():
    assert L.grid_bits(9) == 1
    assert L.grid_bits(4 * 512) == 3 and L.grid_bits(4 * 512 - 1) == 2
    assert L.grid_bits(10 ** 9) == 8
