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


# ------------------------------------------------------------------ training: draw and Adam
import json  # noqa: E402
import os  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")


def test_splitmix64_published_outputs():
    """The draw's generator reproduces SplitMix64's published reference outputs."""
    with open(GOLDEN) as f:
        g = json.load(f)
    for s in g["streams"]:
        want = [int(v, 0) for v in s["outputs"]]
        got = [L.splitmix64_mix(s["initial_state"] + (k + 1) * 0x9E3779B97F4A7C15) for k in range(len(want))]
        assert got == want


def test_draw_is_the_published_stream_mod_n():
    with open(GOLDEN) as f:
        s = json.load(f)["streams"][1]
    want = [int(v) for v in s["outputs"]]
    for n in (1, 7, 1000, 2 ** 31 + 11):
        assert L.draw_indices(n, len(want), s["initial_state"]).tolist() == [v % n for v in want]


def test_draw_is_uniform():
    """Chi-square over 16 buckets of 64k draws stays below the 0.999 quantile (37.7, 15 dof)."""
    idx = L.draw_indices(16, 1 << 16, 12345)
    counts = np.bincount(idx, minlength=16)
    e = len(idx) / 16
    assert ((counts - e) ** 2 / e).sum() < 37.7


def test_adam_first_step_moves_by_lr_times_sign():
    """At t = 1 bias correction gives m_hat = g and v_hat = g^2: p - lr g / (|g| + eps)."""
    p = np.array([1.0, -2.0, 0.5, 3.0, 0.0])
    g = np.array([0.3, -4.0, 0.0, 1e-3, -2e-8])
    q, m, v = L.adam_step(p, g, np.zeros(5), np.zeros(5), 0.01, 1)
    e = 1e-8
    want = [1.0 - 0.01 * 0.3 / (0.3 + e), -2.0 + 0.01 * 4.0 / (4.0 + e), 0.5,
            3.0 - 0.01 * 1e-3 / (1e-3 + e), 0.01 * 2e-8 / (2e-8 + e)]
    assert np.allclose(q, want, rtol=0, atol=1e-14)
    assert np.allclose(q[:2], [0.99, -1.99], atol=1e-9)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_moves_linearly():
    """A constant gradient keeps m_hat = g and v_hat = g^2 at every step: k steps move by
    k lr g / (|g| + eps)."""
    p = np.array([1.0, 2.0])
    g = np.array([0.5, -0.25])
    m = v = np.zeros(2)
    q = p
    for t in range(1, 8):
        q, m, v = L.adam_step(q, g, m, v, 0.1, t)
    assert np.allclose(q, p - 7 * 0.1 * np.sign(g), atol=1e-7)


def test_adam_two_steps_worked_by_hand():
    """g = 1 then g = -1 (lr = 1): after step 1, p = 1 - 1/(1 + eps); at step 2,
    m = 0.9 * 0.1 - 0.1 = -0.01, m_hat = -0.01 / 0.19 = -1/19; v = 0.999 * 0.001 + 0.001,
    v_hat = 0.001999 / 0.001999 = 1, so p moves by +(1/19) / (1 + eps)."""
    eps = 1e-8
    q, m, v = L.adam_step(np.array([1.0]), np.array([1.0]), np.zeros(1), np.zeros(1), 1.0, 1)
    assert abs(q[0] - (1 - 1 / (1 + eps))) < 1e-15
    q, m, v = L.adam_step(q, np.array([-1.0]), m, v, 1.0, 2)
    assert abs(m[0] + 0.01) < 1e-15 and abs(v[0] - 0.001999) < 1e-15
    assert abs(q[0] - (1 - 1 / (1 + eps) + (1 / 19) / (1 + eps))) < 1e-12


def test_adam_zero_gradient_keeps_parameters():
    q, m, v = L.adam_step(np.array([1.0, -1.0]), np.zeros(2), np.array([0.2, 0.0]), np.array([0.0, 0.0]), 0.1, 3)
    # m decays, v stays 0: the move is lr * m_hat / eps on the first entry, none on the second
    assert abs(m[0] - 0.18) < 1e-15 and q[1] == -1.0


def test_train_on_one_sample_is_one_adam_step_on_its_gradient():
    """n = 1: every draw picks sample 0, so one training step is p - lr g / (|g| + eps) with g
    the sample's gradient, here taken by central differences."""
    params, x, y = random_problem(11, n=1)
    lr = 1e-3
    q, losses = L.train(params, x, y, steps=1, batch=4, lr=lr, seed=9)
    h = 1e-6
    k_list = np.random.default_rng(3).choice(L.N_PARAMS, 40, replace=False)
    for k in k_list:
        e = np.zeros(L.N_PARAMS)
        e[k] = h
        g = (L.loss(params + e, x, y) - L.loss(params - e, x, y)) / (2 * h)
        if abs(g) > 1e-5:
            assert abs(q[k] - (params[k] - lr * np.sign(g))) < 1e-9, k
    assert abs(losses[0] - L.loss(params, x, y)) < 1e-12


def test_train_with_zero_rate_reports_the_drawn_minibatch_losses():
    params, x, y = random_problem(12, n=50)
    q, losses = L.train(params, x, y, steps=3, batch=6, lr=0.0, seed=2 ** 63 + 5)
    assert np.array_equal(q, params)
    # the step seeds wrap modulo 2^64; every loss is one of the per-sample means over 6 draws
    per = np.array([L.loss(params, x[i:i + 1], y[i:i + 1]) for i in range(50)])
    for t, Lt in enumerate(losses):
        idx = L.draw_indices(50, 6, (2 ** 63 + 5 + (t + 1) * 0x51ED2701) % 2 ** 64)
        assert abs(Lt - per[idx].mean()) < 1e-12
