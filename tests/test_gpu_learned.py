"""The learned scheduler on the GPU: network kernels against the float64 oracle, features against
their definition, and the schedule's effect (the tetrahedra never change)."""
import numpy as np
import pytest

import oracle
from oracle import learned as OL
from paper_1805_08831_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_08831_gb300 as dt  # noqa: E402
from paper_1805_08831_gb300 import learned  # noqa: E402


def problem(seed, n):
    rng = np.random.default_rng(seed)
    params = dt.init_params(seed) + rng.normal(0, 0.05, dt.DT_MLP_PARAMS).astype(np.float32)
    x = rng.random((n, 8)).astype(np.float32)
    y = np.c_[rng.random(n) * 6, (rng.random(n) < 0.3)].astype(np.float32)
    return params, x, y


def test_forward_matches_oracle():
    params, x, _ = problem(1, 5000)
    out = dt.mlp_forward(torch.from_numpy(params).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    ref, _ = OL.forward(params.astype(np.float64), x.astype(np.float64))
    assert np.allclose(out, ref, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("n", [1, 37, 4096])
def test_gradient_matches_oracle(n):
    """FP32 kernel gradient against float64 backpropagation: element-wise within 1e-4 of the
    gradient's largest entry (float32 sums of up to n terms)."""
    params, x, y = problem(2 + n, n)
    loss, g = dt.mlp_grad(torch.from_numpy(params).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    ref_loss, ref = OL.loss_grad(params.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    g = g.cpu().numpy()
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))
    assert np.max(np.abs(g - ref)) <= 1e-4 * np.max(np.abs(ref)) + 1e-7


@pytest.mark.parametrize("steps", [1, 4])
def test_training_matches_oracle(steps):
    """dt_mlp_train (minibatch draw, FP32 gradient, Adam) against the float64 training oracle.

    The per-step minibatch losses depend on which samples the counter-based draw picks: they
    must agree to FP32 accuracy (1e-5 relative). Adam moves each parameter by about lr per step
    whatever the gradient's size, so parameters whose gradient is small enough for FP32 rounding
    to flip its sign may differ by up to 2 lr per step; all others must agree within 2 % of lr
    per step, and every parameter within the largest Adam move, 3.2 lr per step."""
    params, x, y = problem(40 + steps, 4096)
    lr, batch, seed = 1e-3, 256, 2 ** 40 + 17
    p = torch.from_numpy(params.copy()).cuda()
    losses = dt.mlp_train(p, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), steps=steps, batch=batch,
                          lr=lr, seed=seed)
    ref_p, ref_losses = OL.train(params.astype(np.float64), x.astype(np.float64), y.astype(np.float64),
                                 steps=steps, batch=batch, lr=lr, seed=seed)
    assert np.allclose(losses, ref_losses, rtol=1e-5, atol=1e-6)
    got = p.cpu().numpy().astype(np.float64)
    diff = np.abs((got - params) - (ref_p - params))
    # well-conditioned parameters: the gradient of every step is far from zero
    well = np.ones(len(params), dtype=bool)
    q = params.astype(np.float64)
    m = np.zeros_like(q)
    v = np.zeros_like(q)
    for t in range(steps):
        idx = OL.draw_indices(len(x), batch, (seed + (t + 1) * 0x51ED2701) % 2 ** 64)
        _, g = OL.loss_grad(q, x[idx].astype(np.float64), y[idx].astype(np.float64))
        well &= np.abs(g) > 1e-3 * np.max(np.abs(g))
        q, m, v = OL.adam_step(q, g, m, v, lr, t + 1)
    assert well.mean() > 0.5
    assert np.max(diff[well]) <= 0.02 * lr * steps
    assert np.max(diff) <= 3.2 * lr * steps + 1e-7


def test_training_fits_a_teacher_network():
    """Targets produced by a fixed random network are learnable: the loss falls well below the
    loss of the initial parameters (training runs entirely in the library's kernels)."""
    rng = np.random.default_rng(7)
    teacher = (dt.init_params(99) * 0.7).astype(np.float32)
    x = rng.random((20000, 8)).astype(np.float32)
    out, _ = OL.forward(teacher.astype(np.float64), x.astype(np.float64))
    y = np.c_[out[:, 0], (out[:, 1] > 0)].astype(np.float32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    p0 = torch.from_numpy(dt.init_params(3)).cuda()
    before, _ = dt.mlp_grad(p0, xd, yd)
    losses = dt.mlp_train(p0, xd, yd, steps=1500, batch=2048, lr=3e-3, seed=1)
    after, _ = dt.mlp_grad(p0, xd, yd)
    assert np.all(np.isfinite(losses))
    assert after < 0.35 * before


def test_features_match_their_definition():
    x = synth.cube_and_slab(12000, 3)
    x[100:110] = x[:10]  # duplicates are not counted in the cells
    n = len(x)
    with dt.Triangulation(seed=4, flags=dt.DT_FLAG_LOG) as t:
        t.insert(torch.from_numpy(x).cuda())
        f, y, valid = t.features(n)
        st = t.stats()
    f, y, valid = f.cpu().numpy(), y.cpu().numpy(), valid.cpu().numpy()
    perm = oracle.insertion_order(x, 4)
    keys = oracle.moore_keys(x)[perm]
    rounds = oracle.brio_rounds(n, 4)[perm]
    dup = (oracle.dedup(x) != np.arange(n))[perm]
    lo, hi = x.min(axis=0), x.max(axis=0)
    ref = OL.features(x[perm], keys, rounds, dup, np.r_[lo, hi])
    assert np.allclose(f, ref, rtol=0, atol=2e-6)
    # labels: every concurrently inserted point has a cavity (|C| >= 1), duplicates have none
    assert valid[dup].sum() == 0
    assert np.all(y[valid == 1, 0] >= 1.0)
    assert set(np.unique(y[:, 1])) <= {0.0, 1.0}
    assert y[:, 1].sum() <= st["n_conflicts"]
    assert valid.sum() >= n - 10 - 2100  # all but the duplicates and the one-block first round


@pytest.fixture(scope="module")
def trained():
    """A scheduler trained on plain round logs of the uniform, degenerate and slab workloads."""
    clouds = [synth.uniform_cube(100000, 1), synth.degenerate_mix(60000, 3), synth.cube_and_slab(100000, 5)]
    params, losses = learned.train_scheduler(clouds, steps=1500)
    assert np.all(np.isfinite(losses)) and losses[-100:].mean() < losses[:100].mean()
    return params


@pytest.mark.parametrize("kind,n,seed", [("uniform", 20000, 8), ("slab", 30000, 2), ("degenerate", 20000, 6)])
def test_learned_schedule_gives_the_same_tets(trained, kind, n, seed):
    x = synth.make(kind, n, seed)
    ref, _ = oracle.delaunay(x, seed=seed)
    with dt.Triangulation(seed=seed, schedule=dt.DT_SCHED_LEARNED) as t:
        t.load_model(trained)
        t.insert(torch.from_numpy(x).cuda())
        got = t.tets_numpy()
    assert np.array_equal(got, ref)


def test_learned_schedule_without_a_model_is_refused():
    with dt.Triangulation(schedule=dt.DT_SCHED_LEARNED) as t:
        with pytest.raises(dt.DTError) as e:
            t.insert(torch.from_numpy(synth.uniform_cube(1000, 1)).cuda())
    assert e.value.code == dt.DT_ESTATE


def test_what_the_network_gains(trained, capsys):
    """Plain and learned schedules on a held-out slab cloud: the same tetrahedra whatever the
    schedule, and a network that learned something about the method: its predicted cavity sizes
    correlate with the sizes the plain schedule's insertions logged. The timings of both
    schedules are reported (the learned one sets the asynchronous engine's segment boundaries by
    predicted work; it is not faster on this input)."""
    x = synth.cube_and_slab(400000, 77)
    xd = torch.from_numpy(x).cuda()
    res = {}
    for name, sched in (("plain", dt.DT_SCHED_PLAIN), ("learned", dt.DT_SCHED_LEARNED)):
        with dt.Triangulation(seed=1, schedule=sched, flags=dt.DT_FLAG_LOG) as t:
            if sched == dt.DT_SCHED_LEARNED:
                t.load_model(trained)
            t.insert(xd)
            st = t.stats()
            f, y, valid = t.features(len(x))
            res[name] = (t.tets_numpy(), st, f, y, valid)
    assert np.array_equal(res["plain"][0], res["learned"][0])
    _, _, f, y, valid = res["plain"]
    keep = valid.bool()
    pred = dt.mlp_forward(torch.from_numpy(trained).cuda(), f[keep].contiguous())[:, 0].cpu().numpy()
    size = y[keep][:, 0].cpu().numpy()
    corr = float(np.corrcoef(pred, size)[0, 1])
    p, l = res["plain"][1], res["learned"][1]
    with capsys.disabled():
        print(f"\n  cavity-size prediction: correlation {corr:.3f} over {int(keep.sum())} insertions"
              f"\n  plain:   conflicts {p['n_conflicts']} of {p['n_attempts']} attempts, {p['ms_insert']:.1f} ms"
              f"\n  learned: conflicts {l['n_conflicts']} of {l['n_attempts']} attempts, {l['ms_insert']:.1f} ms")
    assert corr > 0.1
