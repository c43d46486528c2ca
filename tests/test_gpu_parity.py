"""GPU path vs the CPU oracle, through the C ABI (bit-exact: integer and index results)."""
import numpy as np
import pytest

import oracle
from paper_1805_08831_gb300 import synth
from tests.inputs import DEGENERATE_SETS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_08831_gb300 as dt  # noqa: E402


def gpu_tets(x, seed=0, **kw):
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    with dt.Triangulation(seed=seed, **kw) as t:
        t.insert(xt)
        tets = t.tets_numpy(canonical=True)
        st = t.stats()
    return tets, st


def assert_same(a, b):
    assert a.shape == b.shape, (a.shape, b.shape)
    if not np.array_equal(a, b):
        bad = np.nonzero((a != b).any(axis=1))[0]
        raise AssertionError(f"{len(bad)} rows differ; first at {bad[:5]}: {a[bad[:3]]} vs {b[bad[:3]]}")


# ----------------------------------------------------------------------------- predicates
def _tuples(rng, n):
    p = rng.random((n, 5, 3))
    kind = rng.integers(0, 4, n)
    for i in np.nonzero(kind == 1)[0]:  # box corners: exactly co-spherical
        lo, hi = rng.random(3), rng.random(3) + 1.0
        c = np.array([[hi[0] if j & 1 else lo[0], hi[1] if j & 2 else lo[1], hi[2] if j & 4 else lo[2]]
                      for j in range(8)])
        p[i] = c[rng.permutation(8)[:5]]
    for i in np.nonzero(kind == 2)[0]:  # four points on an axis plane
        p[i, :4, 2] = p[i, 0, 2]
    for i in np.nonzero(kind == 3)[0]:  # one-ulp nudge of a co-spherical set
        lo, hi = rng.random(3), rng.random(3) + 1.0
        c = np.array([[hi[0] if j & 1 else lo[0], hi[1] if j & 2 else lo[1], hi[2] if j & 4 else lo[2]]
                      for j in range(8)])
        p[i] = c[rng.permutation(8)[:5]]
        p[i, 4, 0] = np.nextafter(p[i, 4, 0], 10.0)
    return p


def test_device_predicates_match_oracle():
    rng = np.random.default_rng(3)
    n = 4000
    p = _tuples(rng, n)
    ids = np.stack([rng.permutation(100)[:5] for _ in range(n)]).astype(np.int64)
    pt = torch.from_numpy(p).cuda()
    it = torch.from_numpy(ids).cuda()
    o = dt.eval_predicates(0, pt).cpu().numpy()
    s = dt.eval_predicates(1, pt).cpu().numpy()
    q = dt.eval_predicates(2, pt, it).cpu().numpy()
    o32 = dt.eval_predicates(3, pt).cpu().numpy()
    q32 = dt.eval_predicates(4, pt, it).cpu().numpy()
    for i in range(n):
        ref_o = oracle.orient3d(*p[i, :4])
        assert o[i] == ref_o and o32[i] == ref_o, i
        assert s[i] == oracle.insphere(*p[i]), i
        if ref_o > 0:
            ref_q = oracle.insphere_sos(p[i], ids[i])
            assert q[i] == ref_q and q32[i] == ref_q, i


def test_exact_stages_on_lattice_tuples():
    """Lattice coordinates (i / 99, scaled by powers of two, negated, shifted) are exactly
    co-spherical and coplanar in many tuples: the integer exact stage decides them, and tuples
    whose exponents spread too far take the expansion arithmetic; both against the oracle."""
    rng = np.random.default_rng(23)
    n = 6000
    p = rng.integers(0, 5, (n, 5, 3)).astype(np.float64) / 99.0
    scale = 2.0 ** rng.integers(-30, 30, n)
    p *= scale[:, None, None]
    flip = rng.random(n) < 0.3
    p[flip] *= -1.0
    shift = rng.random(n) < 0.2
    p[shift] += rng.integers(-3, 3, (shift.sum(), 1, 3)) * scale[shift][:, None, None]
    far = rng.random(n) < 0.1  # one coordinate 2^40 times larger: the integer stage declines
    p[far, 0, 0] += 2.0 ** 40 * scale[far]
    ids = np.stack([rng.permutation(100)[:5] for _ in range(n)]).astype(np.int64)
    pt = torch.from_numpy(p).cuda()
    o = dt.eval_predicates(0, pt).cpu().numpy()
    s = dt.eval_predicates(1, pt).cpu().numpy()
    q = dt.eval_predicates(2, pt, torch.from_numpy(ids).cuda()).cpu().numpy()
    zeros = 0
    for i in range(n):
        ref_o = oracle.orient3d(*p[i, :4])
        ref_s = oracle.insphere(*p[i])
        zeros += ref_s == 0
        assert o[i] == ref_o, i
        assert s[i] == ref_s, i
        if ref_o > 0:
            assert q[i] == oracle.insphere_sos(p[i], ids[i]), i
    assert zeros > n // 20  # many tuples are exactly co-spherical


def test_fp32_stage_on_nearly_cospherical_tuples():
    """Points a few ulps off a common sphere, at several scales and offsets: the FP32 stage
    must either be right or defer, never return a wrong sign."""
    rng = np.random.default_rng(17)
    n = 20000
    p = np.empty((n, 5, 3))
    for i in range(n):
        scale = 10.0 ** rng.uniform(-6, 0)
        off = rng.uniform(-1e3, 1e3, 3) * (rng.random() < 0.3)
        d = rng.normal(size=(5, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        p[i] = off + scale * d
        k = rng.integers(0, 15)
        p[i].flat[k] = np.nextafter(p[i].flat[k], np.inf if rng.random() < 0.5 else -np.inf)
    ids = np.stack([rng.permutation(100)[:5] for _ in range(n)]).astype(np.int64)
    pt = torch.from_numpy(p).cuda()
    o32 = dt.eval_predicates(3, pt).cpu().numpy()
    q32 = dt.eval_predicates(4, pt, torch.from_numpy(ids).cuda()).cpu().numpy()
    for i in range(n):
        ref_o = oracle.orient3d(*p[i, :4])
        assert o32[i] == ref_o, i
        if ref_o > 0:
            assert q32[i] == oracle.insphere_sos(p[i], ids[i]), i


# ----------------------------------------------------------------------------- order
@pytest.mark.parametrize("n", [1, 5, 2047, 2049, 14337, 100000])
def test_moore_keys_and_insertion_order(n):
    x = synth.uniform_cube(n, 21)
    x[n // 2:n // 2 + min(5, n // 4)] = x[:min(5, n // 4)]  # duplicates share a key
    xt = torch.from_numpy(x).cuda()
    with dt.Triangulation(seed=99) as t:
        try:
            t.insert(xt)
        except dt.DTError as e:
            assert e.code == dt.DT_EDEGENERATE and n < 4
            return
        keys, perm, rounds = t.order(n)
    assert np.array_equal(keys, oracle.moore_keys(x))
    assert np.array_equal(rounds, oracle.brio_rounds(n, 99))
    assert np.array_equal(perm, oracle.insertion_order(x, 99))


# ----------------------------------------------------------------------------- triangulations
@pytest.mark.parametrize("name", sorted(DEGENERATE_SETS))
def test_degenerate_sets(name):
    x = DEGENERATE_SETS[name]
    ref, _ = oracle.delaunay(x)
    got, _ = gpu_tets(x)
    assert_same(got, ref)


@pytest.mark.parametrize("n", [4, 5, 7, 30, 200, 2047, 2049, 20000])
def test_uniform_small_and_ragged(n):
    x = synth.uniform_cube(n, 1000 + n)
    ref, _ = oracle.delaunay(x, seed=5)
    got, _ = gpu_tets(x, seed=5)
    assert_same(got, ref)


def test_uniform_1e5_bit_exact():
    x = synth.uniform_cube(100000, 1)
    ref, _ = oracle.delaunay(x, seed=1)
    got, st = gpu_tets(x, seed=1)
    assert_same(got, ref)
    assert st["n_unique"] == 100000 and st["n_exact"] == 0


def test_degenerate_mix_bit_exact():
    x = synth.degenerate_mix(30000, 3)
    x[-3000:] = x[-6000:-3000]  # repeated lattice sites
    ref, ost = oracle.delaunay(x, seed=3)
    got, st = gpu_tets(x, seed=3)
    assert_same(got, ref)
    assert st["n_unique"] == ost["n_unique"]


def test_slab_bit_exact():
    x = synth.cube_and_slab(30000, 5)
    ref, _ = oracle.delaunay(x, seed=2)
    got, _ = gpu_tets(x, seed=2)
    assert_same(got, ref)


def test_schedule_does_not_change_tets():
    x = synth.uniform_cube(20000, 8)
    ref, _ = oracle.delaunay(x, seed=1)
    for seg in (1, 7, 64, 4096):
        got, _ = gpu_tets(x, seed=1, segments=seg)
        assert_same(got, ref)
    got, _ = gpu_tets(x, seed=12345)
    assert_same(got, ref)


@pytest.mark.parametrize("kind,n,seed", [("uniform", 20000, 8), ("degenerate", 30000, 3), ("slab", 30000, 5),
                                         ("uniform", 5, 1)])
def test_certificate_holds_where_the_oracle_agrees(kind, n, seed):
    """dt_check on meshes equal to the oracle's: every adjacency reciprocal, every finite
    tetrahedron positively oriented, every facet locally Delaunay under the perturbed predicates,
    and its counts equal to the oracle's (tetrahedra, distinct vertices)."""
    x = synth.make(kind, n, seed)
    ref, ost = oracle.delaunay(x, seed=seed)
    with dt.Triangulation(seed=seed) as t:
        t.insert(torch.from_numpy(x).cuda())
        cert = t.check()
        got = t.tets_numpy(canonical=True)
        st = t.stats()
    assert_same(got, ref)
    assert cert == {"tets": len(ref), "bad_adjacency": 0, "bad_orientation": 0, "not_delaunay": 0,
                    "vertices": ost["n_unique"]}
    assert st["n_unique"] == ost["n_unique"]


def test_certificate_states():
    """dt_check on a handle without a mesh counts nothing, and after a batch (whose clouds are
    separate meshes) it is refused."""
    with dt.Triangulation() as t:
        assert t.check() == {"tets": 0, "bad_adjacency": 0, "bad_orientation": 0, "not_delaunay": 0,
                             "vertices": 0}
        xyz, off = synth.batched_clouds(3, 9, lo=50, hi=200)
        t.batch(torch.from_numpy(xyz).cuda(), off)
        with pytest.raises(dt.DTError) as e:
            t.check()
        assert e.value.code == dt.DT_ESTATE


@pytest.mark.parametrize("name", sorted(DEGENERATE_SETS))
def test_certificate_on_degenerate_sets(name):
    x = DEGENERATE_SETS[name]
    ref, ost = oracle.delaunay(x)
    with dt.Triangulation() as t:
        t.insert(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda())
        before = t.stats()
        cert = t.check()
        after = t.stats()
    assert cert["bad_adjacency"] == cert["bad_orientation"] == cert["not_delaunay"] == 0
    assert cert["tets"] == len(ref) and cert["vertices"] == ost["n_unique"]
    before.pop("n_launches"), after.pop("n_launches")  # the check's own two launches count
    assert before == after  # the check leaves the handle's statistics alone


def test_successive_inserts_extend_the_triangulation():
    x = synth.uniform_cube(12000, 17)
    x[11000:11010] = x[100:110]  # duplicates across calls keep the earlier (smaller) index
    ref, _ = oracle.delaunay(x, seed=4)
    with dt.Triangulation(seed=4) as t:
        t.insert(torch.from_numpy(x[:5000]).cuda())
        t.insert(torch.from_numpy(x[5000:]).cuda())
        got = t.tets_numpy()
        st = t.stats()
    assert_same(got, ref)
    assert st["n_points"] == 12000 and st["n_unique"] == 11990


def test_host_entry_points_match_device_ones():
    x = synth.uniform_cube(5000, 6)
    ref, _ = oracle.delaunay(x)
    with dt.Triangulation() as t:
        t.insert_host(x)
        assert_same(t.tets_host(), ref)
        # the handle keeps its device buffers between calls: a second, smaller insert reuses them
        t.clear()
        t.insert_host(x[:3000])
        ref2, _ = oracle.delaunay(x[:3000])
        assert_same(t.tets_host(), ref2)
        # a caller's buffer: filled when large enough, replaced when too small
        big = np.full((len(ref2) + 10, 4), 7, dtype=np.uint32)
        got = t.tets_host(out=big)
        assert got.base is big or got is big or np.shares_memory(got, big)
        assert_same(got, ref2)
        small = np.zeros((5, 4), dtype=np.uint32)
        assert_same(t.tets_host(out=small), ref2)
        # unsorted output holds the same set, into pageable memory (a copy) or page-locked
        # memory (written by the kernel through its mapped address)
        raw = t.tets_host(canonical=False)
        pinned = torch.zeros((len(ref2) + 3, 4), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        raw_pinned = t.tets_host(canonical=False, out=pinned)
        for r in (raw, raw_pinned):
            assert len(r) == len(ref2)
            rot = np.sort(r, axis=1)
            assert_same(rot[np.lexsort(rot.T[::-1])], (lambda q: q[np.lexsort(q.T[::-1])])(np.sort(ref2, axis=1)))
        assert not pinned[len(ref2):].any()  # nothing written past the count


def test_errors_are_reported_not_raised_on_device():
    plane = np.c_[synth.uniform_cube(100, 1)[:, :2], np.zeros(100)]
    with pytest.raises(dt.DTError) as e:
        gpu_tets(plane)
    assert e.value.code == dt.DT_EDEGENERATE
    bad = synth.uniform_cube(100, 1)
    bad[7, 2] = np.inf
    with pytest.raises(dt.DTError) as e:
        gpu_tets(bad)
    assert e.value.code == dt.DT_EINVAL


# ----------------------------------------------------------------------------- both engines
@pytest.mark.parametrize("engine", ["async", "rounds", "async_subdet"])
@pytest.mark.parametrize("kind,n,seed", [("uniform", 60000, 21), ("degenerate", 30000, 22), ("slab", 40000, 23)])
def test_each_engine_alone_is_bit_exact(monkeypatch, engine, kind, n, seed):
    """The asynchronous engine (per-warp segments under ownership words) and the round-based one
    (claim words, three kernels a round) each give the oracle's tetrahedra on their own: DT_ASYNC=0
    keeps every pass on the rounds; DT_ASYNC_MIN_RETRY=1 sends even short retry lists to the
    asynchronous engine. DT_SUBDET=1 runs the asynchronous engine's conflict tests through the
    sub-determinant cache (the ablation of Section 2.4)."""
    if engine == "rounds":
        monkeypatch.setenv("DT_ASYNC", "0")
    else:
        monkeypatch.setenv("DT_ASYNC_MIN_RETRY", "1")
    if engine == "async_subdet":
        monkeypatch.setenv("DT_SUBDET", "1")
    x = synth.make(kind, n, seed)
    ref, _ = oracle.delaunay(x, seed=seed)
    got, st = gpu_tets(x, seed=seed)
    assert_same(got, ref)
    if engine == "rounds":
        assert st["n_async"] == 0
    else:
        assert st["n_inserted_async"] > 0
