"""dt_batch: many independent clouds in one persistent launch, every cloud bit-exact against the
oracle run on that cloud alone (the perturbed Delaunay triangulation is unique, so batching,
block shape and round size cannot change it)."""
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


def run_batch(clouds, seed=0):
    off = np.zeros(len(clouds) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(c) for c in clouds])
    xyz = np.ascontiguousarray(np.concatenate(clouds, axis=0), dtype=np.float64)
    with dt.Triangulation(seed=seed) as t:
        t.batch(torch.from_numpy(xyz).cuda(), off)
        tets, coff = t.tets_batch(canonical=True)
        st = t.stats()
    return [tets[int(coff[c]):int(coff[c + 1])] for c in range(len(clouds))], st


def split(xyz, off):
    return [xyz[int(off[c]):int(off[c + 1])] for c in range(len(off) - 1)]


def assert_clouds_match(clouds, got):
    for c, x in enumerate(clouds):
        ref, _ = oracle.delaunay(x)
        if not np.array_equal(got[c], ref):
            raise AssertionError(f"cloud {c} ({len(x)} points): {len(got[c])} vs {len(ref)} tetrahedra")


def test_batch_of_uneven_uniform_clouds_matches_oracle():
    xyz, off = synth.batched_clouds(48, 11, lo=50, hi=6000)
    clouds = split(xyz, off)
    got, st = run_batch(clouds)
    assert_clouds_match(clouds, got)
    assert st["n_clouds_degenerate"] == 0
    assert st["batch_warps"] in (4, 8, 16, 32)
    assert st["n_unique"] == len(xyz)


def test_batch_clouds_spanning_several_brio_rounds():
    # 2048 / 14336 / 100352 are the first BRIO round ends: these clouds use three rounds
    clouds = [synth.uniform_cube(n, 300 + n) for n in (2047, 2049, 14337, 30000)]
    got, _ = run_batch(clouds, seed=5)
    assert_clouds_match(clouds, got)


def test_batch_of_degenerate_clouds_and_duplicates():
    clouds = [DEGENERATE_SETS[k] for k in sorted(DEGENERATE_SETS)]
    mix = synth.degenerate_mix(6000, 7)
    mix[-500:] = mix[:500]  # duplicates inside the cloud
    clouds.append(mix)
    clouds.append(synth.cube_and_slab(5000, 9))
    got, st = run_batch(clouds)
    assert_clouds_match(clouds, got)
    assert st["n_exact"] > 0 and st["n_sos"] > 0


def test_batch_cloud_without_volume_is_skipped_not_fatal():
    plane = np.c_[synth.uniform_cube(200, 1)[:, :2], np.zeros(200)]
    clouds = [synth.uniform_cube(300, 2), plane, synth.uniform_cube(4, 3), synth.uniform_cube(5, 4)]
    got, st = run_batch(clouds)
    assert st["n_clouds_degenerate"] == 1
    assert len(got[1]) == 0
    for c in (0, 2, 3):
        ref, _ = oracle.delaunay(clouds[c])
        assert np.array_equal(got[c], ref)


def test_batch_equals_single_cloud_inserts():
    xyz, off = synth.batched_clouds(6, 21, lo=500, hi=20000)
    clouds = split(xyz, off)
    got, _ = run_batch(clouds, seed=3)
    for c, x in enumerate(clouds):
        with dt.Triangulation(seed=3) as t:
            t.insert(torch.from_numpy(np.ascontiguousarray(x)).cuda())
            single = t.tets_numpy()
        assert np.array_equal(got[c], single)


def test_batch_output_into_page_locked_host_memory():
    """Unsorted rows written by the collection kernel straight into page-locked host memory hold
    each cloud's tetrahedra (the sorted device output, as sets); pageable memory is refused by
    the C ABI and the binding falls back to its own array."""
    xyz, off = synth.batched_clouds(12, 41, lo=50, hi=6000)
    with dt.Triangulation(seed=3) as t:
        t.batch(torch.from_numpy(xyz).cuda(), off)
        ref, roff = t.tets_batch(canonical=True)
        pinned = torch.zeros((len(ref) + 7, 4), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        got, goff = t.tets_batch(canonical=False, out=pinned)
        assert np.shares_memory(got, pinned) and np.array_equal(goff, roff)
        assert not pinned[len(ref):].any()
        pageable, poff = t.tets_batch(canonical=False, out=np.zeros((len(ref), 4), dtype=np.uint32))
        assert np.array_equal(poff, roff)
    for res in (got, pageable):
        for c in range(len(roff) - 1):
            a = np.sort(res[int(roff[c]):int(roff[c + 1])], axis=1)
            b = np.sort(ref[int(roff[c]):int(roff[c + 1])], axis=1)
            assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])


@pytest.mark.parametrize("warps", [8, 16, 32])
def test_every_block_shape_gives_the_same_tets(warps, monkeypatch):
    monkeypatch.setenv("DT_BATCH_WARPS", str(warps))
    monkeypatch.setenv("DT_BATCH_ALPHA", "0.3")
    xyz, off = synth.batched_clouds(20, 31, lo=50, hi=4000)
    clouds = split(xyz, off)
    got, st = run_batch(clouds)
    assert st["batch_warps"] == warps
    assert_clouds_match(clouds, got)


def test_batch_at_scale_sampled_clouds():
    """4096 clouds, sizes log-uniform in [50, 50000]: every cloud's tetrahedron count and a
    sample of clouds checked element by element against the oracle."""
    xyz, off = synth.batched_clouds(4096, 4)
    with dt.Triangulation(seed=0) as t:
        t.batch(torch.from_numpy(xyz).cuda(), off)
        tets, coff = t.tets_batch(canonical=True)
        st = t.stats()
    assert st["n_clouds_degenerate"] == 0 and st["device_error"] == 0
    assert st["n_unique"] == len(xyz)
    # between n and 7 n tetrahedra per cloud (about 6.7 n for large uniform clouds)
    counts = np.diff(coff.astype(np.int64))
    sizes = np.diff(off.astype(np.int64))
    assert np.all(counts > sizes) and np.all(counts < 7 * sizes)
    rng = np.random.default_rng(0)
    for c in rng.choice(4096, 12, replace=False):
        x = xyz[int(off[c]):int(off[c + 1])]
        ref, _ = oracle.delaunay(x)
        assert np.array_equal(tets[int(coff[c]):int(coff[c + 1])], ref), c


def test_repeated_batch_replays_its_graph_on_new_data():
    """The second call with the same buffer and cloud sizes replays the captured CUDA graph; the
    graph computes everything that depends on the coordinates on the device, so new values in
    the same buffer give their own triangulations."""
    xyz, off = synth.batched_clouds(30, 41, lo=50, hi=3000)
    xd = torch.from_numpy(xyz).cuda()
    with dt.Triangulation(seed=0) as t:
        t.batch(xd, off)
        first, c1 = t.tets_batch()
        t.clear()
        t.batch(xd, off)
        again, c2 = t.tets_batch()
        st = t.stats()
        assert st["batch_graph"] == 1
        assert np.array_equal(first, again) and np.array_equal(c1, c2)
        xyz2 = synth.uniform(99, 3 * len(xyz)).reshape(-1, 3)  # same cloud sizes, new coordinates
        xd.copy_(torch.from_numpy(xyz2 * 3.0 - 1.0))
        t.clear()
        t.batch(xd, off)
        new, c3 = t.tets_batch()
        assert t.stats()["batch_graph"] == 1
    clouds = split(xyz2 * 3.0 - 1.0, off)
    assert_clouds_match(clouds, [new[int(c3[c]):int(c3[c + 1])] for c in range(30)])
