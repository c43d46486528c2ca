"""dt_refine (Section 4, Algorithm 2 loop on a box) against the refinement oracle: the points it
adds (coordinates and input indices, bit for bit), the iterations, and the tetrahedra of the
refined mesh (bit for bit), on box surfaces, a cloud with its box corners and a surface whose
near-flat tetrahedra have rounding-dominated circumcentres; then the loop's properties at a size
the oracle does not repeat."""
import numpy as np
import pytest

import oracle
from oracle import refine as R
from paper_1805_08831_gb300 import synth
from tests.test_oracle_refine import check_refined

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_08831_gb300 as dt  # noqa: E402

UNIT = (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
CORNERS = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=np.float64)


def gpu_refine(X, size, box=UNIT, max_iters=100, seed=0, **kw):
    with dt.Triangulation(seed=seed) as t:
        t.insert(torch.from_numpy(np.ascontiguousarray(X)).cuda())
        added, iters = t.refine(size, box, max_iters=max_iters, **kw)
        P = t.points().cpu().numpy()
        tets = t.tets_numpy()
        st = t.stats()
    assert st["device_error"] == 0
    return P, tets, added, iters


def assert_matches_oracle(X, size, box=UNIT, max_iters=100, **kw):
    P, tets, added, iters = gpu_refine(X, size, box, max_iters, **kw)
    Pr, tr, ir, counts = R.refine(X, size, box, max_iters=max_iters, **kw)
    assert iters == ir and added == sum(counts)
    assert P.shape == Pr.shape
    assert np.array_equal(P, Pr)                  # every added point, bit for bit, in order
    assert np.array_equal(tets, tr)               # the refined mesh
    return P, tets, counts


@pytest.mark.parametrize("k", [4, 8, 12])
def test_refine_box_surface_matches_oracle(k):
    X = synth.box_surface(k)
    P, tets, counts = assert_matches_oracle(X, 1.0 / k)
    check_refined(P, tets, len(X), counts, 1.0 / k, UNIT)


@pytest.mark.parametrize("rebuild", ["0", "0.25", "0.000001"])
def test_refine_rebuilds_give_the_incremental_mesh(monkeypatch, rebuild):
    """An iteration that adds many points may rebuild the mesh from all its points instead of
    inserting into it (DT_REFINE_REBUILD: never, at a quarter of the mesh's points, at every
    iteration); the triangulation is unique, so the points and the mesh equal the oracle's."""
    monkeypatch.setenv("DT_REFINE_REBUILD", rebuild)
    X = synth.box_surface(10)
    assert_matches_oracle(X, 1.0 / 10)


def test_refine_cloud_with_corners_matches_oracle():
    X = np.r_[synth.uniform_cube(1500, 8), CORNERS]
    P, tets, counts = assert_matches_oracle(X, 0.05)
    check_refined(P, tets, len(X), counts, 0.05, UNIT)


def test_refine_near_flat_surface_matches_oracle():
    """24 intervals per edge: near-flat co-circular tetrahedra whose rounded circumcentres land on
    existing vertices; the existing-point filter must drop them on both sides alike."""
    X = synth.box_surface(24)
    P, tets, counts = assert_matches_oracle(X, 1.0 / 24)
    check_refined(P, tets, len(X), counts, 1.0 / 24, UNIT)


def test_refine_other_thresholds_and_a_smaller_box():
    X = np.r_[synth.uniform_cube(800, 9) * 2.0 - 0.5, CORNERS * 2.0 - 0.5]
    assert_matches_oracle(X, 0.08, box=(-0.5, -0.5, -0.5, 1.5, 1.5, 1.5), ratio=1.2, spacing=0.6)
    # a box inside the hull: only centres inside it are candidates
    assert_matches_oracle(X, 0.1, box=(0.0, 0.0, 0.0, 1.0, 1.0, 1.0))


def test_refine_stops_after_max_iters():
    X = synth.box_surface(16)
    P1, t1, added, iters = gpu_refine(X, 1.0 / 16, max_iters=1)
    Pr, tr, ir, counts = R.refine(X, 1.0 / 16, UNIT, max_iters=1)
    assert iters == 1 == ir and np.array_equal(P1, Pr) and np.array_equal(t1, tr)
    # a second call carries on from there and ends where one call would
    with dt.Triangulation(seed=0) as t:
        t.insert(torch.from_numpy(X).cuda())
        t.refine(1.0 / 16, max_iters=1)
        t.refine(1.0 / 16)
        both = t.points().cpu().numpy()
    full, _, _, _ = R.refine(X, 1.0 / 16, UNIT)
    assert np.array_equal(both, full)


def test_refine_with_nothing_to_do():
    X = synth.box_surface(6)
    P, tets, added, iters = gpu_refine(X, 10.0)           # every tetrahedron is small
    assert added == 0 and iters == 0 and np.array_equal(P, X)
    assert np.array_equal(tets, oracle.delaunay(X)[0])


def test_refine_errors():
    X = synth.box_surface(4)
    with dt.Triangulation() as t:
        with pytest.raises(dt.DTError) as e:
            t.refine(0.1)                                   # no triangulation yet
        assert e.value.code == dt.DT_ESTATE
        t.insert(torch.from_numpy(X).cuda())
        for bad in [dict(size=0.0), dict(size=-1.0), dict(size=float("nan")), dict(size=0.1, ratio=0.0),
                    dict(size=0.1, spacing=-1.0), dict(size=0.1, box=(0, 0, 0, 1, 0, 1)),
                    dict(size=0.1, box=(0, 0, 0, 1, 1, float("inf"))), dict(size=1e-9)]:
            with pytest.raises(dt.DTError) as e:
                t.refine(**bad)
            assert e.value.code == dt.DT_EINVAL, bad
        assert t.points().shape == (len(X), 3)              # nothing was added


def test_points_returns_the_inputs_by_index():
    X = synth.uniform_cube(5000, 3)
    X[-100:] = X[3000:3100]                                 # duplicates (within one call) keep their rows
    with dt.Triangulation() as t:
        t.insert(torch.from_numpy(X[:3000]).cuda())
        t.insert(torch.from_numpy(X[3000:]).cuda())
        assert np.array_equal(t.points().cpu().numpy(), X)


def test_refine_at_scale_properties():
    """A 64-interval box surface refined to about 1.2e5 points (6.5e5 tetrahedra): the oracle's
    triangulation of the final points equals the GPU's mesh, and the loop's properties hold."""
    X = synth.box_surface(64)
    P, tets, added, iters = gpu_refine(X, 1.0 / 64)
    assert added > 50000 and iters < 20
    ref, _ = oracle.delaunay(P)
    assert np.array_equal(tets, ref)
    lo, hi = np.zeros(3), np.ones(3)
    new = P[len(X):]
    assert np.all((new > lo) & (new < hi))
    # spacing and termination, as the oracle's loop leaves them
    check_refined(P, tets, len(X), [added], 1.0 / 64, UNIT)
