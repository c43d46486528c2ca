"""Pins of the refinement oracle (oracle/refine.py) against what does not depend on it: closed
forms of circumcentres, the bisector equations, brute-force filters written out here, and the
properties the loop must leave behind (Section 4, Algorithm 2). The last test plants mistakes
in the oracle and checks that a pin catches each."""
import itertools

import numpy as np
import pytest

from oracle import refine as R
from paper_1805_08831_gb300 import synth

UNIT = [0.0, 0.0, 0.0, 1.0, 1.0, 1.0]


def centre_of(pts):
    P = np.asarray(pts, dtype=np.float64)
    C, r2, tup = R.circumcentres(P, np.array([[0, 1, 2, 3]]))
    return C[0], r2[0]


def test_corner_tetrahedron_closed_form():
    """(0, e1, e2, e3): centre (1/2, 1/2, 1/2), r^2 = 3/4, exactly; also scaled by 2^k and moved
    by a dyadic offset, where every operation stays exact."""
    c, r2 = centre_of([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    assert np.array_equal(c, [0.5, 0.5, 0.5]) and r2 == 0.75
    for k in (-6, 3):
        s = 2.0 ** k
        off = np.array([0.25, -1.5, 3.0])
        c, r2 = centre_of(off + s * np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]))
        assert np.array_equal(c, off + s * 0.5) and r2 == 0.75 * s * s


def test_regular_tetrahedron_closed_form():
    """Alternate cube corners: a regular tetrahedron with edge 2 sqrt 2, centre 0, R^2 = 3."""
    c, r2 = centre_of([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])
    assert np.array_equal(c, [0.0, 0.0, 0.0]) and r2 == 3.0


def test_centre_solves_the_bisector_equations():
    """2 (v_k - v_0) . c = |v_k|^2 - |v_0|^2 for k = 1..3, solved independently by LAPACK."""
    rng = np.random.default_rng(1)
    P = rng.random((400, 3))
    tets = np.array([rng.choice(400, 4, replace=False) for _ in range(300)])
    C, r2, tup = R.circumcentres(P, tets)
    for t in range(len(tets)):
        V = P[tets[t]]
        A = 2.0 * (V[1:] - V[0])
        if abs(np.linalg.det(A)) < 1e-3:
            continue
        x = np.linalg.solve(A, (V[1:] ** 2).sum(1) - (V[0] ** 2).sum())
        assert np.allclose(C[t], x, rtol=0, atol=1e-8 * max(1.0, np.abs(x).max()))
        d2 = ((V - x) ** 2).sum(1)
        assert np.allclose(r2[t], d2, rtol=1e-8)
        assert list(tup[t]) == sorted(tets[t])


def test_centre_does_not_depend_on_vertex_order():
    rng = np.random.default_rng(2)
    P = rng.random((50, 3))
    t = rng.choice(50, 4, replace=False)
    ref = R.circumcentres(P, t[None, :])
    for perm in itertools.permutations(range(4)):
        got = R.circumcentres(P, t[list(perm)][None, :])
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def brute_filter(C, r2, tup, thr):
    """Written out pair by pair: i survives unless some j with a larger r^2 (equal r^2: smaller
    index tuple) lies at squared distance below thr."""
    keep = []
    for i in range(len(C)):
        ok = True
        for j in range(len(C)):
            if j == i:
                continue
            d = C[i] - C[j]
            if (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] < thr:
                better = r2[j] > r2[i] or (r2[j] == r2[i] and list(tup[j]) < list(tup[i]))
                if better:
                    ok = False
        keep.append(ok)
    return np.array(keep)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_filter_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    m = 300
    C = rng.random((m, 3)) * 0.5
    C[: m // 5] = C[m // 5: 2 * (m // 5)]                 # exact duplicates
    r2 = np.round(rng.random(m), 2)                         # many equal radii
    tup = np.sort(rng.integers(0, 40, (m, 4)), axis=1)
    tup[:10] = tup[10:20]                                   # equal tuples too
    thr = 0.05 ** 2
    assert np.array_equal(R.filter_keep(C, r2, tup, thr), brute_filter(C, r2, tup, thr))


def test_far_from_points_equals_brute_force():
    rng = np.random.default_rng(3)
    P = rng.random((500, 3))
    C = np.r_[rng.random((200, 3)), P[:20] + 1e-3]
    thr = 0.04 ** 2
    want = np.array([min(((P - c) ** 2).sum(1)) >= thr for c in C])
    assert np.array_equal(R.far_from_points(C, P, thr), want)


def check_refined(P, tets, n0, counts, size, box, ratio=1.4, spacing=0.7):
    """The properties the loop leaves behind."""
    from scipy.spatial import cKDTree

    lo, hi = np.asarray(box[:3]), np.asarray(box[3:])
    added = P[n0:]
    assert len(added) == sum(counts) and len(counts) >= 1
    assert np.all((added > lo) & (added < hi))
    thr_d2 = (spacing * size) ** 2
    # every added point is at squared distance >= thr from every other point
    tree = cKDTree(P)
    for k, ids in enumerate(tree.query_ball_point(added, np.sqrt(thr_d2) * (1 + 1e-6))):
        others = [j for j in ids if j != n0 + k]
        if others:
            d = P[others] - added[k]
            assert np.all(((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]) >= thr_d2)
    # the loop stopped: every large tetrahedron's centre inside the box has a point next to it
    with np.errstate(divide="ignore", invalid="ignore"):
        C, r2, _ = R.circumcentres(P, tets)
    big = (r2 > (ratio * size) ** 2) & np.all((C > lo) & (C < hi), axis=1)
    if big.any():
        d, _ = tree.query(C[big])
        assert np.all(d < np.sqrt(thr_d2) * (1 + 1e-9))


@pytest.mark.parametrize("case", ["surface12", "cloud"])
def test_refine_leaves_a_spaced_terminated_mesh(case):
    if case == "surface12":
        X, size = synth.box_surface(12), 1.0 / 12
    else:
        corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float)
        X, size = np.r_[synth.uniform_cube(1500, 8), corners], 0.05
    P, tets, iters, counts = R.refine(X, size, UNIT)
    assert iters == len(counts) and iters < 20
    check_refined(P, tets, len(X), counts, size, UNIT)
    # each iteration's points are circumcentres of large tetrahedra of the previous mesh
    import oracle
    start = len(X)
    Q = X
    for c in counts:
        prev, _ = oracle.delaunay(Q)
        C, r2, _ = R.sample(Q, prev, UNIT, (1.4 * size) ** 2)
        new = P[start:start + c]
        as_rows = {tuple(x) for x in C}
        assert all(tuple(x) in as_rows for x in new)
        Q = P[:start + c]
        start += c


def test_refine_of_a_near_degenerate_surface_terminates():
    """24 intervals per edge produce co-circular near-flat tetrahedra whose rounded circumcentres
    fall next to existing vertices; the existing-point filter must stop them."""
    X = synth.box_surface(24)
    P, tets, iters, counts = R.refine(X, 1.0 / 24, UNIT, max_iters=30)
    assert iters < 30
    check_refined(P, tets, len(X), counts, 1.0 / 24, UNIT)


def run_pins():
    test_corner_tetrahedron_closed_form()
    test_regular_tetrahedron_closed_form()
    test_centre_solves_the_bisector_equations()
    for s in (0, 1, 2):
        test_filter_equals_brute_force(s)
    test_far_from_points_equals_brute_force()
    test_refine_of_a_near_degenerate_surface_terminates()


def _cross_sign_slip(p, q):
    return np.stack([p[..., 1] * q[..., 2] - p[..., 2] * q[..., 1],
                     p[..., 0] * q[..., 2] - p[..., 2] * q[..., 0],
                     p[..., 0] * q[..., 1] - p[..., 1] * q[..., 0]], axis=-1)


def _dot_dropped_term(p, q):
    return p[..., 0] * q[..., 0] + p[..., 1] * q[..., 1]


def _outranks_reversed(r2_j, tup_j, r2_i, tup_i):
    return (r2_j < r2_i) | ((r2_j == r2_i) & R.tuple_less(tup_j, tup_i))


def _no_point_filter(C, P, thr_d2):
    return np.ones(len(C), dtype=bool)


@pytest.mark.parametrize("name,repl", [("_cross", _cross_sign_slip), ("_dot", _dot_dropped_term),
                                       ("outranks", _outranks_reversed),
                                       ("far_from_points", _no_point_filter)])
def test_planted_mistakes_are_caught(name, repl, monkeypatch):
    monkeypatch.setattr(R, name, repl)
    with pytest.raises(AssertionError):
        run_pins()
