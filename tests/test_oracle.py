"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* rational arithmetic on the definitions of the predicates (the 4x4 [p, 1] and 5x5 lifted
  determinants of Section 2.4, evaluated by sympy on exact rationals);
* the worked example of the inSphere expansion (Section 2.4), Fig. 2's adjacency encoding and
  Table 2's BRIO round sizes (fixtures under tests/golden/);
* the limit definition of the lifting perturbation, evaluated with an explicit tiny rational
  perturbation;
* Qhull (scipy.spatial.Delaunay) on points in general position;
* brute-force enumeration of all 4-subsets (the definition of DT, Section 2);
* invariants of any triangulation of the hull: Euler's relation, total volume = hull volume,
  hull facets = 2 * hull vertices - 4, order independence of the perturbed DT;
* Moore-curve properties (bijection, face adjacency of consecutive cells, closedness).
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1805_08831_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- helpers
def frac_det(m):
    """Exact determinant of a square matrix of Fractions (sympy's rational det)."""
    sympy = pytest.importorskip("sympy")
    d = sympy.Matrix([[sympy.Rational(x.numerator, x.denominator) for x in row] for row in m]).det()
    d = sympy.Rational(d)
    return Fraction(int(d.p), int(d.q))


def F(x):
    return Fraction(float(x))


def orient_def(a, b, c, d):
    """Sign convention of the oracle: det[b-a; c-a; d-a] = -det[[p, 1]] (4x4, rows a,b,c,d)."""
    m = [[F(p[0]), F(p[1]), F(p[2]), Fraction(1)] for p in (a, b, c, d)]
    v = -frac_det(m)
    return (v > 0) - (v < 0)


def insphere_def(a, b, c, d, e, eps=None):
    """5x5 lifted determinant with rows (x, y, z, |p|^2 + eps_p, 1); equal to the 4x4 form."""
    rows = []
    for i, p in enumerate((a, b, c, d, e)):
        fp = [F(v) for v in p]
        lift = fp[0] * fp[0] + fp[1] * fp[1] + fp[2] * fp[2]
        if eps is not None:
            lift += eps[i]
        rows.append(fp + [lift, Fraction(1)])
    v = frac_det(rows)
    return (v > 0) - (v < 0)


def canon(t):
    """Even-permutation canonical form of a positive tuple (written independently of C++)."""
    t = list(t)
    k = t.index(min(t))
    perm = {0: (0, 1, 2, 3), 1: (1, 0, 3, 2), 2: (2, 0, 1, 3), 3: (3, 0, 2, 1)}[k]
    r = [t[i] for i in perm]
    rest = r[1:]
    j = rest.index(min(rest))
    return tuple([r[0]] + rest[j:] + rest[:j])


def canon_list(tets, xyz):
    out = []
    for s in tets:
        s = [int(v) for v in s]
        if oracle.orient3d(*[xyz[v] for v in s]) < 0:
            s[2], s[3] = s[3], s[2]
        out.append(canon(s))
    return np.array(sorted(out), dtype=np.uint32).reshape(-1, 4)


def euler_ok(tets):
    V = set()
    E = set()
    Fc = set()
    for t in tets:
        t = sorted(int(v) for v in t)
        V.update(t)
        E.update(itertools.combinations(t, 2))
        Fc.update(itertools.combinations(t, 3))
    return len(V) - len(E) + len(Fc) - len(tets) == 1


def exact_volume6(tets, xyz):
    total = Fraction(0)
    for t in tets:
        a, b, c, d = [[F(v) for v in xyz[i]] for i in t]
        u = [b[k] - a[k] for k in range(3)]
        v = [c[k] - a[k] for k in range(3)]
        w = [d[k] - a[k] for k in range(3)]
        total += (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
                  + u[2] * (v[0] * w[1] - v[1] * w[0]))
    return total


def lattice(k):
    return np.array(list(itertools.product(range(k), repeat=3)), dtype=np.float64)


def sphere9():
    return np.array([p for p in itertools.product(range(-3, 4), repeat=3)
                     if sum(v * v for v in p) == 9], dtype=np.float64)


def cube_centre():
    return np.array(list(itertools.product((0.0, 1.0), repeat=3)) + [[0.5, 0.5, 0.5]])


DEGENERATE_SETS = {
    "lattice3": lattice(3),
    "sphere9": sphere9(),
    "cube_centre": cube_centre(),
    "two_planes": np.array([[x, y, z] for z in (0.0, 1.0) for x in range(3) for y in range(3)]
                           + [[0.5, 0.5, 0.5], [1.5, 0.7, 0.3]], dtype=np.float64),
    "lattice_dups": np.concatenate([lattice(2), lattice(2)[::-1], [[0.5, 0.5, 0.5]]]),
}


# ----------------------------------------------------------------------------- predicates
def test_insphere_worked_example():
    g = golden("insphere_worked.json")
    pts = [g[k] for k in "abcde"]
    assert oracle.orient3d_value(*pts[:4]) == g["orient3d_abcd"]
    assert oracle.insphere_value(*pts) == g["insphere_abcde"]
    assert oracle.insphere(*pts) == -1          # inside a positive tetrahedron => negative
    assert oracle.insphere(*pts[:4], [2.0, 2.0, 2.0]) == 1


def _random_tuples(rng, count):
    """Random, 1-ulp-perturbed and exactly degenerate 5-point tuples."""
    out = []
    for _ in range(count):
        kind = rng.integers(4)
        p = rng.random((5, 3))
        if kind == 1:      # exactly co-spherical: corners of an axis-aligned box
            lo, hi = rng.random(3), rng.random(3) + 1.0
            corners = np.array([[hi[0] if i & 1 else lo[0], hi[1] if i & 2 else lo[1],
                                 hi[2] if i & 4 else lo[2]] for i in range(8)])
            p = corners[rng.permutation(8)[:5]]
        elif kind == 2:    # four points on an axis plane
            p[:4, 2] = p[0, 2]
        elif kind == 3:    # near-degenerate: a box corner nudged by one ulp
            lo, hi = rng.random(3), rng.random(3) + 1.0
            corners = np.array([[hi[0] if i & 1 else lo[0], hi[1] if i & 2 else lo[1],
                                 hi[2] if i & 4 else lo[2]] for i in range(8)])
            p = corners[rng.permutation(8)[:5]].copy()
            p[4, 0] = np.nextafter(p[4, 0], 10.0)
        out.append(p)
    return out


def test_predicates_match_rational_definitions():
    rng = np.random.default_rng(11)
    for p in _random_tuples(rng, 120):
        assert oracle.orient3d(*p[:4]) == orient_def(*p[:4])
        assert oracle.insphere(*p) == insphere_def(*p)


def test_orient3d_axis_plane_zero_and_sign():
    assert oracle.orient3d([0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.2, 0.0]) == 0
    assert oracle.orient3d([0, 0, 0], [1, 0, 0], [0, 1, 0], [0.0, 0.0, 1e-300]) == 1
    assert oracle.orient3d([0, 0, 0], [0, 1, 0], [1, 0, 0], [0.0, 0.0, 1.0]) == -1


def test_perturbation_matches_numeric_limit():
    """Section 2.4 item 3: the symbolic sign equals the sign of the lifted determinant with the
    lifting of point i raised by delta^k_i, k_i = 1 for the largest input index, 2 for the
    next, ... and delta tiny (here 2^-300 on integer coordinates)."""
    rng = np.random.default_rng(5)
    delta = Fraction(1, 2 ** 300)
    checked = 0
    for _ in range(60):
        box = lattice(2) * rng.integers(1, 4, size=3) + rng.integers(-2, 3, size=3)
        sel = rng.permutation(8)[:5]
        pts = box[sel]
        if orient_def(*pts[:4]) <= 0:
            pts[[2, 3]] = pts[[3, 2]]
            if orient_def(*pts[:4]) <= 0:
                continue
        ids = rng.permutation(1000)[:5]
        rank = np.argsort(-ids)          # position 0 = largest id
        k = np.empty(5, dtype=int)
        k[rank] = np.arange(1, 6)
        eps = [delta ** int(k[i]) for i in range(5)]
        assert insphere_def(*pts) == 0
        assert oracle.insphere_sos(pts, ids) == insphere_def(*pts, eps=eps)
        checked += 1
    assert checked > 30


# ----------------------------------------------------------------------------- data structures
def test_fig2_adjacency_encoding():
    g = golden("fig2_adjacency.json")
    nbr = oracle.adjacency(np.array(g["tets"])).reshape(-1)
    for src, dst in g["neighbor_ID"].items():
        ts, fs = src.replace("4*t", "").split("+")
        td, fd = dst.replace("4*t", "").split("+")
        assert nbr[4 * int(ts) + int(fs)] == 4 * int(td) + int(fd)
    # the other facets of the four are unmatched (the figure shows '-')
    assert (nbr == 0xFFFFFFFF).sum() == 16 - 6


def test_brio_round_sizes_table2():
    g = golden("brio_table2.json")
    r = oracle.brio_rounds(g["n"], seed=12345)
    counts = np.bincount(r)
    assert counts.tolist() == g["round_sizes"]
    assert np.cumsum(counts).tolist() == g["mesh_vertices_after_round"]
    assert oracle.brio_rounds(1500, 1).max() == 0
    r = oracle.brio_rounds(2049, 1)
    assert np.bincount(r).tolist() == [2048, 1]


def _moore_all(m):
    q = np.array(list(itertools.product(range(2 ** m), repeat=3)), dtype=np.uint32)[:, ::-1]
    return q, oracle.moore_index(np.ascontiguousarray(q), m)


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_moore_curve_closed_and_face_adjacent(m):
    q, keys = _moore_all(m)
    assert np.array_equal(np.sort(keys), np.arange(8 ** m, dtype=np.uint64))
    walk = q[np.argsort(keys)].astype(np.int64)
    steps = np.abs(np.diff(walk, axis=0)).sum(axis=1)
    assert (steps == 1).all()
    assert np.abs(walk[-1] - walk[0]).sum() == 1          # closed: Moore, not Hilbert
    # self-similarity: each top octant is one contiguous run of keys
    octant = (walk >> (m - 1)) if m > 0 else walk
    changes = (np.abs(np.diff(octant, axis=0)).sum(axis=1) > 0).sum()
    assert changes == 7


def test_moore_keys_quantisation():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.5, 0.25, 0.75]])
    keys = oracle.moore_keys(x)
    cells = np.array([[0, 0, 0], [2 ** 21 - 1] * 3, [2 ** 20, 2 ** 19, 3 * 2 ** 19]], dtype=np.uint32)
    assert np.array_equal(keys, oracle.moore_index(cells, 21))
    assert oracle.moore_keys(np.ones((5, 3))).tolist() == [oracle.moore_index(np.zeros((1, 3)), 21)[0]] * 5


def test_insertion_order_is_lexicographic_sort():
    x = synth.uniform_cube(5000, 9)
    x[100:120] = x[200:220]          # duplicates share keys
    perm = oracle.insertion_order(x, 77)
    keys = oracle.moore_keys(x)
    rounds = oracle.brio_rounds(len(x), 77)
    ref = np.lexsort((np.arange(len(x)), keys, rounds))
    assert np.array_equal(perm, ref)


def test_dedup_keeps_smallest_index():
    x = synth.uniform_cube(50, 2)
    x[[7, 30, 45]] = x[12]
    x[20] = x[3]
    rep = oracle.dedup(x)
    assert rep[12] == 7 and rep[30] == 7 and rep[45] == 7 and rep[7] == 7
    assert rep[20] == 3 and rep[3] == 3
    assert (rep[[0, 1, 2, 5]] == [0, 1, 2, 5]).all()


# ----------------------------------------------------------------------------- triangulations
def test_general_position_matches_qhull():
    from scipy.spatial import Delaunay
    x = synth.uniform_cube(10000, 3)
    tets, st = oracle.delaunay(x, seed=1, validate=True)
    assert st["validate_flags"] == 0
    assert np.array_equal(tets, canon_list(Delaunay(x).simplices, x))


@pytest.mark.parametrize("name", sorted(DEGENERATE_SETS))
def test_bowyer_watson_equals_brute_force(name):
    x = DEGENERATE_SETS[name]
    bf = oracle.brute_force(x)
    tets, st = oracle.delaunay(x, seed=3, validate=True)
    assert st["validate_flags"] == 0
    assert np.array_equal(tets, bf)


def test_brute_force_random_small():
    for seed in range(4):
        x = synth.uniform_cube(30, 100 + seed)
        tets, st = oracle.delaunay(x, seed=seed, validate=True)
        assert st["validate_flags"] == 0
        assert np.array_equal(tets, oracle.brute_force(x))


@pytest.mark.parametrize("name", ["lattice3", "sphere9", "two_planes"])
def test_order_independence(name):
    x = DEGENERATE_SETS[name]
    ref, _ = oracle.delaunay(x)
    rng = np.random.default_rng(1)
    for _ in range(5):
        tets, st = oracle.delaunay(x, order=rng.permutation(len(x)), validate=True)
        assert st["validate_flags"] == 0
        assert np.array_equal(tets, ref)


def test_order_independence_mixed():
    x = synth.degenerate_mix(3000, 4)
    x[2500:2520] = x[2900:2920]      # repeated lattice sites (the full-size mix repeats ~1e6)
    ref, st = oracle.delaunay(x, seed=1, validate=True)
    assert st["validate_flags"] == 0 and st["n_dups"] > 0
    rng = np.random.default_rng(2)
    for _ in range(3):
        tets, _ = oracle.delaunay(x, order=rng.permutation(len(x)))
        assert np.array_equal(tets, ref)


@pytest.mark.parametrize("name", sorted(DEGENERATE_SETS))
def test_triangulation_invariants(name):
    from scipy.spatial import ConvexHull
    x = DEGENERATE_SETS[name]
    tets, st = oracle.delaunay(x, validate=True)
    assert euler_ok(tets)
    assert st["n_ghosts"] == 2 * st["n_hull_vertices"] - 4
    hull = ConvexHull(x)
    vol = float(exact_volume6(tets, x)) / 6.0
    assert abs(vol - hull.volume) <= 1e-12 * hull.volume
    # every point is a vertex (duplicates aside)
    assert len(np.unique(tets)) == st["n_unique"]


def test_uniform_statistics():
    """Section 2.4/2.5: about 6n tetrahedra, cavities of about 20 and balls of about 26;
    Poisson-Delaunay mean 24 pi^2 / 35 = 6.77 tetrahedra per point."""
    x = synth.uniform_cube(100000, 1)
    tets, st = oracle.delaunay(x, seed=1)
    per_point = len(tets) / len(x)
    assert 6.4 < per_point < 24 * np.pi ** 2 / 35
    assert 15 < st["sum_cavity"] / len(x) < 30
    assert 20 < st["sum_ball"] / len(x) < 35


def test_degenerate_inputs_are_reported():
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float))
    assert e.value.code == oracle.EDEGENERATE
    plane = np.c_[synth.uniform_cube(40, 1)[:, :2], np.zeros(40)]
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(plane)
    assert e.value.code == oracle.EDEGENERATE
    bad = synth.uniform_cube(10, 1)
    bad[3, 1] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.delaunay(bad)
    assert e.value.code == oracle.EINVAL


# ----------------------------------------------------------------------------- planted mistakes
def _pins_pass():
    """A compact run of the pins above; False as soon as one fails."""
    checks = [
        test_insphere_worked_example,
        test_predicates_match_rational_definitions,
        test_perturbation_matches_numeric_limit,
        test_brio_round_sizes_table2,
        lambda: test_moore_curve_closed_and_face_adjacent(2),
        test_moore_keys_quantisation,
        lambda: test_bowyer_watson_equals_brute_force("two_planes"),
        lambda: test_bowyer_watson_equals_brute_force("sphere9"),
        test_general_position_matches_qhull,
    ]
    for c in checks:
        try:
            c()
        except (AssertionError, oracle.OracleError):
            return False
    return True


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5, 6, 7, 8])
def test_planted_mistakes_are_caught(mutation):
    """Each planted mistake (a flipped sign, a reversed order, a dropped term, transposed
    operands, a dropped ghost rule, a wrong rotation, an off-by-one round, a dropped bit)
    makes at least one pin fail."""
    assert _pins_pass()
    oracle.set_mutation(mutation)
    try:
        assert not _pins_pass()
    finally:
        oracle.set_mutation(0)
