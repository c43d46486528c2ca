"""Oracle of Delaunay refinement inside a box (TEST INFRASTRUCTURE ONLY: used by the tests and
the benchmark's CPU legs, never by the product path).

Section 4, Algorithm 2, the refinement loop (SamplePoints, FilterPoints, InsertPoints), on a
convex box whose faces are already covered by the input's hull, so that no boundary recovery is
needed. Plain float64 numpy plus the serial triangulation of `oracle.delaunay`, which is
re-run from scratch on the grown point set every iteration (the perturbed Delaunay
triangulation is unique, so that equals inserting the new points incrementally).

Definitions (the paper's thresholds r / h > 1.4 and 0.7 h; the rest is this repository's
reading, stated once here and followed by the CUDA path):
  * candidate: a finite tetrahedron with circumradius r, r^2 > (ratio * h)^2, whose circumcentre
    lies strictly inside the box; the candidate point is the circumcentre;
  * circumcentre of the tetrahedron with vertices a, b, c, d in increasing input index, every
    operation rounded on its own in this order:
        u = b - a, v = c - a, w = d - a
        |u|^2 = (u.x u.x + u.y u.y) + u.z u.z   (likewise |v|^2, |w|^2)
        v x w, w x u, u x v  with (p x q).x = p.y q.z - p.z q.y, .y = p.z q.x - p.x q.z,
                                   .z = p.x q.y - p.y q.x
        den = 2 (u . (v x w))
        o = ((|u|^2 (v x w) + |v|^2 (w x u)) + |w|^2 (u x v)) / den   (per component)
        centre = a + o,  r^2 = o . o
  * priority: candidate j outranks i when r_j^2 > r_i^2, or the radii are equal and the sorted
    input-index tuple of j's tetrahedron is lexicographically smaller;
  * filter, two steps with squared distances (components p - q, summed as above) against
    thr = (spacing * h)^2:
      1. a candidate is dropped when an existing point lies at squared distance < thr (the
         circumcentre of a near-flat tetrahedron is dominated by rounding and can fall on or
         outside its exact circumsphere, next to a vertex; the paper guards the same case by
         aborting a cavity with a vertex too close to the new point);
      2. a remaining candidate is dropped when a remaining candidate that outranks it lies at
         squared distance < thr;
  * insertion: the survivors, in increasing order of their tetrahedra's index tuples, are
    appended to the point set (their input indices follow the last point);
  * the loop ends after an iteration with no survivor, or after max_iters insertions.
Every inserted point is then at squared distance >= thr from every other point, so the loop
ends on any input.
"""
from __future__ import annotations

import numpy as np

import oracle


def _dot(p, q):
    return (p[..., 0] * q[..., 0] + p[..., 1] * q[..., 1]) + p[..., 2] * q[..., 2]


def _cross(p, q):
    return np.stack([p[..., 1] * q[..., 2] - p[..., 2] * q[..., 1],
                     p[..., 2] * q[..., 0] - p[..., 0] * q[..., 2],
                     p[..., 0] * q[..., 1] - p[..., 1] * q[..., 0]], axis=-1)


def circumcentres(P, tets):
    """Circumcentres [T, 3], squared circumradii [T] and sorted index tuples [T, 4] of the
    tetrahedra `tets` (rows of 4 input indices into P), by the fixed formula above."""
    P = np.asarray(P, dtype=np.float64)
    tup = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
    a, b, c, d = (P[tup[:, k]] for k in range(4))
    u, v, w = b - a, c - a, d - a
    lu, lv, lw = _dot(u, u), _dot(v, v), _dot(w, w)
    vw, wu, uv = _cross(v, w), _cross(w, u), _cross(u, v)
    den = 2.0 * _dot(u, vw)
    o = ((lu[:, None] * vw + lv[:, None] * wu) + lw[:, None] * uv) / den[:, None]
    return a + o, _dot(o, o), tup


def tuple_less(a, b):
    """Row-wise lexicographic a < b of integer tuples [k, 4]."""
    less = np.zeros(len(a), dtype=bool)
    open_ = np.ones(len(a), dtype=bool)
    for k in range(a.shape[1]):
        less |= open_ & (a[:, k] < b[:, k])
        open_ &= a[:, k] == b[:, k]
    return less


def outranks(r2_j, tup_j, r2_i, tup_i):
    """Row-wise priority of candidates j over candidates i: the larger r^2, then the smaller
    index tuple."""
    return (r2_j > r2_i) | ((r2_j == r2_i) & tuple_less(tup_j, tup_i))


def filter_keep(C, r2, tup, thr_d2):
    """Boolean mask of the candidates no outranking candidate lies closer to than thr_d2
    (squared). Pairs come from a k-d tree with a slightly larger radius, then each pair is
    decided by the fixed squared distance and the priority."""
    from scipy.spatial import cKDTree

    m = len(C)
    keep = np.ones(m, dtype=bool)
    if m < 2:
        return keep
    pairs = cKDTree(C).query_pairs(np.sqrt(thr_d2) * (1.0 + 1e-6), output_type="ndarray")
    if len(pairs) == 0:
        return keep
    i, j = pairs[:, 0], pairs[:, 1]
    d = C[i] - C[j]
    close = _dot(d, d) < thr_d2
    i, j = i[close], j[close]
    j_wins = outranks(r2[j], tup[j], r2[i], tup[i])
    keep[np.where(j_wins, i, j)] = False
    return keep


def far_from_points(C, P, thr_d2):
    """Boolean mask of the candidates with no point of P at squared distance < thr_d2."""
    from scipy.spatial import cKDTree

    ok = np.ones(len(C), dtype=bool)
    if len(C) == 0:
        return ok
    near = cKDTree(P).query_ball_point(C, np.sqrt(thr_d2) * (1.0 + 1e-6))
    for i, ids in enumerate(near):
        if ids:
            d = P[np.asarray(ids)] - C[i]
            if np.any(_dot(d, d) < thr_d2):
                ok[i] = False
    return ok


def sample(P, tets, box, thr_r2):
    """Candidates of one iteration: centres, r^2 and tuples of the large tetrahedra whose
    circumcentre is strictly inside the box."""
    with np.errstate(divide="ignore", invalid="ignore"):
        C, r2, tup = circumcentres(P, tets)
    lo, hi = np.asarray(box[:3], dtype=np.float64), np.asarray(box[3:], dtype=np.float64)
    inside = np.all((C > lo) & (C < hi), axis=1)
    sel = (r2 > thr_r2) & inside
    return C[sel], r2[sel], tup[sel]


def refine(points, size, box, ratio=1.4, spacing=0.7, max_iters=100):
    """(points [N + added, 3], canonical tetrahedra of their triangulation, iterations that
    inserted points, per-iteration insertion counts)."""
    P = np.ascontiguousarray(np.asarray(points, dtype=np.float64))
    thr_r2 = (ratio * size) * (ratio * size)
    thr_d2 = (spacing * size) * (spacing * size)
    tets, _ = oracle.delaunay(P)
    counts = []
    while len(counts) < max_iters:
        C, r2, tup = sample(P, tets, box, thr_r2)
        ok = far_from_points(C, P, thr_d2)
        C, r2, tup = C[ok], r2[ok], tup[ok]
        if len(C) == 0:
            break
        keep = filter_keep(C, r2, tup, thr_d2)
        C, tup = C[keep], tup[keep]
        order = np.lexsort((tup[:, 3], tup[:, 2], tup[:, 1], tup[:, 0]))
        P = np.ascontiguousarray(np.concatenate([P, C[order]], axis=0))
        counts.append(len(order))
        tets, _ = oracle.delaunay(P)
    return P, tets, len(counts), counts
