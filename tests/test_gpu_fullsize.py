"""Full-size workloads on the GPU.

* Bit-exact parity by digest: the canonical tetrahedron list of each full-size workload
  (1e7 uniform, 1e7 degenerate mix, 1e8 uniform, 1e8 cube + slab) hashes to the SHA-256 the serial
  CPU oracle's list of the same seeded input hashes to (tests/golden/fullsize.json, written by
  tests/golden/make_fullsize.py, which calls only the oracle). On a mismatch the per-chunk digests
  locate the first differing block of rows. The device certificate (dt_check) of each mesh is
  checked too: no faults, and its counts equal the oracle's.
* Beyond 2^30 tetrahedra: 2e8 uniform points, certified on the device.
* The bench's workload (1e7 uniform points, seed 2) is also checked by what holds at any size:
  every facet is shared by at most two tetrahedra, the triangulation is a topological ball
  (Euler characteristic 1), and sampled tetrahedra are positively oriented with an empty
  circumsphere against all 1e7 points (the oracle's exact predicates decide the points that lie
  near a sphere)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1805_08831_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_08831_gb300 as dt  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize.json")
with open(GOLDEN) as _f:
    FULLSIZE = json.load(_f)


@pytest.mark.parametrize("name", ["uniform_1e7", "degenerate_1e7", "uniform_1e8", "slab_1e8"])
def test_fullsize_canonical_list_matches_the_oracle_digest(name):
    rec = FULLSIZE[name]
    x = synth.make(rec["kind"], rec["n"], rec["seed"])
    with dt.Triangulation(seed=rec["seed"]) as t:
        t.insert(torch.from_numpy(x).cuda())
        st = t.stats()
        del x
        cert = t.check()
        tets = t.tets(canonical=True).cpu().numpy().view(np.uint32)
    assert cert == {"tets": rec["n_tets"], "bad_adjacency": 0, "bad_orientation": 0, "not_delaunay": 0,
                    "vertices": rec["n"] - rec["n_dups"]}
    assert st["n_dups"] == rec["n_dups"]
    assert len(tets) == rec["n_tets"]
    t = np.ascontiguousarray(tets, dtype="<u4")
    digest = hashlib.sha256(memoryview(t).cast("B")).hexdigest()
    if digest != rec["sha256"]:
        rows = rec["chunk_rows"]
        for k, want in enumerate(rec["chunks"]):
            got = hashlib.sha256(memoryview(t[k * rows:(k + 1) * rows]).cast("B")).hexdigest()
            if got != want:
                pytest.fail(f"{name}: first differing block of rows starts at {k * rows}; "
                            f"GPU rows there: {t[k * rows:k * rows + 4].tolist()}")
        pytest.fail(f"{name}: digest differs but no block does")
    assert t[:4].tolist() == rec["first_rows"] and t[-4:].tolist() == rec["last_rows"]


def test_uniform_1e7_is_a_delaunay_ball():
    n = 10 ** 7
    x = synth.uniform_cube(n, 2)
    xd = torch.from_numpy(x).cuda()
    with dt.Triangulation(seed=2) as t:
        t.insert(xd)
        tets = t.tets(canonical=False).long()
        st = t.stats()
    T = tets.shape[0]
    assert st["n_unique"] == n and 6.5 * n < T < 6.9 * n
    # facets: each shared by at most two tetrahedra; those on one tetrahedron bound the hull
    s, _ = tets.sort(dim=1)
    fac = torch.cat([s[:, [1, 2, 3]], s[:, [0, 2, 3]], s[:, [0, 1, 3]], s[:, [0, 1, 2]]]).int()
    _, fcount = torch.unique(fac, dim=0, return_counts=True)
    assert int(fcount.max()) <= 2
    F = fcount.numel()
    hull_facets = int((fcount == 1).sum())
    del fac, fcount
    edges = torch.cat([s[:, [0, 1]], s[:, [0, 2]], s[:, [0, 3]], s[:, [1, 2]], s[:, [1, 3]], s[:, [2, 3]]])
    E = torch.unique(edges[:, 0] * n + edges[:, 1]).numel()
    del edges
    V = torch.unique(s).numel()
    assert V == n
    assert V - E + F - T == 1
    assert hull_facets % 2 == 0  # a closed triangulated sphere has an even number of triangles
    # sampled tetrahedra: positive orientation and an empty circumsphere
    rng = np.random.default_rng(5)
    tet_np = tets[torch.from_numpy(rng.choice(T, 24, replace=False)).cuda()].cpu().numpy()
    for v in tet_np:
        a, b, c, d = x[v[0]], x[v[1]], x[v[2]], x[v[3]]
        assert oracle.orient3d(a, b, c, d) > 0
        # circumcentre in float64, then every point's power against the sphere
        A = np.array([b - a, c - a, d - a])
        rhs = 0.5 * np.array([np.dot(b - a, b - a), np.dot(c - a, c - a), np.dot(d - a, d - a)])
        ctr = a + np.linalg.solve(A, rhs)
        r2 = np.dot(ctr - a, ctr - a)
        pw = ((x - ctr) ** 2).sum(axis=1) - r2
        close = np.nonzero(pw < 1e-9 * max(r2, 1e-30))[0]
        for i in close:
            if i in v:
                continue
            # exactly: a point strictly inside the sphere of a positive tetrahedron has insphere < 0
            assert oracle.insphere(a, b, c, d, x[i]) >= 0, (v, i)


@pytest.mark.parametrize("n", [2 * 10 ** 8])
def test_beyond_2_pow_30_tetrahedra(n):
    """2e8 uniform points (1.35e9 tetrahedra, more than 2^30 slots) on one GPU. The oracle's
    list does not fit the host that writes the digests, so the mesh is certified on the device:
    reciprocal adjacency, positive orientation, every facet locally Delaunay under the exact
    perturbed predicates, and every point a vertex."""
    free, _ = torch.cuda.mem_get_info()
    if free < 150e9:
        pytest.skip("needs about 150 GB of free device memory")
    x = synth.uniform_cube(n, 2)
    xd = torch.from_numpy(x).cuda()
    del x
    with dt.Triangulation(seed=2) as t:
        t.insert(xd)
        del xd
        st = t.stats()
        cert = t.check()
    assert st["n_unique"] == n
    assert cert["tets"] > 2 ** 30 and 6.7 * n < cert["tets"] < 6.8 * n
    assert cert["bad_adjacency"] == cert["bad_orientation"] == cert["not_delaunay"] == 0
    assert cert["vertices"] == n
    assert st["device_bytes"] / n < 640
