"""Writes tests/golden/fullsize.json: the serial CPU oracle's canonical tetrahedron lists of the
full-size workloads, as counts and SHA-256 digests.

The Delaunay triangulation under the symbolic perturbation is unique (Section 2.1, Eq. 1 with
exact predicates, Section 2.4), so any correct construction of it gives exactly this list. The
GPU parity test (tests/test_gpu_fullsize.py) hashes the library's canonical list of the same
seeded input and compares.

Calls only `oracle/` and the input generators. Run on a CPU host, one workload at a time for the
1e8 ones (each holds about 45 GB of host memory and runs for tens of minutes):

    python tests/golden/make_fullsize.py uniform_1e7 degenerate_1e7
    python tests/golden/make_fullsize.py uniform_1e8
    python tests/golden/make_fullsize.py slab_1e8

The digest is over the [T, 4] uint32 array in C order, little-endian (the layout of
`dt_get_tets(canonical=1)`). `chunks` holds the digests of consecutive blocks of CHUNK rows, so a
mismatch can be located without the oracle's output.
"""
from __future__ import annotations

import fcntl
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CHUNK = 1 << 22  # rows per chunk digest

# name -> (generator kind, points, seed); the recipes are in paper_1805_08831_gb300/synth.py
WORKLOADS = {
    "uniform_1e7": ("uniform", 10_000_000, 2),
    "degenerate_1e7": ("degenerate", 10_000_000, 3),
    "uniform_1e8": ("uniform", 100_000_000, 2),
    "slab_1e8": ("slab", 100_000_000, 5),
}

OUT = os.path.join(HERE, "fullsize.json")


def digests(tets: np.ndarray) -> tuple[str, list[str]]:
    """SHA-256 of the whole little-endian [T, 4] uint32 list and of each CHUNK-row block."""
    t = np.ascontiguousarray(tets, dtype="<u4")
    whole = hashlib.sha256(memoryview(t).cast("B")).hexdigest()
    chunks = [hashlib.sha256(memoryview(t[i:i + CHUNK]).cast("B")).hexdigest()
              for i in range(0, len(t), CHUNK)]
    return whole, chunks


def run(name: str) -> dict:
    import oracle
    from paper_1805_08831_gb300 import synth
    kind, n, seed = WORKLOADS[name]
    xyz = synth.make(kind, n, seed)
    t0 = time.time()
    tets, st = oracle.delaunay(xyz, seed=seed, cap=int(6.9 * n) + 4096)
    secs = time.time() - t0
    whole, chunks = digests(tets)
    return {
        "kind": kind, "n": n, "seed": seed,
        "n_tets": int(len(tets)), "sha256": whole, "chunk_rows": CHUNK, "chunks": chunks,
        "first_rows": tets[:4].tolist(), "last_rows": tets[-4:].tolist(),
        "n_unique": int(st["n_unique"]), "n_dups": int(st["n_dups"]),
        "n_exact": int(st["n_exact"]), "n_sos": int(st["n_sos"]),
        "oracle_seconds": round(secs, 1),
    }


def main(names: list[str]) -> None:
    for name in names:
        if name not in WORKLOADS:
            raise SystemExit(f"unknown workload {name}; one of {sorted(WORKLOADS)}")
    for name in names:
        rec = run(name)
        with open(OUT + ".lock", "w") as lk:  # several workloads may run side by side
            fcntl.flock(lk, fcntl.LOCK_EX)
            data = {}
            if os.path.exists(OUT):
                with open(OUT) as f:
                    data = json.load(f)
            data[name] = rec
            tmp = OUT + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
                f.write("\n")
            os.replace(tmp, OUT)
        print(name, rec["n_tets"], rec["sha256"], rec["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
