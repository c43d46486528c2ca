"""The paper's CPU thread scheme (oracle/paper_cpu.cpp, Sections 3.2 to 3.4) against the serial
oracle: the perturbed Delaunay triangulation is unique, so every thread count, partition size and
schedule must give the oracle's canonical tetrahedra exactly. Small partitions (a few dozen points
per thread) force aborts at partition borders and many re-partitioned passes."""
import numpy as np
import pytest

import oracle
from oracle import paper_cpu
from paper_1805_08831_gb300 import synth
from tests.inputs import DEGENERATE_SETS


@pytest.mark.parametrize("threads,per_thread", [(1, 3000), (2, 3000), (4, 100), (8, 40), (16, 20)])
def test_uniform_equals_the_serial_oracle(threads, per_thread):
    x = synth.uniform_cube(20000, 3)
    got, st = paper_cpu.delaunay(x, threads, min_per_thread=per_thread)
    assert np.array_equal(got, oracle.delaunay(x)[0])
    assert st["n_tets"] == len(got) and st["n_unique"] == len(x)
    if threads > 2:
        assert st["aborted"] > 0 and st["passes"] > 3 and st["max_threads"] > 1


@pytest.mark.parametrize("name", sorted(DEGENERATE_SETS))
def test_degenerate_sets_equal_the_serial_oracle(name):
    x = DEGENERATE_SETS[name]
    got, _ = paper_cpu.delaunay(x, 4, min_per_thread=2)
    assert np.array_equal(got, oracle.delaunay(x)[0])


@pytest.mark.parametrize("kind", ["degenerate", "slab"])
def test_mixed_inputs_with_duplicates(kind):
    x = synth.make(kind, 20000, 5)
    x[-300:] = x[:300]
    got, st = paper_cpu.delaunay(x, 8, seed=3, min_per_thread=50)
    ref, rst = oracle.delaunay(x, seed=3)
    assert np.array_equal(got, ref) and st["n_unique"] == rst["n_unique"]


def test_repeated_runs_agree():
    """Thread timing changes which points abort and in which pass they land; the output may not."""
    x = synth.uniform_cube(15000, 9)
    first, _ = paper_cpu.delaunay(x, 8, min_per_thread=30)
    for _ in range(3):
        again, _ = paper_cpu.delaunay(x, 8, min_per_thread=30)
        assert np.array_equal(again, first)


def test_errors():
    with pytest.raises(RuntimeError):
        paper_cpu.delaunay(synth.uniform_cube(100, 1), 0)
    with pytest.raises(RuntimeError):
        paper_cpu.delaunay(np.zeros((10, 3)), 2)          # no volume
