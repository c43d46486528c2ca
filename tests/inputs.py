"""Small hand-built point sets shared by the oracle and GPU parity tests (no method arithmetic)."""
import itertools

import numpy as np


def lattice(k):
    return np.array(list(itertools.product(range(k), repeat=3)), dtype=np.float64)


def sphere9():
    return np.array([p for p in itertools.product(range(-3, 4), repeat=3)
                     if sum(v * v for v in p) == 9], dtype=np.float64)


def cube_centre():
    return np.array(list(itertools.product((0.0, 1.0), repeat=3)) + [[0.5, 0.5, 0.5]])


DEGENERATE_SETS = {
    "lattice3": lattice(3),
    "lattice5": lattice(5) / 4.0,
    "sphere9": sphere9(),
    "cube_centre": cube_centre(),
    "two_planes": np.array([[x, y, z] for z in (0.0, 1.0) for x in range(3) for y in range(3)]
                           + [[0.5, 0.5, 0.5], [1.5, 0.7, 0.3]], dtype=np.float64),
    "lattice_dups": np.concatenate([lattice(2), lattice(2)[::-1], [[0.5, 0.5, 0.5]]]),
}
