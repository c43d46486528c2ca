"""Seeded synthetic point clouds shared by the tests, the bench and the oracle runs.

This module only draws random numbers; it holds none of the triangulation arithmetic.
Every stream is the counter-based SplitMix64 generator (Steele, Lea, Flood 2014):
value i of the stream with seed s is mix64(s * 2^32 + (i + 1) * 0x9E3779B97F4A7C15),
and a uniform double is (value >> 11) * 2^-53, a multiple of 2^-53 in [0, 1).
Gaussians use the Box-Muller transform on two uniforms.

The paper measures only i.i.d. uniform clouds in the unit cube (Fig. 6, Fig. 9, Table 1).
The other recipes are the degenerate, batched and slab workloads of the evaluation plan;
their exact recipe is written next to each function.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def u64_stream(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Values offset .. offset+count-1 of the SplitMix64 stream for `seed`."""
    base = np.uint64((seed << 32) & 0xFFFFFFFFFFFFFFFF)
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = base + i * _GAMMA
    return mix64(state)


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1), each a multiple of 2^-53."""
    v = u64_stream(seed, count, offset) >> np.uint64(11)
    return v.astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal doubles by Box-Muller (cosine branch only)."""
    u = uniform(seed, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def uniform_cube(n: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^3, row-major [n, 3] float64."""
    return uniform(seed, 3 * n).reshape(n, 3)


def degenerate_mix(n: int, seed: int, literal_sphere: bool = False) -> np.ndarray:
    """The degenerate / non-uniform mix, in this order of rows:

    * 40 % on the sphere inscribed in the unit cube (centre 1/2, radius 1/2; with
      `literal_sphere` the radius-1 sphere around the origin): normalised Gaussian directions;
    * 40 % in 64 Gaussian clusters (sigma 0.01, centres uniform in the cube, equal shares);
    * 20 % on the integer lattice {0..99}^3 scaled by 1/99 (i, j, k drawn uniformly), which
      repeats sites (exact duplicates), puts 8 box corners on one sphere and 4 points on
      one axis-aligned plane, so exact predicates and the perturbation are exercised.
    """
    n_sph = (2 * n) // 5
    n_clu = (2 * n) // 5
    n_lat = n - n_sph - n_clu
    g = gaussian(seed, 3 * n_sph).reshape(n_sph, 3)
    norm = np.sqrt((g * g).sum(axis=1, keepdims=True))
    norm[norm == 0.0] = 1.0
    d = g / norm
    sph = d if literal_sphere else 0.5 + 0.5 * d
    centres = uniform(seed + 1, 3 * 64).reshape(64, 3)
    which = np.arange(n_clu) % 64
    clu = centres[which] + 0.01 * gaussian(seed + 2, 3 * n_clu).reshape(n_clu, 3)
    ijk = (u64_stream(seed + 3, 3 * n_lat) % np.uint64(100)).astype(np.float64)
    lat = (ijk / 99.0).reshape(n_lat, 3)
    return np.ascontiguousarray(np.concatenate([sph, clu, lat], axis=0))


def cloud_sizes(n_clouds: int, seed: int, lo: int = 50, hi: int = 50000) -> np.ndarray:
    """Cloud sizes round(exp(U[ln lo, ln hi])) for the batched workload."""
    u = uniform(seed, n_clouds)
    s = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))
    return np.clip(s, lo, hi).astype(np.int64)


def batched_clouds(n_clouds: int, seed: int, lo: int = 50, hi: int = 50000):
    """Independent uniform clouds: returns (xyz [sum n_i, 3], offsets [n_clouds + 1])."""
    sizes = cloud_sizes(n_clouds, seed, lo, hi)
    offsets = np.zeros(n_clouds + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(sizes).astype(np.uint64)
    xyz = uniform(seed + 1, 3 * int(offsets[-1])).reshape(-1, 3)
    return xyz, offsets


def cube_and_slab(n: int, seed: int, slab_frac: float = 0.3, thickness: float = 1e-3) -> np.ndarray:
    """70 % uniform in the cube, 30 % in the slab z in [0.5 - t/2, 0.5 + t/2), x, y uniform."""
    n_slab = int(round(n * slab_frac))
    n_cube = n - n_slab
    cube = uniform(seed, 3 * n_cube).reshape(n_cube, 3)
    s = uniform(seed + 1, 3 * n_slab).reshape(n_slab, 3)
    s[:, 2] = (0.5 - 0.5 * thickness) + thickness * s[:, 2]
    return np.ascontiguousarray(np.concatenate([cube, s], axis=0))



def box_surface(k: int) -> np.ndarray:
    """Lattice points (i, j, l) / k of the unit cube's surface, k intervals per edge: the vertices
    of a boundary mesh of the cube with edge length 1 / k, (k + 1)^3 - (k - 1)^3 points, in
    (l, j, i) order."""
    g = np.arange(k + 1, dtype=np.float64) / k
    z, y, x = np.meshgrid(np.arange(k + 1), np.arange(k + 1), np.arange(k + 1), indexing="ij")
    on = (x == 0) | (x == k) | (y == 0) | (y == k) | (z == 0) | (z == k)
    return np.ascontiguousarray(np.c_[g[x[on]], g[y[on]], g[z[on]]])

WORKLOADS = {
    "uniform": uniform_cube,
    "degenerate": degenerate_mix,
    "slab": cube_and_slab,
}


def make(kind: str, n: int, seed: int) -> np.ndarray:
    """Generate one named single-cloud workload."""
    return WORKLOADS[kind](n, seed)
