"""Seeded synthetic point clouds shaped like the multi-agent workloads of
Brodu, "Spherical Indexing for Neighborhood Queries" (Sec. IV.A: randomly
placed objects and query centers in a cubic region, cyclic or not).

This module only draws inputs.  It holds none of the neighborhood-query
arithmetic, so both the CUDA path and the CPU oracle can be fed from it
without sharing any of the method's code.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: value k of stream `seed` is mix(seed + (k + 1) * GOLDEN).

Point layout everywhere: float32 array of shape (n, 4), columns x, y, z and an
unused fourth lane (kept at 0) so that each point is one 16-byte vector.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based splitmix64: uint64 values k = offset .. offset+count-1."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def unit24(u: np.ndarray) -> np.ndarray:
    """Top 24 bits as a float64 in [0, 1) on a 2^-24 grid (exact in float32)."""
    return (u >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


def unit53_open(u: np.ndarray) -> np.ndarray:
    """Top 53 bits as a float64 in (0, 1] (never 0, for Box-Muller's log)."""
    return ((u >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def _to_box_f32(x: np.ndarray, length: float, origin: float) -> np.ndarray:
    """Round to float32 and keep the value inside [origin, origin + length)."""
    hi = np.float32(origin) + np.float32(length)
    x32 = x.astype(np.float32)
    x32 = np.where(x32 >= hi, np.float32(origin), x32)
    x32 = np.where(x32 < np.float32(origin), np.float32(origin), x32)
    return x32


def uniform_points(n: int, seed: int, box=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n points i.i.d. uniform in the box; coordinates on a 2^-24 * L grid."""
    u = splitmix64(seed, 3 * n).reshape(n, 3)
    out = np.zeros((n, 4), dtype=np.float32)
    for a in range(3):
        x = float(origin[a]) + unit24(u[:, a]) * float(box[a])
        out[:, a] = _to_box_f32(x, float(box[a]), float(origin[a]))
    return out


def gaussian_mixture_points(n: int, seed: int, n_comp: int = 64, sigma: float = 0.02,
                            box: float = 1.0) -> np.ndarray:
    """n points from an isotropic Gaussian mixture, centers uniform in the cube
    [0, box)^3, wrapped periodically; equal component weights."""
    cu = splitmix64(seed ^ 0xC0FFEE, 3 * n_comp).reshape(n_comp, 3)
    centers = unit24(cu) * box
    u = splitmix64(seed, 5 * n).reshape(n, 5)
    comp = (u[:, 0] % np.uint64(n_comp)).astype(np.int64)
    # Box-Muller in float64: two uniforms give two normals; a third pair
    # supplies the z normal.
    u1, u2, u3, u4 = (unit53_open(u[:, k]) for k in range(1, 5))
    rad1 = np.sqrt(-2.0 * np.log(u1))
    rad2 = np.sqrt(-2.0 * np.log(u3))
    g = np.stack([rad1 * np.cos(2 * np.pi * u2), rad1 * np.sin(2 * np.pi * u2),
                  rad2 * np.cos(2 * np.pi * u4)], axis=1)
    x = centers[comp] + sigma * g
    x = x - np.floor(x / box) * box
    out = np.zeros((n, 4), dtype=np.float32)
    for a in range(3):
        out[:, a] = _to_box_f32(x[:, a], box, 0.0)
    return out


def terrain_points(n: int, seed: int, flying: float = 0.02, z0: float = 0.5, amp: float = 0.01,
                   waves: int = 3) -> np.ndarray:
    """Agents on a bumpy terrain with a few flying objects: x, y uniform in the
    unit square, z = z0 + amp * sin(2 pi waves x) * sin(2 pi waves y) for all
    but a fraction `flying`, whose z is uniform in [0, 1)."""
    u = splitmix64(seed, 4 * n).reshape(n, 4)
    x, y, f, zf = (unit24(u[:, k]) for k in range(4))
    z = z0 + amp * np.sin(2 * np.pi * waves * x) * np.sin(2 * np.pi * waves * y)
    z = np.where(f < flying, zf, z)
    out = np.zeros((n, 4), dtype=np.float32)
    out[:, 0] = _to_box_f32(x, 1.0, 0.0)
    out[:, 1] = _to_box_f32(y, 1.0, 0.0)
    out[:, 2] = _to_box_f32(z, 1.0, 0.0)
    return out


def normal_steps(n: int, seed: int, step: int) -> np.ndarray:
    """Standard normal (n, 3) float64 increments for time step `step`."""
    u = splitmix64(seed + 0x5DEECE66D * (step + 1), 4 * n).reshape(n, 4)
    u1, u2, u3, u4 = (unit53_open(u[:, k]) for k in range(4))
    rad1 = np.sqrt(-2.0 * np.log(u1))
    rad2 = np.sqrt(-2.0 * np.log(u3))
    return np.stack([rad1 * np.cos(2 * np.pi * u2), rad1 * np.sin(2 * np.pi * u2),
                     rad2 * np.cos(2 * np.pi * u4)], axis=1)


def random_walk_step(pos: np.ndarray, seed: int, step: int, sigma: float,
                     box=(1.0, 1.0, 1.0)) -> np.ndarray:
    """One Gaussian random-walk step x += N(0, sigma^2), wrapped into the box."""
    n = pos.shape[0]
    g = normal_steps(n, seed, step)
    out = np.zeros_like(pos)
    for a in range(3):
        x = pos[:, a].astype(np.float64) + sigma * g[:, a]
        x = x - np.floor(x / box[a]) * box[a]
        out[:, a] = _to_box_f32(x, float(box[a]), 0.0)
    return out


# ---------------------------------------------------------------------------
# Workload descriptions (sizes of the paper-shaped configurations)
# ---------------------------------------------------------------------------

@dataclass
class Scene:
    """One point cloud on one power-of-two cubic-cell lattice."""
    pos: np.ndarray            # (n, 4) float32
    origin: tuple              # region lower corner
    cell_size: float           # side s of a cubic cell
    log2_cells: tuple          # lattice is 2^w cells per axis
    cyclic_mask: int           # bit0 = x, bit1 = y, bit2 = z
    r: float                   # radius query distance
    name: str = ""
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        # the library takes these as float32: keep the values it will see, so
        # that both sides of a comparison use the same radius and lattice
        self.origin = tuple(float(np.float32(o)) for o in self.origin)
        self.cell_size = float(np.float32(self.cell_size))
        self.r = float(np.float32(self.r))

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def box(self) -> tuple:
        return tuple(float(np.float32(self.cell_size) * np.float32(1 << w)) for w in self.log2_cells)


SEEDS = {
    "tiny": 0x51D00001,
    "uniform_1m": 0x51D00002,
    "mixture_1m": 0x51D00012,
    "knn_4m": 0x51D00003,
    "batched": 0x51D00004,
    "walk_1m": 0x51D00005,
}


def tiny_scene(n: int = 20_000, seed: int = SEEDS["tiny"]) -> Scene:
    """N=20k uniform in [0,1)^3, 32^3 lattice, non-cyclic, r=0.03 (K=8 unbounded)."""
    return Scene(uniform_points(n, seed), (0.0, 0.0, 0.0), 1.0 / 32, (5, 5, 5), 0,
                 0.03, "tiny_20k", {"k": 8})


def uniform_1m_scene(n: int = 1_000_000, seed: int = SEEDS["uniform_1m"]) -> Scene:
    """N=1M uniform, fully cyclic unit box, 128^3 lattice, r = 1.5 cell sides."""
    return Scene(uniform_points(n, seed), (0.0, 0.0, 0.0), 1.0 / 128, (7, 7, 7), 7,
                 1.5 / 128, "uniform_1m")


def mixture_1m_scene(n: int = 1_000_000, seed: int = SEEDS["mixture_1m"]) -> Scene:
    """N=1M, 64-component isotropic Gaussian mixture (sigma 0.02), cyclic, 128^3."""
    return Scene(gaussian_mixture_points(n, seed), (0.0, 0.0, 0.0), 1.0 / 128, (7, 7, 7), 7,
                 1.5 / 128, "mixture_1m")


def mixture_250k_scene(n: int = 250_000, seed: int = SEEDS["mixture_1m"]) -> Scene:
    """A quarter of the 1M mixture's components at the same density: 250k
    points, 16 components (sigma 0.02), cyclic, 128^3.  Each component holds
    as many points as one of the 1M mixture's, so the cells are as crowded;
    the smaller case serves profiling."""
    return Scene(gaussian_mixture_points(n, seed, n_comp=16), (0.0, 0.0, 0.0), 1.0 / 128, (7, 7, 7), 7,
                 1.5 / 128, "mixture_250k")


def knn_4m_scene(n: int = 4_000_000, seed: int = SEEDS["knn_4m"]) -> Scene:
    """N=4M uniform, cyclic in x and y, non-cyclic in z, 256^3 lattice, r_max = 4 cells."""
    return Scene(uniform_points(n, seed), (0.0, 0.0, 0.0), 1.0 / 256, (8, 8, 8), 3,
                 4.0 / 256, "knn_4m", {"k": (16, 64)})


def knn_250k_scene(n: int = 250_000, seed: int = SEEDS["knn_4m"]) -> Scene:
    """The 4M K-nearest configuration's density on a sixteenth of its
    region: 250k uniform points, cell side 1/256, 128 x 128 x 64 cells
    (load 0.238), cyclic in x and y, r_max = 4 cells; for profiling."""
    return Scene(uniform_points(n, seed, box=(0.5, 0.5, 0.25)), (0.0, 0.0, 0.0), 1.0 / 256, (7, 7, 6), 3,
                 4.0 / 256, "knn_250k", {"k": (16, 64)})


def batched_scenes(n_scenes: int = 256, seed: int = SEEDS["batched"],
                   n_lo: int = 1_000, n_hi: int = 200_000) -> list:
    """Independent scenes of uneven size: n log-uniform in [n_lo, n_hi], box side
    U[0.5, 4], lattice 2^U{4..7} per axis (cubic), radius U[1, 3] cell sides,
    cyclic mask uniform over the 8 combinations."""
    u = splitmix64(seed, 6 * n_scenes).reshape(n_scenes, 6)
    scenes = []
    for k in range(n_scenes):
        f = unit24(u[k])
        n = int(round(math.exp(math.log(n_lo) + f[0] * (math.log(n_hi) - math.log(n_lo)))))
        side = 0.5 + 3.5 * f[1]
        w = 4 + int(u[k, 2] % np.uint64(4))
        cell = float(np.float32(side / (1 << w)))
        r = float(np.float32((1.0 + 2.0 * f[3]) * cell))
        mask = int(u[k, 4] % np.uint64(8))
        box = float(np.float32(cell) * np.float32(1 << w))
        pos = uniform_points(n, seed + 0x1000 + k, box=(box, box, box))
        scenes.append(Scene(pos, (0.0, 0.0, 0.0), cell, (w, w, w), mask, r,
                            f"scene{k}"))
    return scenes
