"""The five synthetic workloads of the benchmark plan, plus scaled-down variants for tests.

C1  one level-4 icosphere (5120 faces), radius 0.25, centre U[-0.1,0.1]^3, in a
    uniform periodic 64^3 grid on [-1,1]^3; float64; velocity modes kmax=4.
C2  2000 ellipsoids, semi-axes U[0.6,1.4]*R with R=6h (h=2/512), random
    orientation, each a level-3 icosphere (1280 faces), placed without overlap
    in a uniform periodic 512^3 grid; float32; kmax=16.
C3  10^4 bodies, half level-3 and half level-4 icospheres, radius U[4h,10h]
    (h=2/1024), each vertex moved radially by a 5% random spherical-harmonic
    deformation (l<=6); 1024^3 grid, uniform periodic in x and y, tanh-stretched
    (beta=1.5) and walled in z; float32.
C4  C2's geometry run with bfloat16 and float32 field storage.
C5  C3's grid, used to label surrogate training offsets.

Seeds are 1805011130 + config number, with independent substreams for
geometry (0), velocity (1) and forces (2).
"""

from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

from .fields import FourierModes, fourier_modes, forces_np
from .geometry import icosphere, place_bodies, random_rotation, sh_basis, sh_radial_factor
from .grids import tanh_faces, uniform_faces

BASE_SEED = 1805011130


@dataclass
class Workload:
    name: str
    faces: Tuple[np.ndarray, np.ndarray, np.ndarray]   # per axis, n+1 float64 faces
    periodic: Tuple[bool, bool, bool]
    vertices: np.ndarray          # (nv, 3) float64
    tri: np.ndarray               # (nt, 3) int32 indices into vertices
    body_faces: np.ndarray        # (nb+1,) int64 face offsets per body
    modes: FourierModes
    seed: int
    real: str                     # "f64" or "f32": precision of the transfer path
    field_dtype: str              # "f64", "f32" or "bf16": storage of u and f
    notes: dict = field(default_factory=dict)

    @property
    def n(self):
        return tuple(len(f) - 1 for f in self.faces)

    @property
    def n_markers(self):
        return int(len(self.tri))

    def forces(self):
        """Marker forces F[3][M] ~ N(0,1), float64 (cast by the consumer)."""
        return forces_np(np.random.default_rng([self.seed, 2]), self.n_markers)


def _rng(seed, stream):
    return np.random.default_rng([seed, stream])


def _assemble(bodies_v, bodies_f):
    vo, fo = [0], [0]
    for v, f in zip(bodies_v, bodies_f):
        vo.append(vo[-1] + len(v))
        fo.append(fo[-1] + len(f))
    V = np.concatenate(bodies_v, axis=0)
    T = np.concatenate([f + vo[b] for b, f in enumerate(bodies_f)], axis=0).astype(np.int32)
    return V, T, np.asarray(fo, dtype=np.int64)


def c1(n=64, level=4, radius=0.25, real="f64", field_dtype=None):
    seed = BASE_SEED + 1
    g = _rng(seed, 0)
    faces = tuple(uniform_faces(n) for _ in range(3))
    v, f = icosphere(level)
    centre = g.uniform(-0.1, 0.1, size=3)
    V = centre + radius * v
    modes = fourier_modes(_rng(seed, 1), kmax=4)
    return Workload("c1", faces, (True, True, True), V, f.astype(np.int32),
                    np.array([0, len(f)], dtype=np.int64), modes, seed, real,
                    field_dtype or real, {"radius": radius, "level": level})


def c2(n=512, n_bodies=2000, level=3, real="f32", field_dtype=None, seed_offset=2):
    seed = BASE_SEED + seed_offset
    g = _rng(seed, 0)
    h = 2.0 / n
    R = 6.0 * h
    faces = tuple(uniform_faces(n) for _ in range(3))
    axes = g.uniform(0.6, 1.4, size=(n_bodies, 3)) * R
    rot = [random_rotation(g) for _ in range(n_bodies)]
    centres = place_bodies(g, axes.max(axis=1), [-1] * 3, [1] * 3, gap=2 * h, margin=[2 * h] * 3)
    v, f = icosphere(level)
    bv = [centres[b] + (v * axes[b]) @ rot[b].T for b in range(n_bodies)]
    V, T, fo = _assemble(bv, [f] * n_bodies)
    modes = fourier_modes(_rng(seed, 1), kmax=16)
    return Workload("c2", faces, (True, True, True), V, T, fo, modes, seed, real,
                    field_dtype or real, {"R": R, "level": level, "n_bodies": n_bodies})


def c3(n=1024, n_bodies=10000, beta=1.5, real="f32", field_dtype=None):
    seed = BASE_SEED + 3
    g = _rng(seed, 0)
    h = 2.0 / n
    faces = (uniform_faces(n), uniform_faces(n), tanh_faces(n, beta))
    levels = np.where(np.arange(n_bodies) % 2 == 0, 3, 4)
    g.shuffle(levels)
    radii = g.uniform(4.0 * h, 10.0 * h, size=n_bodies)
    bound = radii * 1.05
    centres = place_bodies(g, bound, [-1] * 3, [1] * 3, gap=2 * h,
                           margin=[2 * h, 2 * h, 8 * h])
    spheres = {L: icosphere(L) for L in (3, 4)}
    basis = {L: sh_basis(spheres[L][0], lmax=6) for L in (3, 4)}
    bv, bf = [], []
    for b in range(n_bodies):
        v, f = spheres[int(levels[b])]
        r = radii[b] * sh_radial_factor(basis[int(levels[b])], g, amplitude=0.05)
        bv.append(centres[b] + v * r[:, None])
        bf.append(f)
    V, T, fo = _assemble(bv, bf)
    modes = fourier_modes(_rng(seed, 1), kmax=16)
    return Workload("c3", faces, (True, True, False), V, T, fo, modes, seed, real,
                    field_dtype or real, {"beta": beta, "n_bodies": n_bodies})


WORKLOADS = {"c1": c1, "c2": c2, "c3": c3}


def make_workload(name, **kw):
    return WORKLOADS[name](**kw)
