"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *produces* inputs: triangulated bodies (vertices and
faces), Eulerian grid face coordinates, a Fourier velocity field and random
marker forces.  It holds none of the transfer-function arithmetic (no
centroids, no areas, no weights, no shape functions); those live, written
independently, in ``oracle/`` (CPU reference) and in the CUDA library.
"""

from .geometry import icosphere, random_rotation, place_bodies, sh_basis, sh_radial_factor
from .grids import uniform_faces, tanh_faces
from .fields import FourierModes, fourier_modes, field_at_cells_np, forces_np
from .configs import WORKLOADS, make_workload, Workload

__all__ = [
    "icosphere", "random_rotation", "place_bodies", "sh_basis", "sh_radial_factor",
    "uniform_faces", "tanh_faces",
    "FourierModes", "fourier_modes", "field_at_cells_np", "forces_np",
    "WORKLOADS", "make_workload", "Workload",
]
