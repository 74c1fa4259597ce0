"""Plain, slow, double-precision CPU oracle for the MLS transfer-function path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline leg and its reference arm) may import this
package.  It shares no code with the CUDA library and imports nothing from
it; the only code both sides use is the seeded input generator package
``workloads``.

Every function cites the passage of Spandan, Lohse, de Tullio & Verzicco,
"A fast moving least squares approximation with adaptive Lagrangian mesh
refinement for large scale immersed boundary simulations" (J. Comput. Phys.,
arXiv:1805.01113) that it follows.  Pins (tests that tie the oracle to the
paper and to mathematics rather than to itself) live in
``tests/test_oracle_*.py``; no function here is "parity unpinned".
"""

from . import collision, mlp, refine
from .mls import (
    Grid,
    marker_prep,
    locate,
    support,
    gaussian_weight,
    basis_values,
    shape_exact,
    moment_matrix,
    shape_exact_absolute_basis,
    shape_exact_gradient,
    interpolate_gradient,
    subnode_offsets,
    fast_table,
    shape_fast,
    forcing_scale,
    interpolate,
    spread,
    SparseField,
    direct_forcing,
)

__all__ = [
    "collision", "mlp", "refine", "Grid", "marker_prep", "locate", "support", "gaussian_weight",
    "basis_values", "shape_exact", "moment_matrix", "shape_exact_absolute_basis", "shape_exact_gradient", "interpolate_gradient", "subnode_offsets", "fast_table",
    "shape_fast", "forcing_scale", "interpolate", "spread", "SparseField",
    "direct_forcing",
]
