"""Coarse-grained collision detection on the Eulerian mesh (Section 4), plain CPU.

Test infrastructure only: the GPU library never imports this module.

The method marks a cell as a collision cell when markers of two or more
different bodies have it as their home cell.  The paper keeps an integer per
cell: 0 when no marker occupies it, the body index when the markers in it all
belong to one body, -1 when they belong to several; a marker whose home cell
holds -1 gets a collision force.  The end state does not depend on the order
in which markers are visited, so the oracle is that definition written out:
group the usable markers by home cell and look at the set of body indices.

Readings (the paper's index_of_marker is the home cell used by the MLS
support; body indices start at 1 as in its particle loop; markers without a
usable support and markers with a body index <= 0 take no part).
"""

import numpy as np


def collision_cells(home, ok, body, n):
    """Cell states of the collision array.

    home (3, M) home cells, ok (M,) usable markers, body (M,) body index,
    n = (nx, ny, nz).  Returns (keys, state): the linear indices
    (iz*ny + iy)*nx + ix of the occupied cells, sorted, and their state
    (body index, or -1 for markers of several bodies).
    """
    nx, ny, _ = n
    home = np.asarray(home, dtype=np.int64)
    body = np.asarray(body, dtype=np.int64)
    use = np.asarray(ok, dtype=bool) & (body > 0)
    keys = (home[2] * ny + home[1]) * nx + home[0]
    k, b = keys[use], body[use]
    cells = {}
    for cell, bid in zip(k.tolist(), b.tolist()):
        cells.setdefault(cell, set()).add(bid)
    out_keys = np.array(sorted(cells), dtype=np.int64)
    state = np.array([next(iter(cells[c])) if len(cells[c]) == 1 else -1 for c in out_keys.tolist()],
                     dtype=np.int64)
    return out_keys, state


def collision_flags(home, ok, body, n):
    """Per marker: 1 when its home cell holds markers of more than one body, else 0."""
    nx, ny, _ = n
    keys, state = collision_cells(home, ok, body, n)
    home = np.asarray(home, dtype=np.int64)
    body = np.asarray(body, dtype=np.int64)
    use = np.asarray(ok, dtype=bool) & (body > 0)
    lin = (home[2] * ny + home[1]) * nx + home[0]
    lookup = dict(zip(keys.tolist(), state.tolist()))
    flags = np.array([1 if u and lookup.get(c) == -1 else 0 for c, u in zip(lin.tolist(), use.tolist())],
                     dtype=np.int64)
    return flags
