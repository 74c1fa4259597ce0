"""Pins for the coarse collision detection oracle (Section 4).

The oracle groups markers by home cell (the definition); these tests check it
against the paper's sequential update rule replayed in a Python loop, against
the situation of its schematic (three bodies in one cell), and against
invariances the definition fixes.
"""

import numpy as np

from oracle.collision import collision_cells, collision_flags


def _sequential(home, ok, body, n):
    """The update rule of the paper's listing, visited marker by marker: an
    empty cell takes the marker's body index; a cell holding another value
    than the marker's body becomes -1."""
    nx, ny, nz = n
    coll = np.zeros(nz * ny * nx, dtype=np.int64)
    for m in range(home.shape[1]):
        if not ok[m] or body[m] <= 0:
            continue
        c = (home[2, m] * ny + home[1, m]) * nx + home[0, m]
        if coll[c] == 0:
            coll[c] = body[m]
        if coll[c] != body[m]:
            coll[c] = -1
    return coll


def _random_case(rng, m, n, nbody):
    home = np.stack([rng.integers(0, n[d], m) for d in range(3)])
    ok = rng.random(m) > 0.05
    body = rng.integers(0, nbody + 1, m)          # 0: no body
    return home, ok, body


def test_matches_sequential_rule():
    rng = np.random.default_rng(7)
    n = (5, 4, 3)
    for _ in range(20):
        home, ok, body = _random_case(rng, 200, n, 4)
        seq = _sequential(home, ok, body, n)
        keys, state = collision_cells(home, ok, body, n)
        assert np.array_equal(np.nonzero(seq)[0], keys)
        assert np.array_equal(seq[keys], state)
        flags = collision_flags(home, ok, body, n)
        lin = (home[2] * n[1] + home[1]) * n[0] + home[0]
        want = (ok & (body > 0) & (seq[lin] == -1)).astype(np.int64)
        assert np.array_equal(flags, want)


def test_schematic_three_bodies_one_cell():
    """Three bodies with markers in the same cell: the cell is -1 and all their
    markers there are flagged; a cell with two markers of one body keeps it."""
    n = (4, 4, 4)
    home = np.array([[1, 1, 1, 2, 2], [1, 1, 1, 2, 2], [1, 1, 1, 2, 2]])
    body = np.array([1, 2, 3, 2, 2])
    ok = np.ones(5, dtype=bool)
    keys, state = collision_cells(home, ok, body, n)
    c1 = (1 * 4 + 1) * 4 + 1
    c2 = (2 * 4 + 2) * 4 + 2
    assert keys.tolist() == [c1, c2] and state.tolist() == [-1, 2]
    assert collision_flags(home, ok, body, n).tolist() == [1, 1, 1, 0, 0]


def test_order_invariance_and_relabelling():
    rng = np.random.default_rng(8)
    n = (6, 5, 4)
    home, ok, body = _random_case(rng, 300, n, 5)
    keys, state = collision_cells(home, ok, body, n)
    flags = collision_flags(home, ok, body, n)
    p = rng.permutation(300)
    k2, s2 = collision_cells(home[:, p], ok[p], body[p], n)
    assert np.array_equal(keys, k2) and np.array_equal(state, s2)
    assert np.array_equal(collision_flags(home[:, p], ok[p], body[p], n), flags[p])
    # Renaming bodies renames single-body cells and leaves -1 cells and flags alone.
    body2 = np.where(body > 0, body + 10, body)
    k3, s3 = collision_cells(home, ok, body2, n)
    assert np.array_equal(keys, k3)
    assert np.array_equal(s3, np.where(state > 0, state + 10, state))
    assert np.array_equal(collision_flags(home, ok, body2, n), flags)


def test_unusable_and_bodiless_markers_take_no_part():
    n = (3, 3, 3)
    home = np.zeros((3, 3), dtype=np.int64)
    keys, state = collision_cells(home, np.array([True, False, True]), np.array([1, 2, 0]), n)
    assert keys.tolist() == [0] and state.tolist() == [1]
