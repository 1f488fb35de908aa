"""Pins of the oracle's buffered writes and d-dimensional grid walks (paper
Sec. 3.2.1 pending writes; Sec. 4.1 grid environments).

Buffered writes: flushing recorded (id, value) writes equals building a dict
of them in record order (later writes replace earlier ones) and assigning it.
Grid walks: d = 2, Moore, torus is the random walk; interior moves are uniform
over the 2d (von Neumann) or 3^d - 1 (Moore) neighbours and never stay; in a
bounded box agents never leave it and a corner agent chooses uniformly among
the neighbours inside; a one-cell box keeps agents in place."""
import numpy as np
import pytest
from scipy import stats

import oracle


def test_log_flush_is_dict_update():
    rng = np.random.default_rng(3)
    for dtype in (np.int32, np.uint8):
        col = rng.integers(0, 100, 50).astype(dtype)
        ids = rng.integers(0, 50, 400).astype(np.int32)
        vals = rng.integers(-2 ** 40, 2 ** 40, 400).astype(np.int64)
        pending = {}
        for i, v in zip(ids, vals):
            pending[int(i)] = int(v)
        want = col.copy()
        for i, v in pending.items():
            want[i] = np.array([v], dtype=np.int64).astype(dtype)[0]
        assert np.array_equal(oracle.log_flush(col.copy(), ids, vals), want)
    with pytest.raises(RuntimeError):
        oracle.log_flush(np.zeros(3, dtype=np.int32), [3], [1])


def test_two_dim_moore_torus_is_the_random_walk():
    p = oracle.Population("walk", 3000, seed=4, rep=1, L=37)
    x, y = p.x.copy(), p.y.copy()
    for t in range(12):
        oracle.grid_walk_step([x, y], [37, 37], True, True, 4, 1, t)
    p.step(12)
    assert np.array_equal(x, p.x) and np.array_equal(y, p.y)


def _one_step_offsets(d, moore, torus, size, start, n=30_000, seed=2):
    coords = [np.full(n, start[a], dtype=np.int32) for a in range(d)]
    before = [c.copy() for c in coords]
    oracle.grid_walk_step(coords, [size] * d, moore, torus, seed, 0, 0)
    return np.stack([c - b for c, b in zip(coords, before)], axis=1)


@pytest.mark.parametrize("d,moore", [(1, False), (1, True), (2, False), (3, False), (3, True), (4, True)])
def test_interior_moves_uniform_over_neighbours(d, moore):
    off = _one_step_offsets(d, moore, True, 20, [10] * d)
    assert np.all(np.abs(off) <= 1) and not np.any(np.all(off == 0, axis=1))
    if not moore:
        assert np.all(np.abs(off).sum(axis=1) == 1)
    keys, counts = np.unique(off, axis=0, return_counts=True)
    expected = (3 ** d - 1) if moore else 2 * d
    assert len(keys) == expected
    assert stats.chisquare(counts).pvalue > 1e-3


@pytest.mark.parametrize("moore,expected", [(True, {(1, 0), (0, 1), (1, 1)}), (False, {(1, 0), (0, 1)})])
def test_corner_in_bounded_box(moore, expected):
    off = _one_step_offsets(2, moore, False, 10, [0, 0])
    keys, counts = np.unique(off, axis=0, return_counts=True)
    assert {tuple(k) for k in keys} == expected
    assert stats.chisquare(counts).pvalue > 1e-3


def test_bounded_box_is_never_left_and_one_cell_box_stays():
    rng = np.random.default_rng(0)
    coords = [rng.integers(0, s, 5000).astype(np.int32) for s in (5, 3, 7)]
    for t in range(40):
        oracle.grid_walk_step(coords, [5, 3, 7], t % 2 == 0, False, 9, 0, t)
        for c, s in zip(coords, (5, 3, 7)):
            assert c.min() >= 0 and c.max() < s
    one = [np.zeros(10, dtype=np.int32), np.zeros(10, dtype=np.int32)]
    oracle.grid_walk_step(one, [1, 1], True, False, 1, 0, 0)
    assert np.all(one[0] == 0) and np.all(one[1] == 0)
