"""Pins for the oracle's random walk (paper Sec. 5.1.2, re-cast as Moore moves
on an integer torus; grid environment of Sec. 4.1).

* Invariant of Sec. 5.1.3: every coordinate stays in [0, L); N fixed.
* One step covers the 8 Moore neighbours uniformly and never stays put.
* Closed form: per-axis step distribution {-1: 3/8, 0: 2/8, +1: 3/8}, so the
  unwrapped mean squared displacement after t steps is 1.5 t.
* Brute force on the 2 x 2 torus: exact transition probabilities.
* L = 1 keeps every agent in the single cell.
"""
import numpy as np
from scipy import stats

import oracle


def _wrapped_delta(a, b, L):
    d = (b.astype(np.int64) - a.astype(np.int64)) % L
    d[d > L // 2] -= L
    return d


def test_in_bounds_walk_1000_torus_prefix():
    p = oracle.Population("walk", 200_000, seed=1, L=1000)
    assert p.x.min() >= 0 and p.x.max() < 1000 and p.y.min() >= 0 and p.y.max() < 1000
    p.step(20)
    assert p.x.size == 200_000
    assert p.x.min() >= 0 and p.x.max() < 1000 and p.y.min() >= 0 and p.y.max() < 1000


def test_initial_positions_uniform():
    p = oracle.Population("walk", 100_000, seed=4, L=10)
    cnt = np.bincount(p.y * 10 + p.x, minlength=100)
    assert stats.chisquare(cnt).pvalue > 1e-4


def test_one_step_uniform_over_moore_neighbours():
    L = 1_000_003
    p = oracle.Population("walk", 64_000, seed=3, L=L)
    x0, y0 = p.x.copy(), p.y.copy()
    p.step(1)
    dx = _wrapped_delta(x0, p.x, L)
    dy = _wrapped_delta(y0, p.y, L)
    assert set(np.unique(dx)) <= {-1, 0, 1} and set(np.unique(dy)) <= {-1, 0, 1}
    assert not np.any((dx == 0) & (dy == 0))
    cls = (dy + 1) * 3 + (dx + 1)
    cnt = np.bincount(cls, minlength=9)
    assert cnt[4] == 0
    assert stats.chisquare(np.delete(cnt, 4)).pvalue > 1e-4


def test_mean_squared_displacement_closed_form():
    L = 1_000_003
    n, T = 20_000, 64
    p = oracle.Population("walk", n, seed=8, L=L)
    ux = np.zeros(n, dtype=np.int64)
    uy = np.zeros(n, dtype=np.int64)
    for _ in range(T):
        x0, y0 = p.x.copy(), p.y.copy()
        p.step(1)
        ux += _wrapped_delta(x0, p.x, L)
        uy += _wrapped_delta(y0, p.y, L)
    msd = float(np.mean(ux * ux + uy * uy))
    sem = float(np.std(ux * ux + uy * uy)) / np.sqrt(n)
    assert abs(msd - 1.5 * T) < 5 * sem
    assert abs(float(np.mean(ux))) < 5 * np.sqrt(0.75 * T / n)
    # the two axes are uncorrelated per step
    assert abs(float(np.mean(ux * uy))) < 5 * sem


def test_two_by_two_torus_transition():
    n = 40_000
    p = oracle.Population("walk", n, seed=2, L=2)
    p.x[:] = 0
    p.y[:] = 0
    p.step(1)
    cnt = np.bincount(p.y * 2 + p.x, minlength=4)
    # flip both: 4/8, flip y only: 2/8, flip x only: 2/8, stay: 0
    assert cnt[0] == 0
    exp = np.array([0.5, 0.25, 0.25]) * n  # cells (1,1), (0,1), (1,0)
    obs = np.array([cnt[3], cnt[2], cnt[1]])
    assert stats.chisquare(obs, exp).pvalue > 1e-4


def test_single_cell_grid():
    p = oracle.Population("walk", 100, seed=2, L=1)
    p.step(5)
    assert np.all(p.x == 0) and np.all(p.y == 0)


def test_seam_wraps():
    L = 7
    p = oracle.Population("walk", 4000, seed=6, L=L)
    p.x[:2000] = 0
    p.x[2000:] = L - 1
    p.y[:] = L - 1
    p.step(1)
    assert p.x.min() >= 0 and p.x.max() < L and p.y.min() >= 0 and p.y.max() < L
    assert np.any(p.x[:2000] == L - 1) and np.any(p.x[2000:] == 0) and np.any(p.y == 0)
