"""Pins for the oracle's counting-sort cell index and summary statistics.

* Index (grid environment, paper Sec. 4.1): start[C] = N, start is
  non-decreasing, start[c+1] - start[c] equals the brute-force occupancy of
  cell c, perm is a permutation whose entries in each cell's range sit in that
  cell, in ascending id order (stable).
* Gini: the rank formula against the exact mean-absolute-difference
  definition sum_ij |w_i - w_j| / (2 N sum w) in rationals, plus the closed
  forms (all equal -> 0; one agent holds everything -> (N-1)/N).
* Curve moments: against exact rational weighted mean / variance.
"""
from fractions import Fraction

import numpy as np

import oracle


def test_cell_index_properties():
    rng = np.random.default_rng(5)
    n, L = 5000, 30
    x = rng.integers(0, L, n).astype(np.int32)
    y = rng.integers(0, L, n).astype(np.int32)
    start, perm = oracle.cell_index(x, y, L)
    C = L * L
    assert start[0] == 0 and start[C] == n
    assert np.all(np.diff(start) >= 0)
    occ = np.zeros(C, dtype=np.int64)
    for i in range(n):
        occ[y[i] * L + x[i]] += 1
    assert np.array_equal(np.diff(start), occ)
    assert np.array_equal(np.sort(perm), np.arange(n))
    for c in range(C):
        ids = perm[start[c]:start[c + 1]]
        assert np.all(y[ids] * L + x[ids] == c)
        assert np.all(np.diff(ids) > 0)


def test_cell_index_empty_and_single_cell():
    start, perm = oracle.cell_index(np.zeros(0, np.int32), np.zeros(0, np.int32), 3)
    assert np.all(start == 0) and perm.size == 0
    start, perm = oracle.cell_index(np.zeros(4, np.int32), np.zeros(4, np.int32), 1)
    assert start.tolist() == [0, 4] and perm.tolist() == [0, 1, 2, 3]


def test_occupancy_histogram():
    rng = np.random.default_rng(6)
    n, L = 3000, 40
    x = rng.integers(0, L, n).astype(np.int32)
    y = rng.integers(0, L, n).astype(np.int32)
    occ, hist = oracle.occupancy(x, y, L, hist_len=32)
    assert occ.sum() == n
    assert np.array_equal(hist[:occ.max() + 1], np.bincount(occ, minlength=occ.max() + 1))
    assert hist.sum() == L * L


def _gini_exact(w):
    n = len(w)
    tot = sum(w)
    if tot == 0:
        return Fraction(0)
    s = sum(abs(a - b) for a in w for b in w)
    return Fraction(s, 2 * n * tot)


def test_gini_matches_mean_absolute_difference():
    rng = np.random.default_rng(7)
    for trial in range(20):
        n = int(rng.integers(1, 60))
        w = rng.integers(0, 25, n).astype(np.int32)
        g, num, tot = oracle.gini(w)
        ex = _gini_exact([int(v) for v in w])
        assert Fraction(num, n * tot if tot else 1) == (ex if tot else 0)
        assert abs(g - float(ex)) <= 1e-15 * max(1.0, abs(float(ex)))


def test_gini_closed_forms():
    g, _, _ = oracle.gini(np.full(100, 3, np.int32))
    assert g == 0.0
    w = np.zeros(50, np.int32)
    w[17] = 50
    g, _, _ = oracle.gini(w)
    assert abs(g - 49 / 50) < 1e-15
    g, _, _ = oracle.gini(np.zeros(10, np.int32))
    assert g == 0.0


def test_curve_moments_exact():
    rng = np.random.default_rng(8)
    I = rng.integers(0, 10_000, 300).astype(np.int64)
    I[123] = 20_000
    I[200] = 20_000
    pk, am, mean, var = oracle.curve_moments(I)
    assert pk == 20_000 and am == 124
    t = range(1, I.size + 1)
    s0 = sum(int(v) for v in I)
    m = Fraction(sum(ti * int(v) for ti, v in zip(t, I)), s0)
    v = sum((ti - m) ** 2 * int(iv) for ti, iv in zip(t, I)) / s0
    assert abs(mean - float(m)) <= 1e-13 * float(m)
    assert abs(var - float(v)) <= 1e-12 * float(v)
    assert oracle.curve_moments(np.zeros(5, np.int64)) == (0, 1, 0.0, 0.0)
