"""Pins of the oracle's view primitives (paper Sec. 3.1 / 3.3): full-population
maps, filtered views and scatter views against numpy's own routines (wrapping
integer arithmetic, flatnonzero, ufunc.at), the random-id draw against its
range and exclusion rules and a chi-square test, and the wealth step written
with views against the oracle's wealth rule (pinned by exact enumeration)."""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(7)
NP_OPS = {"add": np.add, "sub": np.subtract, "mul": np.multiply, "min": np.minimum, "max": np.maximum}


def _as(dtype, s):
    """The scalar reduced to the column's type by two's-complement truncation."""
    return np.array([s], dtype=np.int64).astype(dtype)[0]


@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
@pytest.mark.parametrize("op", ["set", "add", "sub", "mul", "min", "max"])
@pytest.mark.parametrize("s", [0, 1, -1, 7, 255, 256, -300, 2 ** 31 - 1, -2 ** 31, 2 ** 33 + 5])
def test_col_map_matches_numpy(dtype, op, s):
    info = np.iinfo(dtype)
    col = RNG.integers(info.min, info.max, 257, endpoint=True).astype(dtype)
    want = np.full_like(col, _as(dtype, s)) if op == "set" else NP_OPS[op](col, _as(dtype, s), dtype=dtype)
    got = oracle.col_map(col.copy(), op, s)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("op", ["set", "add", "sub", "mul", "min", "max"])
def test_col_map_col_matches_numpy(op):
    a = RNG.integers(-2 ** 31, 2 ** 31, 300).astype(np.int32)
    b = RNG.integers(-2 ** 31, 2 ** 31, 300).astype(np.int32)
    u = RNG.integers(0, 256, 300).astype(np.uint8)
    want = b.copy() if op == "set" else NP_OPS[op](a, b, dtype=np.int32)
    assert np.array_equal(oracle.col_map_col(a.copy(), op, b), want)
    # a uint8 source is taken as its (non-negative) value
    want = u.astype(np.int32) if op == "set" else NP_OPS[op](a, u.astype(np.int32), dtype=np.int32)
    assert np.array_equal(oracle.col_map_col(a.copy(), op, u), want)


@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
@pytest.mark.parametrize("cmp", ["==", "!=", "<", "<=", ">", ">="])
@pytest.mark.parametrize("s", [0, 3, -1, 200, 2 ** 40, -2 ** 40])
def test_where_matches_flatnonzero(dtype, cmp, s):
    col = RNG.integers(-5 if dtype == np.int32 else 0, 8, 1000).astype(dtype)
    v = col.astype(np.int64)
    pred = {"==": v == s, "!=": v != s, "<": v < s, "<=": v <= s, ">": v > s, ">=": v >= s}[cmp]
    assert np.array_equal(oracle.where(col, cmp, s), np.flatnonzero(pred))


def test_where_empty_and_full():
    col = np.zeros(10, dtype=np.int32)
    assert oracle.where(col, ">", 0).size == 0
    assert np.array_equal(oracle.where(col, "==", 0), np.arange(10))
    assert oracle.where(np.zeros(0, dtype=np.int32), ">", 0).size == 0


@pytest.mark.parametrize("op", ["add", "sub", "mul", "min", "max"])
def test_view_map_repeats_match_ufunc_at(op):
    col = RNG.integers(-50, 50, 64).astype(np.int32)
    ids = RNG.integers(0, 64, 500).astype(np.int32)  # many repeats
    want = col.copy()
    NP_OPS[op].at(want, ids, np.int32(3))
    assert np.array_equal(oracle.view_map(col.copy(), ids, op, 3), want)


def test_view_map_set_and_bounds():
    col = np.zeros(8, dtype=np.uint8)
    oracle.view_map(col, np.array([1, 1, 5]), "set", 9)
    assert list(col) == [0, 9, 0, 0, 0, 9, 0, 0]
    with pytest.raises(RuntimeError):
        oracle.view_map(col, np.array([8]), "add", 1)


def test_draw_range_exclusion_and_uniformity():
    n = 7
    ids = np.repeat(np.arange(n, dtype=np.int32), 3000)
    for step in (0, 1, 99):
        r = oracle.view_draw(ids, 5, 2, step, 0, n, True)
        assert np.all((r >= 0) & (r < n)) and np.all(r != ids)
    # agent 3's recipient over many steps: uniform over the 6 others
    r = np.concatenate([oracle.view_draw(np.array([3], dtype=np.int32), 5, 2, t, 0, n, True) for t in range(6000)])
    counts = np.bincount(r, minlength=n)
    assert counts[3] == 0
    exp = 6000 / 6
    chi2 = float(((counts[np.arange(n) != 3] - exp) ** 2 / exp).sum())
    assert chi2 < 20.5  # 5 dof, p ~ 0.001
    # without exclusion every id in range may come up, the agent itself included
    r = oracle.view_draw(np.zeros(5000, dtype=np.int32), 1, 0, 0, 2, 4, False)
    assert set(np.unique(r)) <= {0, 1, 2, 3}
    with pytest.raises(RuntimeError):
        oracle.view_draw(np.zeros(1, dtype=np.int32), 1, 0, 0, 0, 1, True)


def _wealth_step_by_views(w, seed, rep, t):
    """The paper's wealth rule written with the view API (Sec. 3.1): donors =
    where(wealth > 0); donors.wealth -= 1; one random other agent per donor;
    scatter_add(wealth=1) over the recipients."""
    n = w.size
    if n < 2:
        return w
    donors = oracle.where(w, ">", 0)
    oracle.view_map(w, donors, "sub", 1)
    recipients = oracle.view_draw(donors, seed, rep, t, 0, n, True)
    oracle.view_map(w, recipients, "add", 1)
    return w


@pytest.mark.parametrize("n,seed,rep,w_init", [(2, 0, 0, 1), (3, 1, 0, 2), (50, 9, 4, 1), (1000, 0, 0, 1),
                                               (777, 123, 5, 3)])
def test_wealth_by_views_equals_wealth_rule(n, seed, rep, w_init):
    ref = oracle.Population("wealth", n, seed=seed, rep=rep, w_init=w_init)
    w = ref.w.copy()
    for t in range(30):
        _wealth_step_by_views(w, seed, rep, t)
        ref.step(1)
        assert np.array_equal(w, ref.w), t


@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
def test_view_where_is_boolean_indexing(dtype):
    col = RNG.integers(0, 9, 500).astype(dtype)
    ids = RNG.integers(0, 500, 2000).astype(np.int32)  # a scatter view with repeats
    for cmp, s in [(">", 4), ("==", 3), ("!=", 0), ("<=", 2)]:
        v = col[ids].astype(np.int64)
        pred = {">": v > s, "==": v == s, "!=": v != s, "<=": v <= s}[cmp]
        assert np.array_equal(oracle.view_where(col, ids, cmp, s), ids[pred])
    # where(A).where(B) == where(A and B)
    other = RNG.integers(0, 5, 500).astype(np.int32)
    a = oracle.where(col, ">", 2)
    ab = oracle.view_where(other, a, "==", 1)
    assert np.array_equal(ab, np.flatnonzero((col.astype(np.int64) > 2) & (other == 1)))


@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
def test_view_add_values_is_add_at(dtype):
    col = RNG.integers(0, 100, 64).astype(dtype)
    ids = RNG.integers(0, 64, 700).astype(np.int32)
    vals = RNG.integers(-1000, 1000, 700).astype(np.int32)
    want = col.copy()
    np.add.at(want, ids, vals.astype(dtype))
    assert np.array_equal(oracle.view_add_values(col.copy(), ids, vals), want)
