"""The view API on the GPU (paper Sec. 3.1, 3.3) against the oracle, element by
element: full-population maps, filtered views (order-preserving compaction
across tiles with ragged tails), updates through views with repeated ids
(atomics and compare-and-swap for uint8), counter-based random ids, and the
wealth step written with views equal to the oracle's wealth rule and to the
fused wealth kernel."""
import numpy as np
import pytest

import oracle
from paper_2601_16292_gb300 import amb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# around the 16,384-row write tiles and the 32,768 / 65,536-row spans of `where`
SIZES = [0, 1, 5, 17, 4095, 4099, 16383, 16384, 16385, 32767, 32768, 32769, 3 * 16384 + 13, 65535, 65537,
         2 * 65536 + 1, (1 << 20) + 7]
RNG = np.random.default_rng(11)


@pytest.fixture(scope="module")
def stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch.cuda.Stream()


def _table(n, stream, cols):
    t = amb.Table(n, stream)
    for name, arr in cols.items():
        t.add_column(name, "i32" if arr.dtype == np.int32 else "u8")
        t.write(name, arr)
    return t


def _rand(dtype, n):
    info = np.iinfo(dtype)
    return RNG.integers(info.min, info.max, n, endpoint=True).astype(dtype)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
def test_map_all_ops(stream, n, dtype):
    col = _rand(dtype, n)
    t = _table(n, stream, {"c": col})
    want = col.copy()
    for op, s in [("add", 7), ("mul", -3), ("sub", 2 ** 31 + 5), ("min", 100), ("max", -7), ("add", 1 << 33), ("set", 42),
                  ("add", -1)]:
        t.map("c", op, s)
        oracle.col_map(want, op, s)
    assert np.array_equal(t.read("c").numpy(), want)
    t.close()


@pytest.mark.parametrize("dd,sd", [(np.int32, np.int32), (np.int32, np.uint8), (np.uint8, np.int32), (np.uint8, np.uint8)])
@pytest.mark.parametrize("op", ["set", "add", "sub", "mul", "min", "max"])
def test_map_col(stream, dd, sd, op):
    n = 5003
    d, s = _rand(dd, n), _rand(sd, n)
    t = _table(n, stream, {"d": d, "s": s})
    t.map_col("d", op, "s")
    assert np.array_equal(t.read("d").numpy(), oracle.col_map_col(d.copy(), op, s))
    t.close()


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
@pytest.mark.parametrize("cmp,s", [(">", 0), ("<=", 3), ("==", 2), ("!=", 2), ("<", -1), (">=", 1 << 40)])
def test_where(stream, n, dtype, cmp, s):
    col = RNG.integers(-3 if dtype == np.int32 else 0, 6, n).astype(dtype)
    t = _table(n, stream, {"c": col})
    with t.where("c", cmp, s) as v:
        assert np.array_equal(v.ids(), oracle.where(col, cmp, s))
    t.close()


def test_where_large_sparse_and_dense(stream):
    n = 10_000_000 + 3
    col = (RNG.random(n) < 0.001).astype(np.int32)
    t = _table(n, stream, {"c": col})
    for cmp in (">", "=="):
        with t.where("c", cmp, 0) as v:
            assert np.array_equal(v.ids(), oracle.where(col, cmp, 0))
    t.close()


def test_where_more_tiles_than_the_fast_count_scan(stream):
    # > 8,192 write tiles of 16,384 rows: the count scan of the last block
    # takes its loop form (more than 16 tiles per thread)
    n = (1 << 27) + (1 << 22) + 5
    col = RNG.integers(0, 3, n).astype(np.uint8)
    t = _table(n, stream, {"c": col})
    with t.where("c", "==", 1) as v:
        ids = v.ids()
        want = np.flatnonzero(col == 1)
        assert ids.size == want.size and np.array_equal(ids, want)
    t.close()


@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
@pytest.mark.parametrize("op,s", [("add", 3), ("sub", 5), ("mul", 3), ("min", 10), ("max", 200), ("set", 9)])
def test_updates_through_views(stream, dtype, op, s):
    n = 3000
    col = _rand(dtype, n)
    t = _table(n, stream, {"c": col})
    want = col.copy()
    # filtered view (unique ids)
    with t.where("c", ">", 50) as v:
        f_ids = v.ids()
        v.map("c", op, s)
    oracle.view_map(want, f_ids, op, s)
    # scatter view with many repeats
    ids = RNG.integers(0, 64, 20_000).astype(np.int32)
    with t.at(ids) as v:
        v.map("c", op, s)
    oracle.view_map(want, ids, op, s)
    # scatter view built on the device
    dev_ids = torch.from_numpy(RNG.integers(0, n, 5000).astype(np.int32)).cuda()
    torch.cuda.synchronize()
    with t.at(dev_ids) as v:
        v.scatter_add("c", 1)
    oracle.view_map(want, dev_ids.cpu().numpy(), "add", 1)
    assert np.array_equal(t.read("c").numpy(), want)
    t.close()


@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
@pytest.mark.parametrize("op,s", [("add", 3), ("mul", 3), ("set", 9), ("max", 200)])
def test_updates_through_views_large(stream, dtype, op, s):
    # a scatter list longer than one pass of the update kernels (a grid of
    # 152 x 16 blocks of 256 threads, 16 ids per thread: 9,961,472 ids)
    n = (1 << 20) + 5
    col = _rand(dtype, n)
    t = _table(n, stream, {"c": col})
    want = col.copy()
    with t.where("c", ">", 50) as v:
        f_ids = v.ids()
        v.map("c", op, s)
    oracle.view_map(want, f_ids, op, s)
    ids = RNG.integers(0, n, 12_000_001).astype(np.int32)
    with t.at(ids) as v:
        v.map("c", op, s)
    oracle.view_map(want, ids, op, s)
    assert np.array_equal(t.read("c").numpy(), want)
    t.close()


@pytest.mark.parametrize("word", [0, 1, 2, 3])
@pytest.mark.parametrize("exclude", [True, False])
def test_draw(stream, word, exclude):
    n = 70_001
    col = RNG.integers(0, 3, n).astype(np.int32)
    t = _table(n, stream, {"c": col})
    with t.where("c", "==", 1) as v, v.draw(17, 3, 41, word, n, exclude) as r:
        want = oracle.view_draw(v.ids(), 17, 3, 41, word, n, exclude)
        assert np.array_equal(r.ids(), want)
    t.close()


def test_wealth_by_views_equals_oracle_and_fused_kernel(stream):
    n, seed, steps = 10_000, 0, 100
    t = amb.Table(n, stream)
    t.add_column("wealth", "i32", fill=1)
    ref = oracle.Population("wealth", n, seed=seed)
    fused = amb.Population("wealth", n, seed=seed, stream=stream)
    for step in range(steps):
        with t.where("wealth", ">", 0) as donors:
            donors.map("wealth", "sub", 1)
            with donors.draw(seed, 0, step, 0, n, True) as recipients:
                recipients.scatter_add("wealth", 1)
    ref.step(steps)
    fused.step(steps)
    got = t.read("wealth").numpy()
    assert np.array_equal(got, ref.w)
    assert np.array_equal(got, fused.column("wealth").cpu().numpy())
    fused.close()
    t.close()


def test_errors(stream):
    t = amb.Table(10, stream)
    t.add_column("c", "u8", fill=3)
    with pytest.raises(amb.AmbError) as e:
        t.add_column("c", "i32")
    assert e.value.status == amb.AMB_EINVAL
    with pytest.raises(amb.AmbError) as e:
        t.at(np.array([1, 10], dtype=np.int32))
    assert e.value.status == amb.AMB_EINVAL
    with pytest.raises(amb.AmbError) as e:
        t.col("missing")
    assert e.value.status == amb.AMB_ENOTFOUND
    v = t.where("c", "==", 3)
    assert v.count() == 10
    with pytest.raises(amb.AmbError) as e:
        v.draw(1, 0, 0, 0, 1, True)
    assert e.value.status == amb.AMB_EINVAL
    # drawn ids address rows: the range is at most the table's n
    with pytest.raises(amb.AmbError) as e:
        v.draw(1, 0, 0, 0, 11, False)
    assert e.value.status == amb.AMB_EINVAL
    with v.draw(1, 0, 0, 0, 10, True) as r:
        assert r.count() == 10 and int(r.ids().max()) < 10
    with pytest.raises(amb.AmbError) as e:
        amb.lib()  # the table refuses to go while a view is alive
        amb._check(amb.lib().amb_table_destroy(t.handle))
    assert e.value.status == amb.AMB_EBUSY
    v.close()
    assert np.array_equal(t.read("c").numpy(), np.full(10, 3, dtype=np.uint8))
    t.close()
    empty = amb.Table(0, stream)
    empty.add_column("c", "i32")
    with empty.where("c", "==", 0) as v:
        assert v.count() == 0
        with v.where("c", ">", 0) as w:
            assert w.count() == 0
        with pytest.raises(amb.AmbError):  # no row to draw
            v.draw(1, 0, 0, 0, 1, False)
    empty.map("c", "add", 1)
    assert empty.read("c").numel() == 0
    empty.close()


@pytest.mark.parametrize("n", [0, 7, 4096, 4100, 3 * 4096 + 5, 300_001])
def test_view_of_view_and_conjunctions(stream, n):
    a = RNG.integers(0, 9, n).astype(np.int32)
    b = RNG.integers(0, 4, n).astype(np.uint8)
    t = _table(n, stream, {"a": a, "b": b})
    with t.where("a", ">", 3) as va, va.where("b", "==", 1) as vab:
        assert np.array_equal(vab.ids(), np.flatnonzero((a > 3) & (b == 1)))
    # over a scatter view: list order and repeats kept
    ids = RNG.integers(0, max(n, 1), 3 * n).astype(np.int32) if n else np.zeros(0, dtype=np.int32)
    with t.at(ids) as vs, vs.where("a", "<=", 2) as vsf:
        assert np.array_equal(vsf.ids(), oracle.view_where(a, ids, "<=", 2))
    t.close()


@pytest.mark.parametrize("dtype", [np.int32, np.uint8])
def test_scatter_add_values(stream, dtype):
    n = 5000
    col = _rand(dtype, n)
    t = _table(n, stream, {"c": col})
    ids = RNG.integers(0, 200, 30_000).astype(np.int32)
    vals = RNG.integers(-2 ** 31, 2 ** 31, 30_000).astype(np.int32)
    with t.at(ids) as v:
        v.scatter_add("c", torch.from_numpy(vals).cuda())
    want = oracle.view_add_values(col.copy(), ids, vals)
    assert np.array_equal(t.read("c").numpy(), want)
    # per-entry values through a filtered view whose length lives on the device
    with t.where("c", ">", 10) as f:
        k = f.count()
        fv = RNG.integers(0, 5, k).astype(np.int32)
        fids = f.ids()
        f.scatter_add("c", torch.from_numpy(fv).cuda())
    oracle.view_add_values(want, fids, fv)
    assert np.array_equal(t.read("c").numpy(), want)
    # too few values: reported, the table stays usable
    with t.at(np.arange(10, dtype=np.int32)) as v:
        v.scatter_add("c", torch.zeros(5, dtype=torch.int32).cuda())
        with pytest.raises(amb.AmbError):
            t.synchronize()
    t.synchronize()
    t.close()
