"""Buffered per-agent writes and d-dimensional grid walks on the GPU against
the oracle: last-write-wins merges over interleaved columns, host and device
records, repeated flushes, capacity and id errors; grid walks for every
dimension, neighbourhood and boundary mode, tiny and ragged sizes, fused steps,
and the 2-D Moore torus case against the population walk."""
import numpy as np
import pytest

import oracle
from paper_2601_16292_gb300 import amb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
RNG = np.random.default_rng(21)


@pytest.fixture(scope="module")
def stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch.cuda.Stream()


def test_log_last_write_wins(stream):
    n = 5000
    t = amb.Table(n, stream)
    t.add_column("a", "i32", fill=7)
    t.add_column("b", "u8", fill=1)
    want = {"a": np.full(n, 7, dtype=np.int32), "b": np.full(n, 1, dtype=np.uint8)}
    log = t.log(100_000)
    for rnd in range(3):
        recs = []
        for j in range(6):
            name = "a" if j % 2 == 0 else "b"
            ids = RNG.integers(0, 300 if j < 3 else n, 4000).astype(np.int32)  # many repeats
            vals = RNG.integers(-2 ** 40, 2 ** 40, 4000).astype(np.int64)
            if j == 5:
                log.record(name, torch.from_numpy(ids).cuda(), torch.from_numpy(vals).cuda())
            else:
                log.record(name, ids, vals)
            recs.append((name, ids, vals))
        assert log.pending() == 6 * 4000
        log.flush()
        assert log.pending() == 0
        for name, ids, vals in recs:
            oracle.log_flush(want[name], ids, vals)
        assert np.array_equal(t.read("a").numpy(), want["a"]), rnd
        assert np.array_equal(t.read("b").numpy(), want["b"]), rnd
    # errors: capacity, ids out of range (host and device); the table stays usable
    small = t.log(10)
    with pytest.raises(amb.AmbError):
        small.record("a", np.arange(11), np.zeros(11))
    with pytest.raises(amb.AmbError):
        small.record("a", np.array([n]), np.zeros(1))
    with pytest.raises(amb.AmbError):
        small.record("a", torch.tensor([0, n], dtype=torch.int32).cuda(), torch.zeros(2, dtype=torch.int64).cuda())
    assert small.pending() == 0
    small.record("a", np.array([3, 3]), np.array([1, 2]))
    small.flush()
    want["a"][3] = 2
    assert np.array_equal(t.read("a").numpy(), want["a"])
    small.close()
    log.close()
    t.close()


def test_log_record_numbers_restart(stream):
    # flushes numbered near 2^31 - 1: the log restarts its numbers from 0 with
    # the winner words cleared, and a stale winner word never matches
    n = 3000
    t = amb.Table(n, stream)
    t.add_column("a", "i32", fill=0)
    want = np.zeros(n, dtype=np.int32)
    log = t.log(10_000)
    ids = RNG.integers(0, 200, 5000).astype(np.int32)
    vals = RNG.integers(-100, 100, 5000).astype(np.int64)
    log.debug_base((1 << 31) - 6000)  # this flush fits below 2^31 - 1
    log.record("a", ids, vals)
    log.flush()
    oracle.log_flush(want, ids, vals)
    assert np.array_equal(t.read("a").numpy(), want)
    # the next one would pass it: restart
    ids2 = RNG.integers(0, 200, 5000).astype(np.int32)
    vals2 = RNG.integers(-100, 100, 5000).astype(np.int64)
    log.record("a", ids2, vals2)
    log.flush()
    oracle.log_flush(want, ids2, vals2)
    assert np.array_equal(t.read("a").numpy(), want)
    # rows written before the restart and not after keep their values; a few
    # records on fresh numbers
    log.record("a", np.array([7, 7, 9], dtype=np.int32), np.array([1, 2, 3], dtype=np.int64))
    log.flush()
    want[7], want[9] = 2, 3
    assert np.array_equal(t.read("a").numpy(), want)
    with pytest.raises(amb.AmbError):
        log.debug_base(1 << 31)
    log.close()
    t.close()


CASES = [(1, False, True, [7]), (1, True, False, [2]), (2, True, True, [33, 17]), (2, False, False, [5, 9]),
         (2, True, False, [1, 40]), (3, True, True, [6, 5, 4]), (3, False, False, [3, 3, 3]),
         (3, True, False, [2, 2, 2]), (4, True, True, [3, 4, 5, 6]), (4, False, False, [2, 3, 1, 4]),
         (4, True, False, [9, 9, 9, 9])]


@pytest.mark.parametrize("d,moore,torus,sizes", CASES)
def test_grid_walk_equals_oracle(stream, d, moore, torus, sizes):
    n = 10_007
    names = ["c%d" % q for q in range(d)]
    coords = [RNG.integers(0, s, n).astype(np.int32) for s in sizes]
    t = amb.Table(n, stream)
    for name, c in zip(names, coords):
        t.add_column(name, "i32")
        t.write(name, c)
    want = [c.copy() for c in coords]
    step = 0
    for k in (1, 3, 8):
        t.grid_walk(names, sizes, moore, torus, seed=13, rep=2, step=step, steps=k)
        for j in range(k):
            oracle.grid_walk_step(want, sizes, moore, torus, 13, 2, step + j)
        step += k
        for name, w in zip(names, want):
            assert np.array_equal(t.read(name).numpy(), w), (name, k)
    t.close()


def test_two_dim_moore_torus_equals_population_walk(stream):
    n, L = 4000, 57
    p = amb.Population("walk", n, seed=8, rep=1, L=L, stream=stream)
    t = amb.Table(n, stream)
    t.add_column("x", "i32")
    t.add_column("y", "i32")
    t.write("x", p.column("x"))
    t.write("y", p.column("y"))
    t.grid_walk(["x", "y"], [L, L], True, True, seed=8, rep=1, step=0, steps=25)
    p.step(25)
    assert torch.equal(t.read("x", device="cuda"), p.column("x"))
    assert torch.equal(t.read("y", device="cuda"), p.column("y"))
    # coordinates outside the box are reported, and the table stays usable
    t.write("x", np.full(n, L, dtype=np.int32))
    t.grid_walk(["x", "y"], [L, L], True, True, seed=8, step=30)
    with pytest.raises(amb.AmbError):
        t.synchronize()
    t.synchronize()
    p.close()
    t.close()
