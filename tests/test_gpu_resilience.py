"""Checkpoint / resume and bounded waits on the GPU.

Resume: the state is integer (or float32) columns plus the step index and the
random draws are keyed by (seed, replicate, id, step), so a population read
after t steps, written into a fresh population with the same key and set to
step t continues bit-identically (every model and SIR path).
Bounded waits: a look-back wait on a predecessor that never publishes gives up
after its limit, reports AMB_ETIMEOUT, and the device keeps working."""
import numpy as np
import pytest

from paper_2601_16292_gb300 import amb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    ("wealth", dict(n=5000), ("wealth",)),
    ("wealth", dict(n=70_000, w_init=2), ("wealth",)),
    ("walk", dict(n=20_000, L=300), ("x", "y")),
    ("sir", dict(n=60_000, L=320, beta=0.2, gamma=0.03, n0=60), ("x", "y", "state")),
    ("sir", dict(n=30_000, L=200, beta=0.3, gamma=0.05, n0=30, variant=amb.AMB_SIR_GENERIC), ("x", "y", "state")),
    ("cwalk", dict(n=10_000, w=50.0, h=40.0, s=1.0), ("x", "y")),
    ("csir", dict(n=3000, w=60.0, h=60.0, s=0.5, r=3.0, p=0.2, rec_steps=7, n0=10), ("x", "y", "state", "days")),
]


@pytest.fixture(scope="module")
def stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch.cuda.Stream()


def _make(model, kw, stream):
    if model in ("cwalk", "csir"):
        return amb.CPopulation(model, seed=5, rep=2, stream=stream, **kw)
    return amb.Population(model, seed=5, rep=2, stream=stream, **kw)


@pytest.mark.parametrize("model,kw,cols", CASES, ids=[c[0] + "-" + str(i) for i, c in enumerate(CASES)])
def test_resume_is_bit_identical(stream, model, kw, cols):
    t1, t2 = 17, 23
    a = _make(model, kw, stream)
    a.step(t1)
    saved = {c: a.column(c) for c in cols}
    b = _make(model, kw, stream)
    for c in cols:
        b.write(c, saved[c])
    b.set_step(t1)
    assert b.t == t1
    a.step(t2)
    b.step(t2)
    for c in cols:
        assert torch.equal(a.column(c), b.column(c)), c
    ca, cb = a.counts(), b.counts()
    assert np.array_equal(ca[t1:], cb[t1:])
    assert np.all(cb[:t1] == 0)
    assert b.invariants()["ok"]
    a.close()
    b.close()


def test_bounded_wait_times_out_and_device_stays_usable(stream):
    import ctypes
    waited = ctypes.c_double()
    rc = amb.lib().amb_selfcheck_wait_timeout(amb._stream_handle(stream), ctypes.byref(waited))
    assert rc == amb.AMB_ETIMEOUT
    assert 1.5 < waited.value < 30.0
    p = amb.Population("sir", 5000, seed=1, L=90, beta=0.2, gamma=0.05, n0=5, stream=stream)
    p.step(5)
    assert p.invariants()["ok"]
    p.close()


def test_written_columns_read_back_and_step_once_rebuilt(stream):
    """Band path: several column writes are staged and the records rebuilt
    once; reads see the written values, and stepping equals a population
    given the same columns by one rebuild per write (the earlier behaviour is
    equivalent to rebuilding after every write)."""
    n, L = 20_000, 150
    rng = np.random.default_rng(4)
    x = rng.integers(0, L, n).astype(np.int32)
    y = rng.integers(0, L, n).astype(np.int32)
    s = rng.integers(0, 3, n).astype(np.uint8)
    a = amb.Population("sir", n, seed=3, L=L, beta=0.3, gamma=0.05, n0=10, stream=stream)
    a.write("x", x)
    a.write("y", y)
    a.write("state", s)
    assert np.array_equal(a.column("x").cpu().numpy(), x)
    assert np.array_equal(a.column("state").cpu().numpy(), s)
    b = amb.Population("sir", n, seed=3, L=L, beta=0.3, gamma=0.05, n0=10, stream=stream)
    b.write("x", x)
    b.column("x")  # forces a rebuild between the writes
    b.write("y", y)
    b.column("y")
    b.write("state", s)
    a.step(12)
    b.step(12)
    for c in ("x", "y", "state"):
        assert torch.equal(a.column(c), b.column(c)), c
    assert np.array_equal(a.counts(), b.counts())
    a.close()
    b.close()


def test_async_counts_equal_counts(stream):
    p = amb.Population("sir", 50_000, seed=9, L=290, beta=0.2, gamma=0.05, n0=50, stream=stream)
    rows = torch.zeros((20, 4), dtype=torch.int64, pin_memory=True)
    for k in range(20):
        p.step(1)
        amb.amb_counts_async(p.handle, k, 1, rows[k])
    p.synchronize()
    assert np.array_equal(rows.numpy(), p.counts())
    with pytest.raises(amb.AmbError):
        amb.amb_counts_async(p.handle, 20, 1, rows[0])
    p.close()


@pytest.mark.parametrize("model", ["sir", "walk", "wealth"])
def test_async_counts_across_series_growth_resume_and_destroy(stream, model):
    # copies still queued when the count series is reallocated (it grows past
    # 64 and 128 rows), when the step counter is moved back, and at destroy;
    # a twin population run the same way gives the expected rows
    kw = dict(L=120) if model != "wealth" else {}
    if model == "sir":
        kw.update(beta=0.3, gamma=0.05, n0=20)
    p = amb.Population(model, 8_000, seed=4, stream=stream, **kw)
    q = amb.Population(model, 8_000, seed=4, stream=stream, **kw)
    steps = 200
    rows = torch.zeros((steps, 4), dtype=torch.int64, pin_memory=True)
    for k in range(steps):
        p.step(1)
        amb.amb_counts_async(p.handle, k, 1, rows[k])
    q.step(steps)
    want = q.counts()
    tail = torch.zeros((10, 4), dtype=torch.int64, pin_memory=True)
    amb.amb_counts_async(p.handle, steps - 10, 10, tail)
    p.set_step(150)  # synchronises: the queued copies finish before rows are rewritten
    assert np.array_equal(rows.numpy(), want)
    assert np.array_equal(tail.numpy(), want[-10:])
    q.set_step(150)
    p.step(1)
    q.step(1)
    last = torch.zeros((1, 4), dtype=torch.int64, pin_memory=True)
    amb.amb_counts_async(p.handle, 150, 1, last)
    p.close()  # destroy with the copy queued: it completes first
    assert np.array_equal(last.numpy(), q.counts()[150:151])
    q.close()
