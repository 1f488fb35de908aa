"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element on the same seeded inputs.  Integer state must match bit for bit
(all columns at several steps, the per-step count series, the cell index
start array, occupancy); summary statistics within 1e-12 relative."""
import numpy as np
import pytest

import oracle
from oracle_jobs import canonical_ids
from paper_2601_16292_gb300 import amb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def host(t):
    return t.cpu().numpy()


def assert_columns(g, o, model):
    if model == "wealth":
        assert np.array_equal(host(g.column("wealth")), o.w)
    else:
        assert np.array_equal(host(g.column("x")), o.x)
        assert np.array_equal(host(g.column("y")), o.y)
        if model == "sir":
            assert np.array_equal(host(g.column("state")), o.state)


def run_pair(model, n, checkpoints, variant=0, **kw):
    g = amb.Population(model, n, variant=variant, **kw)
    o = oracle.Population(model, n, **kw)
    t = 0
    assert_columns(g, o, model)
    for cp in checkpoints:
        g.step(cp - t)
        o.step(cp - t)
        t = cp
        assert_columns(g, o, model)
    assert np.array_equal(g.counts(), o.counts())
    return g, o


def assert_index(g, o):
    start, ids = g.index()
    start, ids = host(start), host(ids)
    ostart, operm = oracle.cell_index(o.x, o.y, o.L)
    assert np.array_equal(start.astype(np.int64), ostart)
    # order inside a cell is free: compare each cell's id set
    assert np.array_equal(canonical_ids(start, ids), operm)


def assert_occupancy(g, o):
    occ = host(g.occupancy())
    oocc, ohist = oracle.occupancy(o.x, o.y, o.L, hist_len=int(occ.max()) + 1 if occ.size else 1)
    assert np.array_equal(occ, oocc)
    st, hist = g.stats()
    assert st["max_occupancy"] == int(oocc.max())
    assert np.array_equal(hist, ohist[: hist.size])


# ------------------------------------------------------------------ wealth --
def test_wealth_ten_thousand_agents_hundred_steps():
    g, o = run_pair("wealth", 10_000, [1, 2, 50, 100], seed=0)
    assert np.all(g.counts()[:, 1] == 10_000)
    st, hist = g.stats()
    gini, num, tot = oracle.gini(o.w)
    assert st["gini_numerator"] == num and st["total_wealth"] == tot
    assert abs(st["gini"] - gini) <= REL * abs(gini)
    assert np.array_equal(hist, np.bincount(o.w - o.w.min()))
    inv = g.invariants()
    assert inv["ok"] == 1
    g.close()


@pytest.mark.parametrize("n", [0, 1, 2, 3, 33, 1000, 4095, 4096, 4097, 20_001, 36864, 36865, 50_000])
def test_wealth_sizes(n):
    g, o = run_pair("wealth", n, [1, 7, 12], seed=5, rep=3, w_init=2)
    if n:
        st, _ = g.stats()
        gini, num, _ = oracle.gini(o.w)
        assert st["gini_numerator"] == num
        assert abs(st["gini"] - gini) <= REL * max(abs(gini), 1e-300)
    assert g.invariants()["ok"] == 1
    g.close()


@pytest.mark.parametrize("n", [777, 20_000, 60_000])
def test_wealth_written_column(n):
    rng = np.random.default_rng(11)
    w0 = rng.integers(0, 6, n).astype(np.int32)
    g = amb.Population("wealth", n, seed=9)
    o = oracle.Population("wealth", n, seed=9)
    g.write("wealth", torch.from_numpy(w0).cuda())
    o.w[:] = w0
    g.step(9)
    o.step(9)
    assert np.array_equal(host(g.column("wealth")), o.w)
    assert np.array_equal(g.counts(), o.counts())
    assert g.invariants()["ok"] == 1
    g.close()


# -------------------------------------------------------------------- walk --
def test_walk_million_agents_two_hundred_steps():
    g, o = run_pair("walk", 1_000_000, [1, 2, 200], seed=1, L=1000)
    assert_occupancy(g, o)
    assert g.invariants()["ok"] == 1
    g.close()


@pytest.mark.parametrize("n,L", [(0, 5), (1, 1), (7, 1), (1000, 2), (1001, 3), (4097, 64), (5000, 1_000_003)])
def test_walk_edges(n, L):
    g, o = run_pair("walk", n, [1, 3, 10], seed=4, rep=2, L=L)
    if L * L < 2 ** 31 and n:
        assert_index(g, o)
    g.close()


def test_walk_seams():
    n, L = 4000, 9
    x = np.where(np.arange(n) % 2 == 0, 0, L - 1).astype(np.int32)
    y = np.where(np.arange(n) % 3 == 0, 0, L - 1).astype(np.int32)
    g = amb.Population("walk", n, seed=6, L=L)
    o = oracle.Population("walk", n, seed=6, L=L)
    g.write("x", torch.from_numpy(x).cuda())
    g.write("y", torch.from_numpy(y))
    o.x[:] = x
    o.y[:] = y
    g.step(4)
    o.step(4)
    assert_columns(g, o, "walk")
    g.close()


# --------------------------------------------------------------------- SIR --
SIR_CASES = [
    dict(n=20_000, L=183, beta=0.3, gamma=0.05, n0=20),
    dict(n=5000, L=1, beta=0.01, gamma=0.1, n0=3),
    dict(n=12, L=2, beta=0.6, gamma=0.3, n0=2),
    dict(n=3000, L=40, beta=0.0, gamma=0.1, n0=300),
    dict(n=3000, L=40, beta=1.0, gamma=1.0, n0=30),
    dict(n=3000, L=20, beta=0.2, gamma=0.0, n0=0),
    dict(n=3000, L=20, beta=0.2, gamma=0.1, n0=3000),
    dict(n=0, L=7, beta=0.2, gamma=0.1, n0=0),
    dict(n=1, L=3, beta=0.2, gamma=0.1, n0=1),
    dict(n=2000, L=500, beta=0.9, gamma=0.01, n0=1000),
    dict(n=70_000, L=30, beta=0.002, gamma=0.01, n0=50),
]


@pytest.mark.parametrize("variant", [amb.AMB_SIR_GENERIC, amb.AMB_SIR_AUTO])
@pytest.mark.parametrize("case", SIR_CASES, ids=lambda c: "n%d-L%d-b%g-g%g" % (c["n"], c["L"], c["beta"], c["gamma"]))
def test_sir_cases(case, variant):
    g, o = run_pair("sir", case["n"], [1, 2, 9, 25], variant=variant, seed=2, rep=1, L=case["L"], beta=case["beta"],
                    gamma=case["gamma"], n0=case["n0"])
    if case["n"]:
        assert_index(g, o)
        assert_occupancy(g, o)
    st, _ = g.stats()
    pk, am, mean, var = oracle.curve_moments(o.counts()[:, 1])
    assert st["peak_infected"] == pk and st["peak_step"] == am
    assert abs(st["curve_mean"] - mean) <= REL * abs(mean)
    assert abs(st["curve_var"] - var) <= REL * abs(var)
    assert g.invariants()["ok"] == 1
    g.close()


@pytest.mark.parametrize("variant", [amb.AMB_SIR_GENERIC, amb.AMB_SIR_AUTO])
def test_sir_written_columns(variant):
    n, L = 6000, 50
    rng = np.random.default_rng(3)
    x = rng.integers(0, L, n).astype(np.int32)
    y = rng.integers(0, L, n).astype(np.int32)
    s = rng.choice(np.array([0, 1, 2], np.uint8), n, p=[0.8, 0.15, 0.05])
    g = amb.Population("sir", n, seed=8, L=L, beta=0.25, gamma=0.1, n0=10, variant=variant)
    o = oracle.Population("sir", n, seed=8, L=L, beta=0.25, gamma=0.1, n0=10)
    g.step(2)
    o.step(2)
    g.write("x", torch.from_numpy(x).cuda())
    g.write("y", y)
    g.write("state", torch.from_numpy(s).cuda())
    o.x[:], o.y[:], o.state[:] = x, y, s
    g.step(6)
    o.step(6)
    assert_columns(g, o, "sir")
    assert np.array_equal(g.counts(), o.counts())
    assert_index(g, o)
    g.close()


@pytest.mark.parametrize("n,L", [(24_000, 156), (25_000, 157), (300_000, 700), (600_000, 1000), (40, 900),
                                 (200_000, 64), (9_000, 32), (9_000, 33), (30_000, 1), (40_000, 2), (70_000, 2)])
def test_sir_band_geometries(n, L):
    """Single band (L*L fits one CTA), one-row bands, several-row bands with a
    short last band, nearly empty grids and dense cells, band path forced."""
    g, o = run_pair("sir", n, [1, 2, 7], variant=amb.AMB_SIR_BAND, seed=3, rep=5, L=L, beta=0.2, gamma=0.05,
                    n0=max(1, n // 100))
    assert_index(g, o)
    assert_occupancy(g, o)
    assert g.invariants()["ok"] == 1
    g.close()


def test_sir_band_dense_rows_use_wide_counters():
    """150,000 agents packed into two grid rows: the bands next to them see
    more than 65,535 source records and take the 32-bit counters, the others
    keep the packed 16-bit ones, in the same launch."""
    n, L = 200_000, 200
    rng = np.random.default_rng(21)
    y = np.where(np.arange(n) < 150_000, rng.integers(0, 2, n), rng.integers(0, L, n)).astype(np.int32)
    x = rng.integers(0, L, n).astype(np.int32)
    g = amb.Population("sir", n, seed=4, L=L, beta=0.05, gamma=0.02, n0=500, variant=amb.AMB_SIR_BAND)
    o = oracle.Population("sir", n, seed=4, L=L, beta=0.05, gamma=0.02, n0=500)
    g.write("x", x)
    g.write("y", y)
    o.x[:], o.y[:] = x, y
    for k in (1, 2, 3):
        g.step(k)
        o.step(k)
        assert_columns(g, o, "sir")
    assert np.array_equal(g.counts(), o.counts())
    assert_index(g, o)
    g.close()


# ---------------------------------------------- 16-bit band counters --
@pytest.mark.parametrize("n,L", [(9_000, 8), (30_000, 32), (24_000, 160), (300_000, 704), (1_000_000, 2048),
                                 (0, 16), (1, 8)])
def test_sir_band16_geometries(n, L):
    """16-bit shared counters forced: one band for the whole grid, one-row
    and several-row bands with a short last band, very dense cells (the
    8 x 8 grid holds 140 agents per cell: cells reach 16 infected agents and
    their bands are redone with 32-bit counters)."""
    g, o = run_pair("sir", n, [1, 2, 7], variant=amb.AMB_SIR_BAND16, seed=3, rep=5, L=L, beta=0.2, gamma=0.05,
                    n0=max(1, n // 100) if n else 0)
    assert_index(g, o)
    assert_occupancy(g, o)
    assert g.invariants()["ok"] == 1
    g.close()


@pytest.mark.parametrize("n,L", [
    (40_000, 64),   # ~10 agents per cell: cells with 16 or more infected agents
    (300_000, 64),  # ~4,700 agents per grid row: rows past the 12-bit offsets
    (20_000, 8),    # ~310 agents per cell: cells past 255 agents
])
def test_sir_band16_overflow_redoes_the_band(n, L):
    """Bands whose counts do not fit 16-bit counters are redone with 32-bit
    counters in the same step, and the trajectory stays the oracle's."""
    g, o = run_pair("sir", n, [1, 2, 5, 12], variant=amb.AMB_SIR_BAND16, seed=9, rep=2, L=L, beta=0.5,
                    gamma=0.05, n0=n // 20)
    assert_index(g, o)
    assert g.invariants()["ok"] == 1
    g.close()


def test_sir_band16_and_band32_agree_long_run():
    """The same population with 16-bit and with 32-bit band counters, 60
    steps: identical columns and count series, equal to the oracle."""
    kw = dict(seed=13, rep=0, L=2400, beta=0.3, gamma=0.02, n0=2000)
    n = 2_000_000
    a = amb.Population("sir", n, variant=amb.AMB_SIR_BAND16, **kw)
    b = amb.Population("sir", n, variant=amb.AMB_SIR_BAND32, **kw)
    a.step(60)
    b.step(60)
    for name in ("x", "y", "state"):
        assert torch.equal(a.column(name), b.column(name))
    assert np.array_equal(a.counts(), b.counts())
    o = oracle.Population("sir", n, **kw).step(60)
    assert_columns(a, o, "sir")
    assert np.array_equal(a.counts(), o.counts())
    a.close()
    b.close()


def test_sir_band_and_generic_agree_long_run():
    kw = dict(seed=12, rep=0, L=400, beta=0.1, gamma=0.03, n0=100)
    a = amb.Population("sir", 96_000, variant=amb.AMB_SIR_BAND, **kw)
    b = amb.Population("sir", 96_000, variant=amb.AMB_SIR_GENERIC, **kw)
    a.step(80)
    b.step(80)
    for name in ("x", "y", "state"):
        assert torch.equal(a.column(name), b.column(name))
    assert np.array_equal(a.counts(), b.counts())
    o = oracle.Population("sir", 96_000, **kw).step(80)
    assert_columns(a, o, "sir")
    a.close()
    b.close()


def test_sir_ten_million_agents_full_run_equals_oracle():
    """The 10M-agent SIR workload on the 4096 x 4096 torus (the benchmark's
    population and launch configuration) over its full 300 steps: every
    column, the cell index (start[] and each cell's ids) at t = 1, 2, 150 and
    300, and the whole count series equal the oracle.  The oracle (one host
    thread, a few tenths of a second per step) runs beside the GPU."""
    import queue
    import threading

    n, L, steps = 10_000_000, 4096, 300
    checkpoints = [1, 2, 150, 300]
    kw = dict(seed=2, L=L, beta=0.05, gamma=0.02, n0=10_000)
    snaps = queue.Queue()

    def run_oracle():
        try:
            o = oracle.Population("sir", n, **kw)
            t = 0
            for cp in checkpoints:
                o.step(cp - t)
                t = cp
                snaps.put((cp, o.x.copy(), o.y.copy(), o.state.copy()))
            snaps.put(("counts", o.counts()))
        except Exception as e:  # surfaced in the main thread
            snaps.put(("error", e))

    th = threading.Thread(target=run_oracle, daemon=True)
    th.start()
    g = amb.Population("sir", n, **kw)
    t = 0
    for cp in checkpoints:
        g.step(cp - t)
        t = cp
        gx, gy, gs = host(g.column("x")), host(g.column("y")), host(g.column("state"))
        start, ids = g.index()
        start, ids = host(start), host(ids)
        got = snaps.get(timeout=900)
        assert got[0] != "error", got[1]
        assert got[0] == cp
        _, ox, oy, os_ = got
        assert np.array_equal(gx, ox), cp
        assert np.array_equal(gy, oy), cp
        assert np.array_equal(gs, os_), cp
        ostart, operm = oracle.cell_index(ox, oy, L)
        assert np.array_equal(start.astype(np.int64), ostart), cp
        assert np.array_equal(canonical_ids(start, ids), operm), cp
    got = snaps.get(timeout=900)
    assert got[0] == "counts", got
    assert np.array_equal(g.counts(), got[1])
    assert g.invariants()["ok"] == 1
    th.join()
    g.close()


def test_sir_ten_million_agents_chunking():
    # the same 300 steps taken as one call and as calls of 1, 6, 93 and 200
    # steps give identical populations and count series (the oracle
    # comparison of the full run is the test above)
    n, L, steps = 10_000_000, 4096, 300
    kw = dict(seed=2, L=L, beta=0.05, gamma=0.02, n0=10_000)
    a = amb.Population("sir", n, **kw)
    b = amb.Population("sir", n, **kw)
    a.step(steps)
    for k in (1, 6, 93, 200):
        b.step(k)
    c = a.counts()
    assert c.shape == (steps, 4)
    assert np.all(c[:, :3].sum(axis=1) == n)
    assert np.all(np.diff(c[:, 2]) >= 0) and c[0, 2] >= 0
    s_prev = np.concatenate([[n - 10_000], c[:-1, 0]])
    assert np.all(c[:, 3] == s_prev - c[:, 0])  # every new infection leaves S
    assert np.array_equal(c, b.counts())
    for name in ("x", "y", "state"):
        assert torch.equal(a.column(name), b.column(name)), name
    assert a.invariants()["ok"] == 1
    a.close()
    b.close()


def test_write_column_rejects_out_of_range():
    g = amb.Population("sir", 100, seed=1, L=10, beta=0.1, gamma=0.1, n0=1)
    bad = np.zeros(100, np.uint8)
    bad[5] = 3
    with pytest.raises(amb.AmbError) as e:
        g.write("state", bad)
    assert e.value.status == amb.AMB_EINVAL
    bx = np.zeros(100, np.int32)
    bx[7] = 10
    with pytest.raises(amb.AmbError):
        g.write("x", bx)
    with pytest.raises(amb.AmbError):
        g.write("wealth", np.zeros(100, np.int32))
    with pytest.raises(amb.AmbError):
        g.write("x", np.zeros(99, np.int32))
    # still usable and unchanged
    o = oracle.Population("sir", 100, seed=1, L=10, beta=0.1, gamma=0.1, n0=1)
    g.step(3)
    o.step(3)
    assert_columns(g, o, "sir")
    g.close()


def test_create_rejects_bad_params():
    for kw in (dict(model="sir", n=10, seed=1, L=0), dict(model="sir", n=10, seed=1, L=10, beta=1.5),
               dict(model="sir", n=10, seed=1, L=10, n0=11), dict(model="walk", n=10, seed=2 ** 32, L=3),
               dict(model="sir", n=10, seed=1, L=50_000), dict(model="sir", n=10, seed=1, L=12, variant=5),
               dict(model="sir", n=10, seed=1, L=12, variant=amb.AMB_SIR_BAND16),
               dict(model="sir", n=10, seed=1, L=8200, variant=amb.AMB_SIR_BAND16)):
        model = kw.pop("model")
        with pytest.raises(amb.AmbError) as e:
            amb.Population(model, **kw)
        assert e.value.status == amb.AMB_EINVAL


# ------------------------------------------------------------ cell index --
@pytest.mark.parametrize("n,L", [(0, 4), (1, 1), (5000, 30), (100_003, 317), (2_000_000, 1500)])
def test_stateless_cell_index(n, L):
    rng = np.random.default_rng(n + L)
    x = rng.integers(0, L, n).astype(np.int32)
    y = rng.integers(0, L, n).astype(np.int32)
    start = torch.empty(L * L + 1, dtype=torch.int32, device="cuda")
    ids = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    amb.amb_cell_index(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), L, start, ids[:n] if n else ids[:0])
    ostart, operm = oracle.cell_index(x, y, L)
    assert np.array_equal(host(start).astype(np.int64), ostart)
    got = host(ids)[:n].copy()
    for c in np.nonzero(np.diff(ostart) > 1)[0]:
        a, b = ostart[c], ostart[c + 1]
        got[a:b] = np.sort(got[a:b])
    assert np.array_equal(got, operm)


def test_stateless_cell_index_reports_out_of_range():
    L = 8
    x = torch.tensor([0, 3, 8, 2], dtype=torch.int32, device="cuda")
    y = torch.tensor([0, 1, 2, -1], dtype=torch.int32, device="cuda")
    start = torch.empty(L * L + 1, dtype=torch.int32, device="cuda")
    ids = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(amb.AmbError) as e:
        amb.amb_cell_index(x, y, L, start, ids)
    assert e.value.status == amb.AMB_EINVAL
    assert int(start[-1]) == 2


@pytest.mark.parametrize("n", [5_000, 30_000])
def test_wealth_wraps_like_the_oracle(n):
    # wealth arithmetic wraps modulo 2^32 on both sides (agents at the int32
    # maximum that receive a unit turn negative and stop donating)
    rng = np.random.default_rng(23)
    w0 = rng.integers(0, 4, n).astype(np.int32)
    w0[rng.choice(n, 50, replace=False)] = np.iinfo(np.int32).max
    g = amb.Population("wealth", n, seed=4)
    o = oracle.Population("wealth", n, seed=4)
    g.write("wealth", torch.from_numpy(w0).cuda())
    o.w[:] = w0
    g.step(12)
    o.step(12)
    assert np.array_equal(host(g.column("wealth")), o.w)
    assert np.array_equal(g.counts(), o.counts())
    g.close()
