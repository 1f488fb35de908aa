"""The continuous-space models on the GPU (the paper's random walk and SIR as
stated in Sec. 5.1.2) against the oracle, bit for bit: float32 positions after
every kind of step (interior, clamped at the walls, a step wider than the box),
SIR states, days infected and per-step counts for the paper's setting (100 x 100
box, radius 5, p = 0.1, recovery after 14 steps, 5 initial infected; 500,
1,000 and 5,000 agents over 50 steps), moving agents, degenerate radii and
probabilities, columns written by the caller, invariants and curve statistics."""
import numpy as np
import pytest

import oracle
from paper_2601_16292_gb300 import amb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch.cuda.Stream()


def _same(gpu, orc, cols):
    for c in cols:
        assert np.array_equal(gpu.column(c).cpu().numpy(), getattr(orc, c)), c
    assert np.array_equal(gpu.counts(), orc.counts())


@pytest.mark.parametrize("n,w,h,s,seed", [(0, 10.0, 10.0, 1.0, 1), (1, 5.0, 5.0, 0.5, 2), (1000, 100.0, 100.0, 1.0, 3),
                                          (100_000, 37.5, 12.25, 0.75, 4), (3000, 4.0, 4.0, 50.0, 5),
                                          (2000, 0.0, 10.0, 1.0, 6)])
def test_walk_equals_oracle(stream, n, w, h, s, seed):
    g = amb.CPopulation("cwalk", n, seed=seed, rep=1, w=w, h=h, s=s, stream=stream)
    o = oracle.CPopulation("cwalk", n, seed=seed, rep=1, w=w, h=h, s=s)
    _same(g, o, ("x", "y"))
    for k in (1, 7, 22):
        g.step(k)
        o.step(k)
        _same(g, o, ("x", "y"))
    assert g.invariants()["ok"]
    g.close()


@pytest.mark.parametrize("n", [500, 1000, 5000])
def test_sir_paper_setting_equals_oracle(stream, n):
    kw = dict(w=100.0, h=100.0, s=0.0, r=5.0, p=0.1, rec_steps=14, n0=5)
    g = amb.CPopulation("csir", n, seed=7, stream=stream, **kw)
    o = oracle.CPopulation("csir", n, seed=7, **kw)
    for k in (1, 4, 45):
        g.step(k)
        o.step(k)
        _same(g, o, ("x", "y", "state", "days"))
    assert g.invariants()["ok"]
    st, _ = g.stats()
    pk, am, mean, var = oracle.curve_moments(o.counts()[:, 1])
    assert st["peak_infected"] == pk and st["peak_step"] == am
    assert abs(st["curve_mean"] - mean) <= 1e-12 * max(1.0, abs(mean))
    assert abs(st["curve_var"] - var) <= 1e-12 * max(1.0, abs(var))
    g.close()


@pytest.mark.parametrize("kw", [
    dict(n=3000, w=100.0, h=60.0, s=1.5, r=4.0, p=0.3, rec_steps=5, n0=30),   # moving agents
    dict(n=400, w=1.0, h=1.0, s=0.2, r=2.0, p=0.4, rec_steps=2, n0=3),        # everyone in contact (one cell)
    dict(n=2000, w=50.0, h=50.0, s=0.0, r=0.0, p=1.0, rec_steps=3, n0=50),   # radius 0: coincident agents only
    dict(n=2000, w=30.0, h=30.0, s=0.5, r=3.0, p=1.0, rec_steps=1, n0=10),   # certain infection, one-step illness
    dict(n=1500, w=30.0, h=30.0, s=0.5, r=3.0, p=0.0, rec_steps=9, n0=100),  # no transmission
    dict(n=0, w=10.0, h=10.0, s=1.0, r=1.0, p=0.5, rec_steps=4, n0=0),
    dict(n=20_000, w=200.0, h=200.0, s=0.5, r=5.0, p=0.05, rec_steps=14, n0=20),
])
def test_sir_cases_equal_oracle(stream, kw):
    g = amb.CPopulation("csir", seed=9, rep=3, stream=stream, **kw)
    o = oracle.CPopulation("csir", seed=9, rep=3, **kw)
    steps = 6 if kw["n"] > 10_000 else 25
    g.step(steps)
    o.step(steps)
    _same(g, o, ("x", "y", "state", "days"))
    assert g.invariants()["ok"]
    g.close()


def test_written_columns(stream):
    n = 300
    g = amb.CPopulation("csir", n, seed=2, w=20.0, h=20.0, s=0.0, r=3.0, p=0.5, rec_steps=6, n0=0, stream=stream)
    o = oracle.CPopulation("csir", n, seed=2, w=20.0, h=20.0, s=0.0, r=3.0, p=0.5, rec_steps=6, n0=0)
    rng = np.random.default_rng(1)
    o.x[:] = rng.uniform(0, 20, n).astype(np.float32)
    o.state[:] = rng.integers(0, 3, n).astype(np.uint8)
    o.days[:] = np.where(o.state == 1, rng.integers(0, 5, n), 0).astype(np.int32)
    g.write("x", o.x)
    g.write("state", o.state)
    g.write("days", o.days)
    g.step(10)
    o.step(10)
    _same(g, o, ("x", "y", "state", "days"))
    with pytest.raises(amb.AmbError):
        g.write("x", np.full(n, 20.5, dtype=np.float32))
    with pytest.raises(amb.AmbError):
        g.write("state", np.full(n, 3, dtype=np.uint8))
    g.close()


def test_bad_parameters_and_batches_refuse(stream):
    with pytest.raises(amb.AmbError):
        amb.CPopulation("csir", 10, seed=1, r=-1.0, stream=stream)
    with pytest.raises(amb.AmbError):
        amb.CPopulation("csir", 10, seed=1, rec_steps=0, stream=stream)
    with pytest.raises(amb.AmbError):
        amb.CPopulation("cwalk", 10, seed=1, w=float("nan"), stream=stream)
    with pytest.raises(amb.AmbError):
        amb.Batch([dict(model="csir", n=10, seed=1, steps=1)])
