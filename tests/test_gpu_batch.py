"""Batched runs (many jobs per launch, one CUDA graph) against the oracle:
every job's columns and per-step counts must equal a lone run of the same job,
whatever the batching options (graph or not, band-height cap, autotuner)."""
import numpy as np
import pytest

import oracle
from paper_2601_16292_gb300 import amb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

JOBS = [
    dict(model="sir", n=20_000, L=183, beta=0.3, gamma=0.05, n0=20, seed=2, rep=1, steps=9),
    dict(model="sir", n=70_000, L=30, beta=0.002, gamma=0.01, n0=50, seed=3, rep=0, steps=6),
    dict(model="sir", n=500, L=29, beta=0.5, gamma=0.1, n0=5, seed=4, rep=2, steps=11),
    dict(model="sir", n=3000, L=40, beta=0.2, gamma=0.1, n0=30, seed=5, rep=3, steps=0),
    dict(model="wealth", n=5000, seed=6, steps=8),
    dict(model="wealth", n=60_000, seed=7, rep=1, steps=5, w_init=2),
    dict(model="walk", n=10_000, L=100, seed=8, steps=13),
    dict(model="sir", n=600_000, L=1000, beta=0.05, gamma=0.02, n0=600, seed=9, steps=4),
    dict(model="sir", n=1, L=3, beta=0.2, gamma=0.1, n0=1, seed=10, steps=3),
    dict(model="wealth", n=0, seed=11, steps=4),
]


@pytest.fixture(scope="module")
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def expected(_cuda):
    out = []
    for j in JOBS:
        kw = {k: v for k, v in j.items() if k not in ("model", "steps")}
        o = oracle.Population(j["model"], **kw).step(j["steps"])
        out.append(o)
    return out


def _check_batch(b, expected):
    for i, (j, o) in enumerate(zip(JOBS, expected)):
        v = b.population(i)
        assert v.t == j["steps"]
        if j["model"] == "wealth":
            assert np.array_equal(v.column("wealth").cpu().numpy(), o.w), i
        else:
            assert np.array_equal(v.column("x").cpu().numpy(), o.x), i
            assert np.array_equal(v.column("y").cpu().numpy(), o.y), i
            if j["model"] == "sir":
                assert np.array_equal(v.column("state").cpu().numpy(), o.state), i
        assert np.array_equal(v.counts(), o.counts()), i


@pytest.mark.parametrize("opts", [dict(), dict(use_graph=False), dict(band_rows_cap=4), dict(autotune=True)],
                         ids=["graph", "direct", "cap4", "autotune"])
def test_batch_equals_oracle(expected, opts):
    stream = torch.cuda.Stream()
    b = amb.Batch(JOBS, stream=stream)
    ms = b.run(**opts)
    assert ms > 0
    info = b.info()
    assert info["n_jobs"] == len(JOBS)
    assert info["agent_steps"] == sum(j["n"] * j["steps"] for j in JOBS)
    if opts.get("band_rows_cap"):
        assert info["band_rows_cap"] == opts["band_rows_cap"]
    _check_batch(b, expected)
    # the populations step on alone after the batch
    v = b.population(0)
    v.step(2)
    j = JOBS[0]
    kw = {k: val for k, val in j.items() if k not in ("model", "steps")}
    o = oracle.Population("sir", **kw).step(j["steps"] + 2)
    assert np.array_equal(v.column("state").cpu().numpy(), o.state)
    b.close()


def test_batch_runs_once():
    stream = torch.cuda.Stream()
    b = amb.Batch(JOBS[:2], stream=stream)
    b.run()
    with pytest.raises(amb.AmbError):
        b.run()
    b.close()


def test_batch_is_three_persistent_launches(expected):
    # the whole run (every job, every step) is three kernel launches: one for
    # the SIR jobs, one for the small wealth jobs, one for the large wealth
    # and walk jobs
    stream = torch.cuda.Stream()
    b = amb.Batch(JOBS, stream=stream)
    b.run()
    assert b.info()["launches"] == 3
    _check_batch(b, expected)
    b.close()


def test_many_uneven_jobs_equal_lone_runs(_cuda):
    # 60 jobs of every kind with uneven sizes and step counts share one
    # persistent launch (steps of different jobs interleave in its queue);
    # each equals the same job stepped alone
    rng = np.random.default_rng(17)
    jobs = []
    for i in range(60):
        kind = ("sir", "wealth", "walk")[i % 3]
        n = int(rng.integers(0, 90_000)) if i % 7 else int(rng.integers(0, 40))
        steps = int(rng.integers(0, 40))
        if kind == "sir":
            L = max(1, int(rng.integers(1, 400)))
            jobs.append(dict(model="sir", n=n, L=L, beta=float(rng.uniform(0, 0.4)), gamma=float(rng.uniform(0, 0.2)),
                             n0=min(n, int(rng.integers(0, 50))), seed=100 + i, rep=i, steps=steps))
        elif kind == "wealth":
            jobs.append(dict(model="wealth", n=n, seed=100 + i, rep=i, steps=steps, w_init=int(rng.integers(0, 3))))
        else:
            jobs.append(dict(model="walk", n=n, L=max(1, int(rng.integers(1, 300))), seed=100 + i, rep=i, steps=steps))
    stream = torch.cuda.Stream()
    b = amb.Batch(jobs, stream=stream)
    b.run()
    assert b.info()["launches"] <= 3
    for i, j in enumerate(jobs):
        kw = {k: v for k, v in j.items() if k not in ("model", "steps")}
        alone = amb.Population(j["model"], stream=stream, **kw).step(j["steps"])
        v = b.population(i)
        assert v.t == j["steps"]
        assert np.array_equal(v.counts(), alone.counts()), (i, j)
        cols = ("wealth",) if j["model"] == "wealth" else (("x", "y", "state") if j["model"] == "sir" else ("x", "y"))
        for c in cols:
            assert torch.equal(v.column(c), alone.column(c)), (i, j, c)
        alone.close()
    b.close()
