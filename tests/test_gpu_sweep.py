"""The parameter sweep (1,024 wealth and SIR replicates of uneven size, 200
steps each) advanced as one batch: a stratified sample of the jobs equals the
oracle bit for bit, every job keeps the models' invariants in its per-step
counts, and the largest jobs equal a lone run of the same job."""
import numpy as np
import pytest

import oracle
from paper_2601_16292_gb300 import amb, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sweep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    jobs = workloads.sweep_jobs()
    stream = torch.cuda.Stream()
    b = amb.Batch(jobs, stream=stream)
    b.run(autotune=True)
    yield jobs, b, stream
    b.close()


def _sample(jobs, per_model=5, max_n=120_000):
    """Smallest, largest (up to max_n) and evenly spaced sizes of each model."""
    out = []
    for model in ("wealth", "sir"):
        idx = sorted((i for i, j in enumerate(jobs) if j["model"] == model and j["n"] <= max_n),
                     key=lambda i: jobs[i]["n"])
        pick = np.linspace(0, len(idx) - 1, per_model).round().astype(int)
        out += [idx[p] for p in pick]
    return out


def test_sweep_sample_equals_oracle(sweep):
    jobs, b, _ = sweep
    for i in _sample(jobs):
        j = jobs[i]
        kw = {k: v for k, v in j.items() if k not in ("model", "steps")}
        o = oracle.Population(j["model"], **kw).step(j["steps"])
        v = b.population(i)
        assert v.t == j["steps"]
        assert np.array_equal(v.counts(), o.counts()), i
        if j["model"] == "wealth":
            assert np.array_equal(v.column("wealth").cpu().numpy(), o.w), i
        else:
            assert np.array_equal(v.column("state").cpu().numpy(), o.state), i
            assert np.array_equal(v.column("x").cpu().numpy(), o.x), i
            assert np.array_equal(v.column("y").cpu().numpy(), o.y), i


def test_sweep_invariants_every_job(sweep):
    jobs, b, _ = sweep
    for i, j in enumerate(jobs):
        c = b.population(i).counts()
        assert c.shape == (j["steps"], 4)
        if j["model"] == "wealth":
            assert np.all(c[:, 1] == j["n"]), i  # total wealth conserved
        else:
            assert np.all(c[:, :3].sum(axis=1) == j["n"]), i  # S + I + R = N
            assert np.all(np.diff(c[:, 2]) >= 0), i  # R never decreases


def test_sweep_largest_jobs_equal_lone_runs(sweep):
    jobs, b, stream = sweep
    for model in ("wealth", "sir"):
        i = max((k for k, j in enumerate(jobs) if j["model"] == model), key=lambda k: jobs[k]["n"])
        j = jobs[i]
        kw = {k: v for k, v in j.items() if k not in ("model", "steps")}
        alone = amb.Population(model, stream=stream, **kw).step(j["steps"])
        v = b.population(i)
        assert np.array_equal(v.counts(), alone.counts())
        for col in (("wealth",) if model == "wealth" else ("x", "y", "state")):
            assert torch.equal(v.column(col), alone.column(col)), (model, col)
        alone.close()
