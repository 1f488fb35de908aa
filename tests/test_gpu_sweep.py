"""The parameter sweep (1,024 wealth and SIR replicates of uneven size, 200
steps each) advanced as one batch: a stratified sample of 32 jobs (16 per
model, evenly spaced by size rank, the smallest and the largest included, up
to 10^6 agents at full length) equals the oracle bit for bit, every job keeps
the models' invariants in its per-step counts, and the largest jobs equal a
lone run of the same job."""
import numpy as np
import pytest

from oracle_jobs import oracle_pool, stratified, submit_oracle_jobs
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


def test_sweep_sample_equals_oracle(sweep):
    jobs, b, _ = sweep
    sample = stratified(jobs, {"wealth": 16, "sir": 16})
    assert len(sample) == 32
    assert max(jobs[i]["n"] for i in sample) == max(j["n"] for j in jobs)
    with oracle_pool(len(sample)) as pool:
        futs = submit_oracle_jobs([jobs[i] for i in sample], pool)
        for i, f in zip(sample, futs):
            j = jobs[i]
            o = f.result()
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
