"""The serving loop: jobs submitted while others run are admitted in arrival
order under the memory budget, advanced together, and each job's result (its
per-step counts and final columns) is the same as the job stepped alone, and
as the oracle for the small ones."""
import time

import numpy as np
import pytest

import oracle
from oracle_jobs import oracle_pool, stratified, submit_oracle_jobs
from paper_2601_16292_gb300 import amb, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RESERVE = 512 << 20  # the server's fixed reserve for per-iteration tables

MIX = [
    dict(model="sir", n=50_000, L=289, beta=0.15, gamma=0.03, n0=50, seed=11, rep=0, steps=37),
    dict(model="wealth", n=20_000, seed=12, rep=1, steps=41),
    dict(model="walk", n=120_000, L=447, seed=13, rep=2, steps=29),
    dict(model="sir", n=300_000, L=707, beta=0.05, gamma=0.01, n0=300, seed=14, rep=3, steps=23),
    dict(model="wealth", n=90_000, seed=15, rep=4, steps=17, w_init=3),
    dict(model="sir", n=2_000, L=58, beta=0.2, gamma=0.05, n0=2, seed=16, rep=5, steps=50),
    dict(model="sir", n=80_000, L=365, beta=0.1, gamma=0.02, n0=80, seed=17, rep=6, steps=0),
    dict(model="walk", n=5_000, L=91, seed=18, rep=7, steps=61),
    dict(model="sir", n=150_000, L=500, beta=0.08, gamma=0.04, n0=150, seed=19, rep=8, steps=31),
]


@pytest.fixture(scope="module")
def stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch.cuda.Stream()


def _lone(job, stream):
    kw = {k: v for k, v in job.items() if k not in ("model", "steps")}
    p = amb.Population(job["model"], stream=stream, **kw)
    p.step(job["steps"])
    cols = ("wealth",) if job["model"] == "wealth" else (("x", "y", "state") if job["model"] == "sir" else ("x", "y"))
    out = {c: p.column(c).cpu().numpy() for c in cols}
    out["counts"] = p.counts()
    p.close()
    return out


@pytest.mark.parametrize("chunk,extra_mb", [(8, 24), (64, 400)], ids=["tight-budget", "roomy"])
def test_mix_equals_alone(stream, chunk, extra_mb):
    budget = RESERVE + (extra_mb << 20)
    srv = amb.Server(budget, stream, chunk_steps=chunk)
    tickets = []
    for i, j in enumerate(MIX):
        tickets.append(srv.submit(j, keep_columns=True))
        if i == 3:
            time.sleep(0.005)  # the rest arrive while the first ones run
    res = [srv.wait(t, 120.0) for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(MIX) and st["failed"] == 0
    assert st["hbm_peak"] <= budget
    # admission in arrival order
    admits = [r["admit_s"] for r in res]
    assert admits == sorted(admits)
    for t, j, r in zip(tickets, MIX, res):
        assert r["status"] == amb.AMB_OK and r["steps"] == j["steps"]
        assert r["submit_s"] <= r["admit_s"] <= r["done_s"]
        ref = _lone(j, stream)
        c = srv.counts(t)
        assert np.array_equal(c, ref["counts"]), j
        if j["steps"]:
            assert list(r["last"]) == list(c[-1])
        else:
            assert list(r["last"]) == [0, 0, 0, 0]
        for col, v in ref.items():
            if col != "counts":
                assert np.array_equal(srv.column(t, col), v), (j, col)
    srv.close()


def test_small_jobs_equal_oracle(stream):
    srv = amb.Server(RESERVE + (64 << 20), stream, chunk_steps=5)
    small = [j for j in MIX if j["n"] <= 50_000]
    tickets = [srv.submit(j, keep_columns=True) for j in small]
    srv.drain(120.0)
    for t, j in zip(tickets, small):
        kw = {k: v for k, v in j.items() if k not in ("model", "steps")}
        o = oracle.Population(j["model"], **kw).step(j["steps"])
        assert np.array_equal(srv.counts(t), o.counts())
        if j["model"] == "wealth":
            assert np.array_equal(srv.column(t, "wealth"), o.w)
        else:
            assert np.array_equal(srv.column(t, "x"), o.x)
            if j["model"] == "sir":
                assert np.array_equal(srv.column(t, "state"), o.state)
    srv.close()


def test_errors_and_lifecycle(stream):
    srv = amb.Server(RESERVE + (32 << 20), stream)
    # a job that can never fit the budget
    with pytest.raises(amb.AmbError) as e:
        srv.submit(dict(model="sir", n=4_000_000, L=2582, beta=0.1, gamma=0.02, n0=4000, seed=1, steps=10))
    assert e.value.status == amb.AMB_EBUDGET
    with pytest.raises(amb.AmbError) as e:
        srv.submit(dict(model="sir", n=100, L=10, beta=2.0, gamma=0.02, n0=1, seed=1, steps=10))
    assert e.value.status == amb.AMB_EINVAL
    with pytest.raises(amb.AmbError) as e:
        amb.amb_server_poll(srv.handle, 10 ** 9)
    assert e.value.status == amb.AMB_ENOTFOUND
    # a long job is still queued or running right after submission
    t = srv.submit(dict(model="sir", n=400_000, L=816, beta=0.1, gamma=0.02, n0=400, seed=3, steps=400))
    assert srv.poll(t) is None
    with pytest.raises(amb.AmbError) as e:
        srv.release(t)
    assert e.value.status == amb.AMB_EBUSY
    r = srv.wait(t, 120.0)
    assert r["status"] == amb.AMB_OK and r["steps"] == 400
    c = srv.counts(t)
    assert c.shape == (400, 4) and np.all(c[:, :3].sum(axis=1) == 400_000)
    with pytest.raises(amb.AmbError):
        srv.column(t, "x")  # not kept
    srv.release(t)
    with pytest.raises(amb.AmbError) as e:
        srv.poll(t)
    assert e.value.status == amb.AMB_ENOTFOUND
    st = srv.stats()
    assert st["active"] == 0 and st["pending"] == 0 and st["hbm_in_use"] == 0
    srv.close()


def test_destroy_with_work_in_flight(stream):
    srv = amb.Server(RESERVE + (256 << 20), stream, chunk_steps=4)
    for j in workloads.scaled(workloads.serve_trace(n_jobs=40)[1], 200_000):
        srv.submit(j)
    time.sleep(0.01)
    srv.close()  # stops after the current iteration and frees everything
    torch.cuda.synchronize()


def test_injected_creation_failures_fail_only_those_jobs(stream):
    jobs = [dict(model="wealth", n=2000 + i, seed=i, steps=7) for i in range(5)]
    srv = amb.Server(RESERVE + (64 << 20), stream, max_active=1)
    amb.amb_debug_fail_creates(2)
    try:
        tickets = [srv.submit(j) for j in jobs]
        res = [srv.wait(t, 60.0) for t in tickets]
    finally:
        amb.amb_debug_fail_creates(0)
    assert [r["status"] for r in res] == [amb.AMB_ENOMEM] * 2 + [amb.AMB_OK] * 3
    for t, j, r in list(zip(tickets, jobs, res))[2:]:
        assert np.array_equal(srv.counts(t), _lone(j, stream)["counts"])
    st = srv.stats()
    assert st["failed"] == 2 and st["completed"] == 3 and st["hbm_in_use"] == 0
    srv.close()


def test_cancel_queued_and_running_jobs(stream):
    srv = amb.Server(RESERVE + (400 << 20), stream, max_active=1, chunk_steps=1)
    long_job = dict(model="sir", n=1_000_000, L=1291, beta=0.05, gamma=0.02, n0=1000, seed=1, steps=2000)
    a = srv.submit(long_job)
    b = srv.submit(dict(model="walk", n=1000, L=41, seed=2, steps=5))   # queued behind a (one slot)
    c = srv.submit(dict(model="wealth", n=1000, seed=3, steps=5))
    srv.cancel(b)
    rb = srv.wait(b, 5.0)
    assert rb["status"] == amb.AMB_ECANCELED and rb["admit_s"] < 0
    for _ in range(200):  # a is running once it has been admitted
        if srv.stats()["admitted"] >= 1:
            break
        time.sleep(0.01)
    srv.cancel(a)
    ra = srv.wait(a, 60.0)
    assert ra["status"] == amb.AMB_ECANCELED and ra["steps"] < 2000
    rc = srv.wait(c, 60.0)
    assert rc["status"] == amb.AMB_OK and rc["steps"] == 5
    srv.cancel(c)  # finished jobs are left as they are
    assert srv.wait(c, 1.0)["status"] == amb.AMB_OK
    st = srv.stats()
    assert st["cancelled"] == 2 and st["completed"] == 1 and st["active"] == 0 and st["hbm_in_use"] == 0
    with pytest.raises(amb.AmbError):
        srv.counts(a)
    srv.close()


def test_serving_trace_sample_equals_oracle(stream):
    """50 jobs of the 5,000-job serving trace at their own sizes and lengths
    (up to 4 million agents and 500 steps; 17 wealth, 17 walk and 16 SIR jobs
    evenly spaced by size rank, the smallest and the largest of each model
    included), submitted to one server together: each job's count series and
    final columns equal the oracle's run of that job."""
    trace = workloads.serve_trace()[1]
    sample = stratified(trace, {"wealth": 17, "walk": 17, "sir": 16})
    assert len(sample) == 50
    jobs = [trace[i] for i in sample]
    with oracle_pool(len(jobs)) as pool:
        futs = submit_oracle_jobs(jobs, pool)
        srv = amb.Server(RESERVE + (64 << 30), stream, chunk_steps=32)
        tickets = [srv.submit(j, keep_columns=True) for j in jobs]
        srv.drain(600.0)
        for t, j, f in zip(tickets, jobs, futs):
            assert srv.poll(t)["status"] == amb.AMB_OK, j
            o = f.result()
            assert np.array_equal(srv.counts(t), o.counts()), j
            cols = ("wealth",) if j["model"] == "wealth" else (("x", "y", "state") if j["model"] == "sir" else ("x", "y"))
            for c in cols:
                assert np.array_equal(srv.column(t, c), getattr(o, "w" if c == "wealth" else c)), (j, c)
            srv.release(t)
        srv.close()
