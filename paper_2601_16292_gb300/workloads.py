"""Seeded synthetic job lists for the parameter sweep and the serving trace.

Only the inputs are generated here (which model, population size, grid side,
parameters, seeds, arrival times); nothing of the models' step rules.  The same
lists feed the GPU path, the tests and the timing harness.

Sweep (many replicates of uneven size advanced together, the paper's
Experiment / ParallelRunner use, Sec. 4.2): 1,024 jobs, model wealth or SIR
with probability 1/2 each, N log-uniform in [10^3, 10^6], beta ~ U[0.01, 0.2],
gamma ~ U[0.005, 0.05], grid side chosen for a mean density of 0.6 agents per
cell, 200 steps, replicate = job index.

Serving trace: 5,000 jobs with Poisson arrivals at 200 jobs/s, model uniform
over {wealth, walk, SIR}, N log-uniform in [10^3, 4*10^6], steps uniform in
{50, ..., 500}, parameters as in the sweep, replicate = job index and a Philox
key drawn per job.
"""
import math

import numpy as np

DENSITY = 0.6


def grid_side(n, density=DENSITY):
    """Grid side for a mean density of `density` agents per cell (at least 1)."""
    return max(1, int(round(math.sqrt(n / density))))


def initial_infected(n):
    """0.1 % of the population, rounded, at least one (none when n = 0)."""
    return 0 if n == 0 else max(1, int(math.floor(n * 0.001 + 0.5)))


def _log_uniform_int(rng, lo, hi, size):
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size))).astype(np.int64)


def _job(model, n, seed, rep, steps, beta, gamma):
    j = dict(model=model, n=int(n), seed=int(seed), rep=int(rep), steps=int(steps))
    if model in ("walk", "sir"):
        j["L"] = grid_side(n)
    if model == "sir":
        j.update(beta=float(beta), gamma=float(gamma), n0=initial_infected(n))
    if model == "wealth":
        j["w_init"] = 1
    return j


def sweep_jobs(n_jobs=1024, seed=3, steps=200, n_lo=1_000, n_hi=1_000_000):
    """The parameter sweep: list of job dicts (make_job keywords)."""
    rng = np.random.default_rng(seed)
    is_sir = rng.random(n_jobs) < 0.5
    ns = _log_uniform_int(rng, n_lo, n_hi, n_jobs)
    betas = rng.uniform(0.01, 0.2, n_jobs)
    gammas = rng.uniform(0.005, 0.05, n_jobs)
    return [_job("sir" if is_sir[i] else "wealth", ns[i], seed, i, steps, betas[i], gammas[i])
            for i in range(n_jobs)]


def serve_trace(n_jobs=5000, seed=4, rate=200.0, n_lo=1_000, n_hi=4_000_000, steps_lo=50, steps_hi=500):
    """The serving trace: (arrival times in seconds from 0, job dicts)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_jobs))
    models = rng.integers(0, 3, n_jobs)
    ns = _log_uniform_int(rng, n_lo, n_hi, n_jobs)
    steps = rng.integers(steps_lo, steps_hi + 1, n_jobs)
    betas = rng.uniform(0.01, 0.2, n_jobs)
    gammas = rng.uniform(0.005, 0.05, n_jobs)
    keys = rng.integers(0, 2 ** 32, n_jobs, dtype=np.uint64)
    names = ("wealth", "walk", "sir")
    jobs = [_job(names[models[i]], ns[i], keys[i], i, steps[i], betas[i], gammas[i]) for i in range(n_jobs)]
    return arrivals, jobs


def agent_steps(jobs):
    return int(sum(j["n"] * j["steps"] for j in jobs))


def scaled(jobs, max_n):
    """The jobs with N at most max_n (same parameters; grid side and initial
    infected follow N): a small stand-in of a list for quick checks."""
    out = []
    for j in jobs:
        if j["n"] <= max_n:
            out.append(dict(j))
            continue
        k = _job(j["model"], max_n, j["seed"], j["rep"], j["steps"], j.get("beta", 0.0), j.get("gamma", 0.0))
        out.append(k)
    return out
