"""Helpers of the parity tests: oracle runs of many jobs side by side, and the
canonical form of a cell index.

Each job is the plain single-threaded C oracle; several jobs run at once on
host threads, because ctypes releases the interpreter lock for the duration
of each oracle call.  Only the tests use this module.
"""
import concurrent.futures as cf
import os

import numpy as np

import oracle


def oracle_job(job):
    """The oracle population of one job dict (make_job keywords), stepped
    through all of its steps."""
    kw = {k: v for k, v in job.items() if k not in ("model", "steps")}
    return oracle.Population(job["model"], **kw).step(job["steps"])


def workers_for(n_jobs):
    return max(1, min(n_jobs, os.cpu_count() or 1, 16))


def submit_oracle_jobs(jobs, pool):
    """Futures of the oracle runs of `jobs` (largest first, so that no large
    job starts last), in the order of `jobs`."""
    oracle.lib()  # load the library once, before the threads start
    order = sorted(range(len(jobs)), key=lambda i: -jobs[i]["n"] * max(jobs[i]["steps"], 1))
    futs = {i: pool.submit(oracle_job, jobs[i]) for i in order}
    return [futs[i] for i in range(len(jobs))]


def oracle_pool(n_jobs):
    return cf.ThreadPoolExecutor(workers_for(n_jobs))


def canonical_ids(start, ids):
    """The ids of a cell index with each cell's ids in ascending order (the
    order inside a cell is free; the oracle's stable sort gives this form)."""
    start = np.asarray(start, dtype=np.int64)
    ids = np.asarray(ids, dtype=np.int64)
    cell = np.repeat(np.arange(start.size - 1, dtype=np.int64), np.diff(start))
    key = np.sort((cell << 32) | ids, kind="stable")
    return (key & 0xFFFFFFFF).astype(np.int32)


def stratified(jobs, per_model):
    """Indices of an evenly spaced sample by size rank within each model
    (smallest and largest included): per_model maps model -> sample size."""
    out = []
    for model, k in per_model.items():
        idx = sorted((i for i, j in enumerate(jobs) if j["model"] == model), key=lambda i: (jobs[i]["n"], i))
        if not idx:
            continue
        pick = np.unique(np.linspace(0, len(idx) - 1, min(k, len(idx))).round().astype(int))
        out += [idx[p] for p in pick]
    return out
