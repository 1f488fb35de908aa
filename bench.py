"""Throughput benchmark of the columnar agent-step engine on GB300.

Headline workload (one bench step = one synchronous SIR step of the whole
population through the C ABI): 10,000,000 agents on a 4096 x 4096 torus,
10,000 initially infected, beta = 0.05, gamma = 0.02, seed 2 -- the
spatial-SIR configuration (move, cell-index rebuild, per-cell infected
counts, infection / recovery, per-step counters).  Also reported on the same
line: wealth transfer (10,000 agents, 100 steps) and random walk (1,000,000
agents on a 1000 x 1000 torus, 200 steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl amb|reference]

With N > 1 (torchrun, one process per GPU) every rank runs an independent
replicate (replicate = rank): the populations do not exchange data, so the
scaling is weak and the value is the sum over ranks of agent-steps divided by
the slowest rank's time.  --impl reference times the CPU oracle (the plain
single-threaded statement of the same rules) on the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIR_CFG = dict(n=10_000_000, L=4096, beta=0.05, gamma=0.02, n0=10_000, seed=2)
WEALTH_CFG = dict(n=10_000, seed=0, steps=100)
WALK_CFG = dict(n=1_000_000, L=1000, seed=1, steps=200)
L2_BYTES = 129 * 1024 * 1024


def sir_bytes_per_agent_step(n, L):
    """Algorithmic HBM bytes of one SIR step per agent (the method's own count,
    independent of the layout): read and write x, y (int32) and state (uint8)
    = 18 B, the cell-order permutation written and read = 8 B, the cell index
    start[C] written and read = 8 C / N B.  39.42 B at 10M agents on 4096^2."""
    C = L * L
    return 18.0 + 8.0 + 8.0 * C / n


def sir_layout_bytes_per_agent_step(n, L):
    """Compulsory traffic of this build's layout: one 8-byte cell-ordered
    record read and written per agent, start[C] written once: 16 + 4 C / N."""
    return 16.0 + 4.0 * L * L / n


def sir_config(world):
    """The workload's config, the same on both arms: the 10M-agent SIR
    population, one replicate per rank, and the working set against L2 (the
    step's records and cell index, 227 MB, exceed the 129 MB L2, so no flush
    is needed between timed steps)."""
    c = SIR_CFG
    return {"workload": "sir_10M_L4096", "n_agents": c["n"], "grid_side": c["L"], "beta": c["beta"],
            "gamma": c["gamma"], "n_init_infected": c["n0"], "seed": c["seed"],
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "working set %.0f MB > L2 129 MB (no flush needed)" % (
                sir_layout_bytes_per_agent_step(c["n"], c["L"]) * c["n"] / 1e6)}


def profiled(key, field="dram_bytes_per_launch"):
    """A per-launch figure of the kernel from the committed ncu capture (DRAM
    bytes read + written by default), or None when the kernel's sources
    changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)[key]
        h = hashlib.sha1()
        for p in d["source_files"]:
            with open(os.path.join(ROOT, p), "rb") as f:
                h.update(f.read())
        return d.get(field) if h.hexdigest() == d["source_sha1"] else None
    except Exception:
        return None


def profiled_traffic(key):
    return profiled(key)


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle readings (every 10 ms, timestamped) while
    the GPU runs the step kernel; stop() keeps those inside the timed window
    (falling back to the whole loaded period when the window is shorter than
    the sampling interval)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.window = None

    def start(self, wait_first=2.0):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "10"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < wait_first:
                time.sleep(0.005)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, t0, t1):
        """The timed region, in host time."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for t, ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append((t, float(f[2]), float(f[3]), [nm for nm, v in zip(names, f[6:10]) if v.lower() == "active"]))
            except ValueError:
                continue
        inside = [r for r in rows if self.window and self.window[0] - 0.01 <= r[0] <= self.window[1] + 0.01]
        use = inside if inside else rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = sorted(r[1] for r in use)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted({x for r in use for x in r[3]}), "samples": len(use),
                "samples_in_timed_window": len(inside)}


def dist_setup(n_gpus, backend="nccl"):
    """(world, rank, local rank) from the torchrun environment; joins the
    process group when there is more than one rank (only barriers and the
    final max / sum of scalars use it: ranks never exchange data)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return world, rank, local


def partition(items, rank, world):
    """This rank's share of a job list (round robin; every item exactly once)."""
    return items[rank::world]


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------- GPU arm ----
def time_sir(amb, torch, steps, warmup, rank, stream, world=1, sampler=None):
    c = SIR_CFG
    pop = amb.Population("sir", c["n"], seed=c["seed"], rep=rank, L=c["L"], beta=c["beta"], gamma=c["gamma"],
                         n0=c["n0"], stream=stream)
    if sampler is not None:
        sampler.start()
    for _ in range(warmup):
        pop.step(1)
    pop.synchronize()
    launches0 = amb.amb_launch_count(pop.handle)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    barrier(world)
    torch.cuda.synchronize()
    t_start = time.time()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(steps):
            amb.amb_step(pop.handle, 1)
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.mark(t_start, time.time())
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    total_ms = ev[0].elapsed_time(ev[steps])
    launches = amb.amb_launch_count(pop.handle) - launches0
    inv = pop.invariants()
    # the band path launches exactly one kernel per step
    path = "band" if launches == steps else "generic"
    pop.close()
    return total_ms, per, launches, inv, path


def time_model_block(amb, torch, model, cfg, stream, rank):
    """One amb_step(steps) call of the small models, timed on the stream."""
    kw = dict(seed=cfg["seed"], rep=rank, stream=stream)
    if "L" in cfg:
        kw["L"] = cfg["L"]
    pop = amb.Population(model, cfg["n"], **kw)
    # warm-up on a throwaway population so the timed one starts at step 0
    w = amb.Population(model, cfg["n"], **kw)
    w.step(cfg["steps"])
    w.synchronize()
    w.close()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    amb.amb_step(pop.handle, cfg["steps"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = amb.amb_launch_count(pop.handle)
    inv = pop.invariants()
    pop.close()
    return {"agent_steps_per_s": cfg["n"] * cfg["steps"] / (ms / 1e3), "ms": ms, "n": cfg["n"],
            "steps": cfg["steps"], "gpu_launches": launches, "invariants_ok": bool(inv["ok"])}


def run_e2e(amb, torch, steps, rank, stream):
    c = SIR_CFG
    n = c["n"]
    # the initial columns of this replicate, produced once on the host side of
    # the API (read back from a scratch population) and kept in pinned memory
    src = amb.Population("sir", n, seed=c["seed"], rep=rank, L=c["L"], beta=c["beta"], gamma=c["gamma"], n0=c["n0"],
                         stream=stream)
    hx = torch.empty(n, dtype=torch.int32, pin_memory=True)
    hy = torch.empty(n, dtype=torch.int32, pin_memory=True)
    hs = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    amb.amb_read_column(src.handle, "x", hx)
    amb.amb_read_column(src.handle, "y", hy)
    amb.amb_read_column(src.handle, "state", hs)
    src.close()
    pop = amb.Population("sir", n, seed=c["seed"], rep=rank, L=c["L"], beta=c["beta"], gamma=c["gamma"], n0=c["n0"],
                         stream=stream)
    out_state = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    rows = torch.zeros((steps, 4), dtype=torch.int64, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    amb.amb_write_column(pop.handle, "x", hx)
    amb.amb_write_column(pop.handle, "y", hy)
    amb.amb_write_column(pop.handle, "state", hs)
    for k in range(steps):
        amb.amb_step(pop.handle, 1)
        amb.amb_counts_async(pop.handle, k, 1, rows[k])  # each step's counts, read in stream order
    amb.amb_read_column(pop.handle, "state", out_state)  # synchronises
    t1 = time.perf_counter()
    if int(rows[-1].sum()) != 0 and int(rows[-1][:3].sum()) != n:
        raise RuntimeError("end-to-end run lost agents")
    pop.close()
    h2d = 9 * n
    d2h = 32 * steps + n
    return {"value": n * steps / (t1 - t0), "unit": "agent-steps/s", "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps, "seconds": t1 - t0}


def sweep_bench(amb, torch, stream, rank, world):
    """The parameter sweep (1,024 wealth / SIR replicates, 200 steps each;
    ranks split the job list): one batch, graph-captured and autotuned, against
    the same jobs stepped one at a time through amb_step on the same GPU."""
    from paper_2601_16292_gb300 import workloads
    jobs = partition(workloads.sweep_jobs(), rank, world)
    total = workloads.agent_steps(jobs)
    b = amb.Batch(jobs, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ms = b.run(autotune=True)
    wall = time.perf_counter() - t0
    info = b.info()
    # algorithmic bytes of the run: SIR 18 + 8 + 8 C/N per agent-step; wealth
    # 8 per agent-step (read and write w) + 8 per donor (the recipient's
    # read-modify-write), donors taken from each job's own count rows
    alg = 0.0
    for i, j in enumerate(jobs):
        if j["model"] == "sir":
            alg += j["steps"] * (26.0 * j["n"] + 8.0 * j["L"] * j["L"])
        else:
            alg += j["steps"] * 8.0 * j["n"] + 8.0 * float(b.population(i).counts()[:, 0].sum())
    b.close()
    # one job at a time: create, step all its steps, read its counts, destroy
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev_ms = 0.0
    launches = 0
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for j in jobs:
        kw = {k: v for k, v in j.items() if k not in ("model", "steps")}
        p = amb.Population(j["model"], stream=stream, **kw)
        e0.record(stream)
        amb.amb_step(p.handle, j["steps"])
        e1.record(stream)
        p.counts()
        e1.synchronize()
        dev_ms += e0.elapsed_time(e1)
        launches += amb.amb_launch_count(p.handle)
        p.close()
    wall_one = time.perf_counter() - t1
    return {"jobs": len(jobs), "agent_steps": total,
            "batched": {"value": total / (ms / 1e3), "device_ms": ms, "wall_s": wall, "launches": info["launches"],
                        "band_rows_cap": info["band_rows_cap"], "spread_bands": info["spread_bands"],
                        "algorithmic_gbs": alg / (ms / 1e3) / 1e9, "hbm_frac": alg / (ms / 1e3) / 1e9 / load_peaks()[0]},
            "one_at_a_time": {"value": total / (dev_ms / 1e3), "device_ms": dev_ms, "wall_s": wall_one,
                              "wall_value": total / wall_one, "launches": launches},
            "speedup_device": dev_ms / ms, "unit": "agent-steps/s"}


def _latency_summary(lat, total, span):
    import numpy as np
    lat = np.asarray(lat)
    return {"value": total / span, "makespan_s": span, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def serve_bench(amb, torch, stream, rank, world, n_jobs=5000, chunk=32, budget_gb=120, rates=(200.0, 400.0, 800.0),
                iteration_us=None):
    """The serving trace (5,000 jobs, Poisson arrivals at 200/s; ranks split the
    trace), replayed in real time at its own rate and with its arrival times
    compressed to 400 and 800 jobs/s (the same jobs in the same order): served
    by the continuous-batching loop under a 120 GB budget, and by one-at-a-time
    stepping through the plain API (each job created, stepped, its counts read,
    destroyed; a job starts when it has arrived and the previous one is done).
    Also every job queued at t = 0 (capacity).  Latency = arrival to result
    read.  Every served job's count rows must equal the same job's rows run
    alone (the run raises otherwise)."""
    import numpy as np
    from paper_2601_16292_gb300 import workloads
    arrivals, jobs = workloads.serve_trace(n_jobs=n_jobs)
    arrivals, jobs = partition(arrivals, rank, world), partition(jobs, rank, world)
    arrivals = np.asarray(arrivals, dtype=np.float64)
    total = workloads.agent_steps(jobs)
    cfg = dict(chunk_steps=chunk)
    if iteration_us is not None:
        cfg["iteration_us"] = iteration_us

    def served_run(arr, warm=False):
        srv = amb.Server(int(budget_gb * 1e9), stream, **cfg)
        if warm:  # the worker's code paths, on a few throwaway jobs
            for j in workloads.scaled(jobs[:6], 20_000):
                srv.submit(j)
            srv.drain(120.0)
        base = srv.stats()
        tickets = []
        t0 = time.perf_counter()
        for a, j in zip(arr, jobs):
            d = a - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit(j))
        srv.drain(3600.0)
        res = [srv.poll(t) for t in tickets]
        counts = [srv.counts(t) for t in tickets]
        st = srv.stats()
        srv.close()
        if any(r["status"] != amb.AMB_OK for r in res):
            raise RuntimeError("served jobs failed")
        first = min(r["submit_s"] for r in res)
        out = _latency_summary([r["done_s"] - r["submit_s"] for r in res], total,
                               max(r["done_s"] for r in res) - first)
        out.update({"iterations": st["iterations"] - base["iterations"], "launches": st["launches"] - base["launches"],
                    "hbm_peak_gb": st["hbm_peak"] / 1e9, "busy_s": st["busy_s"] - base["busy_s"]})
        return out, counts

    def one_at_a_time(arr, keep=None):
        lat = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, j in zip(arr, jobs):
            d = a - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            kw = {k: v for k, v in j.items() if k not in ("model", "steps")}
            p = amb.Population(j["model"], stream=stream, **kw)
            amb.amb_step(p.handle, j["steps"])
            c = p.counts()
            p.close()
            lat.append(time.perf_counter() - t0 - a)
            if keep is not None:
                keep.append(c)
        return _latency_summary(lat, total, time.perf_counter() - t0 - arr[0])

    def check(counts, alone):
        bad = [i for i, (a, b) in enumerate(zip(counts, alone)) if not np.array_equal(a, b)]
        if bad:
            raise RuntimeError("served results differ from one-at-a-time results: jobs %s" % bad[:10])

    by_rate = {}
    alone = []
    for k, rate in enumerate(rates):
        arr = arrivals * (200.0 / rate)
        served, counts = served_run(arr, warm=(k == 0))
        one = one_at_a_time(arr, alone if k == 0 else None)
        check(counts, alone)
        by_rate["%g" % (rate / world)] = {"served": served, "one_at_a_time": one,
                                          "offered_load": total / float(arr[-1] - arr[0]),
                                          "served_keeps_up": bool(served["makespan_s"] <= 1.1 * float(arr[-1] - arr[0])),
                                          "one_at_a_time_keeps_up":
                                              bool(one["makespan_s"] <= 1.1 * float(arr[-1] - arr[0]))}
    zero = np.zeros_like(arrivals)
    sat_served, counts = served_run(zero)
    check(counts, alone)
    sat_one = one_at_a_time(zero)
    base_key = "%g" % (rates[0] / world)
    return {"jobs": len(jobs), "agent_steps": total, "arrival_rate_per_s": rates[0] / world,
            "budget_gb": budget_gb, "chunk_steps": chunk, "offered_load": by_rate[base_key]["offered_load"],
            "trace": by_rate[base_key], "by_arrival_rate": by_rate,
            "saturated": {"served": sat_served, "one_at_a_time": sat_one,
                          "speedup_throughput": sat_served["value"] / sat_one["value"]},
            "results_equal_alone": {"jobs_checked": len(jobs), "runs": len(rates) + 1,
                                    "what": "every job's per-step count rows, served vs one at a time"},
            "unit": "agent-steps/s"}


def views_bench(amb, torch, stream, hbm, n=100_000_000, reps=5):
    """The view API's kernels on a 100M-row table (400 MB per int32 column,
    larger than L2): achieved algorithmic GB/s per operation (bytes the
    operation must move: every read and written element once; for id-indexed
    updates the id and the element's read and write) against the measured
    copy bandwidth; plus the wealth step written with views (10k agents,
    100 steps) beside the fused wealth kernel."""
    import numpy as np
    t = amb.Table(n, stream)
    t.add_column("c", "i32", fill=0)
    rng = np.random.default_rng(5)
    t.write("c", (rng.integers(0, 2, n, dtype=np.int32) * 2 - 1).astype(np.int32))  # +-1, half positive
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sorted(ms)[len(ms) // 2]

    out = {}
    ms = timed(lambda: t.map("c", "mul", 1))
    out["map_full"] = {"ms": ms, "bytes": 8 * n}
    # each timed call creates its view and frees it again (stream-ordered)
    ms = timed(lambda: t.where("c", ">", 0).close())
    v = t.where("c", ">", 0)
    k = v.count()
    out["where"] = {"ms": ms, "bytes": 4 * n + 4 * k, "selected": k}
    ms = timed(lambda: v.map("c", "mul", 1))
    out["view_map_filtered"] = {"ms": ms, "bytes": 12 * k}
    # a view of that view (conjunction): the list read, the column gathered
    # through it, the selected ids written
    ms = timed(lambda: v.where("c", "==", 1).close())
    out["where_of_view"] = {"ms": ms, "bytes": 8 * k + 4 * k, "selected": k}
    ids = torch.from_numpy(rng.integers(0, n, n // 10, dtype=np.int32)).cuda()
    torch.cuda.synchronize()
    sv = t.at(ids)
    ms = timed(lambda: sv.scatter_add("c", 0))
    out["scatter_add_random"] = {"ms": ms, "bytes": 12 * (n // 10)}
    ms = timed(lambda: v.draw(1, 0, 3, 0, n, True).close())
    out["draw"] = {"ms": ms, "bytes": 8 * k}
    sv.close()
    v.close()
    # buffered writes: 10M records on random rows (repeats included) of the
    # 100M-row column, applied by one flush (last record per row wins); bytes:
    # each record's row id, column index and value read once, each written row
    # written once
    n_rec = 10_000_000
    rec_ids = torch.from_numpy(rng.integers(0, n, n_rec, dtype=np.int32)).cuda()
    rec_vals = torch.from_numpy(rng.integers(-5, 5, n_rec, dtype=np.int64)).cuda()
    rows_written = int(np.unique(rec_ids.cpu().numpy()).size)
    log = t.log(n_rec)
    log.record("c", rec_ids, rec_vals)
    log.flush()  # first flush allocates the winner words
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        log.record("c", rec_ids, rec_vals)
        torch.cuda.synchronize()
        e0.record(stream)
        log.flush()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    out["log_flush_10M_records"] = {"ms": sorted(ms)[len(ms) // 2], "bytes": 16 * n_rec + 4 * rows_written,
                                    "records": n_rec, "rows_written": rows_written}
    log.close()
    t.close()
    # grid walks (k steps fused in registers): 10M agents, 3-D von Neumann in a
    # bounded 256 x 256 x 160 box and 2-D Moore on a 4096^2 torus, 50 steps;
    # bytes: every coordinate read and written once per call
    ng, gsteps = 10_000_000, 50
    tg = amb.Table(ng, stream)
    for name, size in (("gx", 256), ("gy", 256), ("gz", 160)):
        tg.add_column(name, "i32", fill=0)
        tg.write(name, rng.integers(0, size, ng, dtype=np.int32))
    for key, cols, sizes, moore, torus in (("grid_walk_3d_vn_bounded", ["gx", "gy", "gz"], [256, 256, 160], False, False),
                                           ("grid_walk_2d_moore_torus", ["gx", "gy"], [4096, 4096], True, True)):
        tg.grid_walk(cols, sizes, moore=moore, torus=torus, seed=1, step=0, steps=2)
        torch.cuda.synchronize()
        ms = []
        for r in range(reps):
            e0.record(stream)
            tg.grid_walk(cols, sizes, moore=moore, torus=torus, seed=1, step=2 + r * gsteps, steps=gsteps)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = sorted(ms)[len(ms) // 2]
        out[key] = {"ms": m, "bytes": 8 * len(cols) * ng, "agent_steps_per_s": ng * gsteps / (m / 1e3),
                    "bound": "integer multiply (one Philox per agent-step)"}
    tg.close()
    for r in out.values():
        r["gbs"] = r["bytes"] / (r["ms"] / 1e3) / 1e9
        r["frac"] = r["gbs"] / hbm
    # the wealth step written with views
    nw, steps = 10_000, 100
    tw = amb.Table(nw, stream)
    tw.add_column("wealth", "i32", fill=1)
    torch.cuda.synchronize()
    e0.record(stream)
    for step in range(steps):
        donors = tw.where("wealth", ">", 0)
        donors.map("wealth", "sub", 1)
        rec = donors.draw(0, 0, step, 0, nw, True)
        rec.scatter_add("wealth", 1)
        rec.close()
        donors.close()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    tw.close()
    out["wealth_by_views_10k_100steps"] = {"ms": ms, "agent_steps_per_s": nw * steps / (ms / 1e3), "launches": 4 * steps}
    out["table_rows"] = n
    out["peak_gbs"] = hbm
    return out


# The paper's own timings of its vectorised implementation (Table 1; laptop
# CPU, 50 steps, ms), quoted for context beside the same models here.
PAPER_AMBER_MS = {"wealth": {500: 4.4, 1000: 6.4, 5000: 21.0}, "cwalk": {500: 2.7, 1000: 2.7, 5000: 6.2},
                  "csir": {500: 95.0, 1000: 119.0, 5000: 687.0}}


def paper_models_bench(amb, torch, stream, steps=50, reps=3):
    """The paper's three benchmark models as the paper states them (Sec.
    5.1.2): wealth transfer, continuous random walk (100 x 100 box, step 1,
    clamped), continuous SIR (100 x 100, radius 5, p = 0.1, recovery after 14
    steps, 5 initial infected), N = 500 / 1,000 / 5,000, 50 steps.  wall_ms:
    create + 50 steps + read the counts (the paper's whole-run protocol; the
    median of `reps` runs), device_ms: the steps alone (CUDA events)."""
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for model in ("wealth", "cwalk", "csir"):
        for n in (500, 1000, 5000):
            walls, devs = [], []
            for rep in range(reps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if model == "wealth":
                    p = amb.Population("wealth", n, seed=0, rep=rep, stream=stream)
                else:
                    p = amb.CPopulation(model, n, seed=0, rep=rep, w=100.0, h=100.0, s=1.0 if model == "cwalk" else 0.0,
                                        r=5.0, p=0.1, rec_steps=14, n0=5, stream=stream)
                e0.record(stream)
                amb.amb_step(p.handle, steps)
                e1.record(stream)
                p.counts()
                wall = (time.perf_counter() - t0) * 1e3
                dev = e0.elapsed_time(e1)
                p.close()
                if rep:  # the first run warms up
                    walls.append(wall)
                    devs.append(dev)
            w = sorted(walls)[len(walls) // 2]
            d = sorted(devs)[len(devs) // 2]
            out["%s_%d" % (model, n)] = {"wall_ms": w, "device_ms": d,
                                         "agent_steps_per_s": n * steps / (w / 1e3),
                                         "paper_amber_cpu_ms": PAPER_AMBER_MS[model][n]}
    return out


def host_cpu():
    """The host's logical CPU count, CPU model and clock (what Linux reports:
    /proc/cpuinfo, then lscpu, then cpufreq), for the CPU baseline records."""
    info = {"nproc": os.cpu_count(), "model": None, "mhz": None}
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k, _, v = ln.partition(":")
                k = k.strip().lower()
                if k == "model name" and not info["model"]:
                    info["model"] = v.strip()
                elif k == "cpu mhz" and not info["mhz"]:
                    info["mhz"] = float(v)
    except Exception:
        pass
    if not info["model"] or not info["mhz"]:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                k, _, v = ln.partition(":")
                k = k.strip()
                if k == "Model name" and not info["model"]:
                    info["model"] = v.strip()
                elif k in ("CPU max MHz", "CPU MHz") and not info["mhz"]:
                    info["mhz"] = float(v)
        except Exception:
            pass
    if not info["mhz"]:
        try:
            with open("/sys/devices/system/cpu/cpu0/cpufreq/cpuinfo_max_freq") as f:
                info["mhz"] = int(f.read()) / 1000.0
        except Exception:
            pass
    return info


def timed_oracle_runs(p, steps, runs=3):
    """The paper's timing protocol (three runs, the slowest dropped, the other
    two averaged): `runs` consecutive runs of `steps` whole steps of the
    oracle population p.  Returns (mean seconds of the kept runs, all run
    times)."""
    times = []
    for _ in range(runs):
        t0 = time.perf_counter()
        p.step(steps)
        times.append(time.perf_counter() - t0)
    kept = sorted(times)[:-1] if runs > 1 else times
    return sum(kept) / len(kept), times


def cpu_baseline(budget_s=15.0):
    """The oracle as it stands on one host core (it is single-threaded): the
    full 10M-agent SIR population, three runs of k whole steps after one
    untimed step, the slowest run dropped and the other two averaged (the
    paper's protocol), k sized so that the three runs take about budget_s."""
    import oracle
    c = SIR_CFG
    p = oracle.Population("sir", c["n"], seed=c["seed"], L=c["L"], beta=c["beta"], gamma=c["gamma"], n0=c["n0"])
    t0 = time.perf_counter()
    p.step(1)
    one = time.perf_counter() - t0
    k = max(1, min(50, int(budget_s / 3.0 / max(one, 1e-6))))
    mean_s, times = timed_oracle_runs(p, k)
    return {"value": c["n"] * k / mean_s, "unit": "agent-steps/s", "cores": 1, "kind": "oracle",
            "sample": "steps 1..%d of the 10M-agent SIR population (all agents, one thread) as three runs of %d "
                      "steps, slowest dropped, other two averaged" % (3 * k, k),
            "run_s": times, "host": host_cpu()}


def gpu_arm(args):
    import torch
    from paper_2601_16292_gb300 import amb
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=device)
    amb.lib()

    # untimed extras first (they are short): small models and e2e
    only_sir = args.only == "sir"
    wealth = None if only_sir else time_model_block(amb, torch, "wealth", WEALTH_CFG, stream, rank)
    walk = None if only_sir else time_model_block(amb, torch, "walk", WALK_CFG, stream, rank)
    sweep = None if only_sir else sweep_bench(amb, torch, stream, rank, world)
    views = None if only_sir else views_bench(amb, torch, stream, load_peaks()[0])
    paper_models = None if only_sir else paper_models_bench(amb, torch, stream)

    sampler = ClockSampler(local)
    total_ms, per, launches, inv, path = time_sir(amb, torch, args.steps, args.warmup, rank, stream, world, sampler)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    total_ms_max = max_over_ranks(world, total_ms, device)
    agent_steps = sum_over_ranks(world, float(SIR_CFG["n"]) * args.steps, device)
    e2e = None if only_sir else run_e2e(amb, torch, max(args.steps, 3), rank, stream)
    e2e_val = None if only_sir else sum_over_ranks(world, e2e["value"], device)
    serve = None if only_sir else serve_bench(amb, torch, stream, rank, world)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    hbm, peak_kind = load_peaks()
    n, L = SIR_CFG["n"], SIR_CFG["L"]
    b_alg = sir_bytes_per_agent_step(n, L)
    b_layout = sir_layout_bytes_per_agent_step(n, L)
    per_sorted = sorted(per)
    step_ms = per_sorted[len(per_sorted) // 2]
    achieved = b_alg * n / (step_ms / 1e3) / 1e9
    value = agent_steps / (total_ms_max / 1e3)
    traffic = profiled_traffic("sir_%s" % path)
    # the step is issue-bound: its warp instructions (ncu) against the SMs'
    # issue peak, 4 warp instructions per SM per cycle at the sampled clock
    winst = profiled("sir_%s" % path, "warp_instructions_per_launch")
    issue = None
    if winst and clocks and clocks.get("sm_mhz"):
        import torch
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak_issue = sms * 4 * clocks["sm_mhz"] * 1e6
        issue = {"warp_instructions": winst, "achieved_per_s": winst / (step_ms / 1e3), "peak_per_s": peak_issue,
                 "frac": winst / (step_ms / 1e3) / peak_issue, "sms": sms, "sm_mhz": clocks["sm_mhz"]}
    line = {
        "metric": "agent-steps/s (spatial SIR, 10M agents, 4096x4096 torus)",
        "value": value,
        "unit": "agent-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32/u8",
        "data": "synthetic (seeded Philox initial state, no dataset)",
        "config": sir_config(world),
        "sir_path": path,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_kind": peak_kind, "traffic": traffic, "bytes_per_agent_step": b_alg,
                     "layout_bytes_per_agent_step": b_layout, "layout_frac": b_layout * n / (step_ms / 1e3) / 1e9 / hbm,
                     "kernel_ms_median": step_ms, "issue": issue,
                     # the same against the nominal HBM3e bandwidth (context only)
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_gbs": NOMINAL_HBM_GBS},
        "cpu_baseline": None if only_sir else cpu_baseline(),
        "e2e": None if only_sir else {"value": e2e_val, "unit": "agent-steps/s",
                                      "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                                      "d2h_bytes_per_step": e2e["d2h_bytes_per_step"]},
        "gpu_launches": launches,
        "clocks": clocks,
        "invariants_ok": bool(inv["ok"]),
        "models": {"wealth_10k_100steps": wealth, "walk_1M_L1000_200steps": walk},
        "sweep_1024_jobs": sweep,
        "view_api": views,
        "paper_models_50steps": paper_models,
        "serve_5000_jobs": serve,
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------- reference arm ----
def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    c = SIR_CFG
    p = oracle.Population("sir", c["n"], seed=c["seed"], L=c["L"], beta=c["beta"], gamma=c["gamma"], n0=c["n0"])
    # each step is a whole step of the full population; keep the run bounded:
    # three runs of up to 15 steps, the slowest dropped (the paper's protocol)
    steps = max(1, min(args.steps, 15))
    warm = max(0, min(args.warmup, 3))
    for _ in range(warm):
        p.step(1)
    dt, times = timed_oracle_runs(p, steps)
    v = c["n"] * steps / dt
    line = {
        "impl": "reference",
        "metric": "agent-steps/s (spatial SIR, 10M agents, 4096x4096 torus)",
        "value": v,
        "unit": "agent-steps/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": warm,
        "ms_per_step": dt * 1e3 / steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32/u8",
        "data": "synthetic (seeded Philox initial state, no dataset)",
        "config": sir_config(world),
        "cpu_baseline": {"value": v, "unit": "agent-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "steps %d..%d of the full 10M-agent population, one thread, as three runs of %d "
                                   "steps, slowest dropped, other two averaged" % (warm, warm + 3 * steps, steps),
                         "run_s": times, "host": host_cpu()},
        "e2e": {"value": v, "unit": "agent-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="amb", choices=["amb", "reference"])
    ap.add_argument("--only", default="all", choices=["all", "sir", "sweep", "serve", "views", "paper", "models"],
                    help="sir: time the SIR step alone (no extras; for profiling); sweep / serve: that part alone")
    ap.add_argument("--serve-jobs", type=int, default=5000)
    ap.add_argument("--serve-chunk", type=int, default=32)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "amb" and args.only == "sweep":
        import torch
        from paper_2601_16292_gb300 import amb
        torch.cuda.set_device(0)
        print(json.dumps(sweep_bench(amb, torch, torch.cuda.Stream(), 0, 1)))
        return
    if args.impl == "amb" and args.only == "models":
        import torch
        from paper_2601_16292_gb300 import amb
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        print(json.dumps({"wealth_10k_100steps": time_model_block(amb, torch, "wealth", WEALTH_CFG, st, 0),
                          "walk_1M_L1000_200steps": time_model_block(amb, torch, "walk", WALK_CFG, st, 0)}))
        return
    if args.impl == "amb" and args.only == "paper":
        import torch
        from paper_2601_16292_gb300 import amb
        torch.cuda.set_device(0)
        print(json.dumps(paper_models_bench(amb, torch, torch.cuda.Stream())))
        return
    if args.impl == "amb" and args.only == "views":
        import torch
        from paper_2601_16292_gb300 import amb
        torch.cuda.set_device(0)
        print(json.dumps(views_bench(amb, torch, torch.cuda.Stream(), load_peaks()[0])))
        return
    if args.impl == "amb" and args.only == "serve":
        import torch
        from paper_2601_16292_gb300 import amb
        torch.cuda.set_device(0)
        print(json.dumps(serve_bench(amb, torch, torch.cuda.Stream(), 0, 1, n_jobs=args.serve_jobs,
                                     chunk=args.serve_chunk)))
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
