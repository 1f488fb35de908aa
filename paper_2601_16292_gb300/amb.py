"""Python binding of the C ABI in include/amb.h (ctypes, argument marshalling
only).  Every computation runs in libamb.so's CUDA kernels; importing this
module fails loudly when the in-tree library is missing.

Functions carry the C names.  Column buffers may be torch tensors (device or
host) or numpy arrays (host); device tensors are passed as device pointers.
Streams are torch.cuda.Stream objects or raw cudaStream_t integers.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamb.so")

AMB_OK, AMB_EINVAL, AMB_ENOMEM, AMB_ECUDA, AMB_EINVARIANT = 0, 1, 2, 3, 4
AMB_ETIMEOUT, AMB_EBUSY, AMB_EBUDGET, AMB_ENOTFOUND, AMB_ECANCELED = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "AMB_OK", 1: "AMB_EINVAL", 2: "AMB_ENOMEM", 3: "AMB_ECUDA", 4: "AMB_EINVARIANT",
                5: "AMB_ETIMEOUT", 6: "AMB_EBUSY", 7: "AMB_EBUDGET", 8: "AMB_ENOTFOUND", 9: "AMB_ECANCELED"}

AMB_WEALTH, AMB_WALK, AMB_SIR, AMB_CWALK, AMB_CSIR = 0, 1, 2, 3, 4
MODELS = {"wealth": AMB_WEALTH, "walk": AMB_WALK, "sir": AMB_SIR, "cwalk": AMB_CWALK, "csir": AMB_CSIR}
AMB_COL_WEALTH, AMB_COL_X, AMB_COL_Y, AMB_COL_STATE, AMB_COL_DAYS = 0, 1, 2, 3, 4
COLUMNS = {"wealth": AMB_COL_WEALTH, "x": AMB_COL_X, "y": AMB_COL_Y, "state": AMB_COL_STATE, "days": AMB_COL_DAYS}
AMB_S, AMB_I, AMB_R = 0, 1, 2
AMB_SIR_AUTO, AMB_SIR_GENERIC, AMB_SIR_BAND, AMB_SIR_BAND32, AMB_SIR_BAND16 = 0, 1, 2, 3, 4


class AmbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class amb_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("grid_side", ctypes.c_uint32), ("beta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("n_init_infected", ctypes.c_uint32), ("w_init", ctypes.c_int32),
                ("variant", ctypes.c_uint32)]


class amb_invariant_report(ctypes.Structure):
    _fields_ = [("ok", ctypes.c_int32), ("conservation_ok", ctypes.c_int32), ("nonnegative_ok", ctypes.c_int32),
                ("bounds_ok", ctypes.c_int32), ("population_ok", ctypes.c_int32), ("monotone_ok", ctypes.c_int32),
                ("initial_ok", ctypes.c_int32), ("index_ok", ctypes.c_int32), ("first_bad_step", ctypes.c_int64)]


class amb_stats(ctypes.Structure):
    _fields_ = [("gini", ctypes.c_double), ("gini_num_hi", ctypes.c_int64), ("gini_num_lo", ctypes.c_uint64),
                ("total_wealth", ctypes.c_int64), ("min_wealth", ctypes.c_int32), ("max_wealth", ctypes.c_int32),
                ("peak_infected", ctypes.c_int64), ("peak_step", ctypes.c_uint32), ("curve_mean", ctypes.c_double),
                ("curve_var", ctypes.c_double), ("final_s", ctypes.c_int64), ("final_i", ctypes.c_int64),
                ("final_r", ctypes.c_int64), ("max_occupancy", ctypes.c_int32)]


class amb_cparams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("width", ctypes.c_float), ("height", ctypes.c_float), ("step", ctypes.c_float),
                ("radius", ctypes.c_float), ("p_infect", ctypes.c_double), ("recovery_steps", ctypes.c_uint32),
                ("n_init_infected", ctypes.c_uint32)]


class amb_job(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("params", amb_params), ("seed", ctypes.c_uint64),
                ("replicate", ctypes.c_uint32), ("steps", ctypes.c_uint32)]


class amb_tune(ctypes.Structure):
    _fields_ = [("band_rows_cap", ctypes.c_uint32), ("spread_bands", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


class amb_batch_report(ctypes.Structure):
    _fields_ = [("n_jobs", ctypes.c_size_t), ("band_rows_cap", ctypes.c_uint32), ("spread_bands", ctypes.c_int32),
                ("launches", ctypes.c_uint64),
                ("agent_steps", ctypes.c_uint64), ("ms", ctypes.c_double)]


class amb_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_uint32),
                ("chunk_steps", ctypes.c_uint32), ("band_rows_cap", ctypes.c_uint32), ("spread_bands", ctypes.c_int32),
                ("iteration_us", ctypes.c_uint32)]


class amb_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int), ("model", ctypes.c_int), ("n", ctypes.c_uint32),
                ("steps", ctypes.c_uint32), ("last", ctypes.c_int64 * 4), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class amb_server_report(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64), ("agent_steps", ctypes.c_uint64), ("iterations", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("hbm_in_use", ctypes.c_size_t), ("hbm_peak", ctypes.c_size_t),
                ("active", ctypes.c_uint32), ("pending", ctypes.c_uint32), ("busy_s", ctypes.c_double)]


_lib = None


def lib():
    """The loaded libamb.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libamb.so not built: run __graft_entry__.build() (expected at %s)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, u64, i32, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t
        st = ctypes.c_int
        sig = {
            "amb_create": (st, [ctypes.c_int, ctypes.POINTER(amb_params), u64, u32, vp, ctypes.POINTER(vp)]),
            "amb_destroy": (st, [vp]),
            "amb_set_step": (st, [vp, u64]),
            "amb_selfcheck_wait_timeout": (st, [vp, ctypes.POINTER(ctypes.c_double)]),
            "amb_create_continuous": (st, [ctypes.c_int, ctypes.POINTER(amb_cparams), u64, u32, vp,
                                           ctypes.POINTER(vp)]),
            "amb_step": (st, [vp, u32]),
            "amb_write_column": (st, [vp, ctypes.c_int, vp, sz, ctypes.c_int]),
            "amb_read_column": (st, [vp, ctypes.c_int, vp, sz, ctypes.c_int]),
            "amb_counts": (st, [vp, vp, sz, ctypes.POINTER(sz)]),
            "amb_read_index": (st, [vp, vp, vp, ctypes.c_int]),
            "amb_counts_range": (st, [vp, u64, sz, vp]),
            "amb_counts_async": (st, [vp, u64, sz, vp]),
            "amb_launch_count": (u64, [vp]),
            "amb_invariants": (st, [vp, ctypes.POINTER(amb_invariant_report)]),
            "amb_stats_compute": (st, [vp, ctypes.POINTER(amb_stats), vp, sz, ctypes.POINTER(sz)]),
            "amb_occupancy": (st, [vp, vp, ctypes.c_int]),
            "amb_step_index": (u64, [vp]),
            "amb_synchronize": (st, [vp]),
            "amb_last_error": (ctypes.c_char_p, []),
            "amb_sir_thresholds": (st, [ctypes.c_double, ctypes.c_double, u32, vp, ctypes.POINTER(u32),
                                        ctypes.POINTER(u32)]),
            "amb_cell_index": (st, [vp, vp, u32, u32, vp, vp, vp, ctypes.c_int]),
            "amb_cell_index_noalloc": (st, [vp, vp, u32, u32, vp, vp, vp, ctypes.c_int]),
            "amb_version": (ctypes.c_char_p, []),
            "amb_batch_create": (st, [vp, sz, vp, ctypes.POINTER(vp)]),
            "amb_batch_run": (st, [vp, ctypes.POINTER(amb_tune), ctypes.POINTER(ctypes.c_double)]),
            "amb_batch_population": (st, [vp, sz, ctypes.POINTER(vp)]),
            "amb_batch_info": (st, [vp, ctypes.POINTER(amb_batch_report)]),
            "amb_batch_destroy": (st, [vp]),
            "amb_job_bytes": (st, [ctypes.POINTER(amb_job), ctypes.POINTER(sz), ctypes.POINTER(sz)]),
            "amb_server_create": (st, [ctypes.POINTER(amb_server_config), vp, ctypes.POINTER(vp)]),
            "amb_server_submit": (st, [vp, ctypes.POINTER(amb_job), ctypes.c_int, ctypes.POINTER(u64)]),
            "amb_server_poll": (st, [vp, u64, ctypes.POINTER(amb_result)]),
            "amb_server_wait": (st, [vp, u64, ctypes.c_double, ctypes.POINTER(amb_result)]),
            "amb_server_counts": (st, [vp, u64, vp, sz, ctypes.POINTER(sz)]),
            "amb_server_read_column": (st, [vp, u64, ctypes.c_int, vp, sz]),
            "amb_server_release": (st, [vp, u64]),
            "amb_server_cancel": (st, [vp, u64]),
            "amb_debug_fail_creates": (st, [u32]),
            "amb_server_drain": (st, [vp, ctypes.c_double]),
            "amb_server_stats": (st, [vp, ctypes.POINTER(amb_server_report)]),
            "amb_server_destroy": (st, [vp]),
            "amb_table_create": (st, [u32, vp, ctypes.POINTER(vp)]),
            "amb_table_destroy": (st, [vp]),
            "amb_table_add_column": (st, [vp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]),
            "amb_table_find_column": (st, [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]),
            "amb_table_rows": (st, [vp, ctypes.POINTER(u32)]),
            "amb_table_write": (st, [vp, ctypes.c_int, vp, sz, ctypes.c_int]),
            "amb_table_read": (st, [vp, ctypes.c_int, vp, sz, ctypes.c_int]),
            "amb_table_map": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64]),
            "amb_table_map_col": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "amb_table_where": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(vp)]),
            "amb_view_from_ids": (st, [vp, vp, sz, ctypes.c_int, ctypes.POINTER(vp)]),
            "amb_view_draw": (st, [vp, u64, u32, u32, u32, u32, ctypes.c_int, ctypes.POINTER(vp)]),
            "amb_view_map": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64]),
            "amb_view_scatter_add": (st, [vp, ctypes.c_int, ctypes.c_int64]),
            "amb_view_where": (st, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(vp)]),
            "amb_view_scatter_add_values": (st, [vp, ctypes.c_int, vp, sz]),
            "amb_view_count": (st, [vp, ctypes.POINTER(sz)]),
            "amb_view_ids": (st, [vp, vp, sz, ctypes.c_int, ctypes.POINTER(sz)]),
            "amb_view_destroy": (st, [vp]),
            "amb_table_synchronize": (st, [vp]),
            "amb_log_create": (st, [vp, u32, ctypes.POINTER(vp)]),
            "amb_log_record": (st, [vp, ctypes.c_int, vp, vp, sz, ctypes.c_int]),
            "amb_log_pending": (st, [vp, ctypes.POINTER(sz)]),
            "amb_log_flush": (st, [vp]),
            "amb_log_destroy": (st, [vp]),
            "amb_debug_log_base": (st, [vp, u32]),
            "amb_table_grid_walk": (st, [vp, ctypes.POINTER(ctypes.c_int), u32, ctypes.POINTER(u32), ctypes.c_int,
                                         ctypes.c_int, u64, u32, u32, u32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != AMB_OK:
        raise AmbError(rc, (lib().amb_last_error() or b"").decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _buffer(a):
    """(pointer, on_device, element count, itemsize) of a torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):  # torch
        if not a.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a.numel(), a.element_size()
    a = np.asarray(a)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("buffer must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data), 0, a.size, a.itemsize


# ------------------------------------------------------------------ C names --
def amb_create(model, params, seed, replicate=0, stream=None):
    if isinstance(model, str):
        model = MODELS[model]
    if isinstance(params, dict):
        params = amb_params(**params)
    h = ctypes.c_void_p()
    _check(lib().amb_create(int(model), ctypes.byref(params), int(seed), int(replicate), _stream_handle(stream),
                            ctypes.byref(h)))
    return h


def amb_destroy(pop):
    _check(lib().amb_destroy(pop))


def amb_step(pop, k=1):
    _check(lib().amb_step(pop, int(k)))


def amb_write_column(pop, col, src):
    if isinstance(col, str):
        col = COLUMNS[col]
    p, dev, n, _ = _buffer(src)
    _check(lib().amb_write_column(pop, int(col), p, n, dev))


def amb_read_column(pop, col, dst):
    if isinstance(col, str):
        col = COLUMNS[col]
    p, dev, n, _ = _buffer(dst)
    _check(lib().amb_read_column(pop, int(col), p, n, dev))
    return dst


def amb_counts(pop, cap_rows=None):
    steps = int(lib().amb_step_index(pop))
    cap = steps if cap_rows is None else int(cap_rows)
    out = np.zeros((max(cap, 1), 4), dtype=np.int64)
    rows = ctypes.c_size_t()
    _check(lib().amb_counts(pop, ctypes.c_void_p(out.ctypes.data), cap, ctypes.byref(rows)))
    return out[:min(cap, rows.value)]


def amb_counts_range(pop, first, n_rows, out=None):
    if out is None:
        out = np.zeros((max(int(n_rows), 1), 4), dtype=np.int64)
    _check(lib().amb_counts_range(pop, int(first), int(n_rows), ctypes.c_void_p(out.ctypes.data)))
    return out[:int(n_rows)]


def amb_counts_async(pop, first, n_rows, out):
    """Queue a copy of count rows into `out` (pinned torch tensor or numpy
    array of n_rows x 4 int64); read it after amb_synchronize."""
    p, _, _, _ = _buffer(out)
    _check(lib().amb_counts_async(pop, int(first), int(n_rows), p))


def amb_launch_count(pop):
    return int(lib().amb_launch_count(pop))


def amb_read_index(pop, start, ids):
    ps, dev, _, _ = _buffer(start)
    pi, dev2, _, _ = _buffer(ids)
    if dev != dev2:
        raise ValueError("start and ids must both be on the device or both on the host")
    _check(lib().amb_read_index(pop, ps, pi, dev))
    return start, ids


def amb_invariants(pop, raise_on_violation=False):
    r = amb_invariant_report()
    rc = lib().amb_invariants(pop, ctypes.byref(r))
    if rc != AMB_OK and (rc != AMB_EINVARIANT or raise_on_violation):
        _check(rc)
    return {f: getattr(r, f) for f, _ in amb_invariant_report._fields_}


def amb_stats_compute(pop, hist_cap=1 << 16):
    s = amb_stats()
    hist = np.zeros(max(int(hist_cap), 1), dtype=np.int64)
    ln = ctypes.c_size_t()
    _check(lib().amb_stats_compute(pop, ctypes.byref(s), ctypes.c_void_p(hist.ctypes.data), int(hist_cap),
                                   ctypes.byref(ln)))
    d = {f: getattr(s, f) for f, _ in amb_stats._fields_}
    d["gini_numerator"] = (int(d["gini_num_hi"]) << 64) | int(d["gini_num_lo"])
    return d, hist[:min(ln.value, int(hist_cap))].copy()


def amb_occupancy(pop, occ):
    p, dev, _, _ = _buffer(occ)
    _check(lib().amb_occupancy(pop, p, dev))
    return occ


def amb_step_index(pop):
    return int(lib().amb_step_index(pop))


def amb_synchronize(pop):
    _check(lib().amb_synchronize(pop))


def amb_last_error():
    return (lib().amb_last_error() or b"").decode(errors="replace")


def amb_version():
    return lib().amb_version().decode()


def amb_sir_thresholds(beta, gamma, cap):
    cap = max(int(cap), 1)
    t = np.zeros(cap + 1, dtype=np.uint32)
    K = ctypes.c_uint32()
    tr = ctypes.c_uint32()
    _check(lib().amb_sir_thresholds(float(beta), float(gamma), cap, ctypes.c_void_p(t.ctypes.data),
                                    ctypes.byref(K), ctypes.byref(tr)))
    return t[:K.value + 1].copy(), int(tr.value)


def amb_cell_index(x, y, L, start, ids, stream=None, sync=True):
    px, _, n, _ = _buffer(x)
    py, _, _, _ = _buffer(y)
    ps, _, _, _ = _buffer(start)
    pi, _, _, _ = _buffer(ids)
    _check(lib().amb_cell_index(px, py, n, int(L), ps, pi, _stream_handle(stream), int(bool(sync))))
    return start, ids


def amb_cell_index_noalloc(x, y, L, start, ids, stream=None, sync=True):
    """amb_cell_index with its scratch in the library's static device array
    (no allocation; grids of at most 1,048,576 cells)."""
    px, _, n, _ = _buffer(x)
    py, _, _, _ = _buffer(y)
    ps, _, _, _ = _buffer(start)
    pi, _, _, _ = _buffer(ids)
    _check(lib().amb_cell_index_noalloc(px, py, n, int(L), ps, pi, _stream_handle(stream), int(bool(sync))))
    return start, ids


def make_job(model, n, seed, steps, rep=0, L=1, beta=0.0, gamma=0.0, n0=0, w_init=1):
    """amb_job from keyword arguments (the same names as Population)."""
    if isinstance(model, str):
        model = MODELS[model]
    return amb_job(model=int(model), params=amb_params(n=int(n), grid_side=int(L), beta=float(beta),
                                                       gamma=float(gamma), n_init_infected=int(n0),
                                                       w_init=int(w_init), variant=0),
                   seed=int(seed), replicate=int(rep), steps=int(steps))


def amb_batch_create(jobs, stream=None):
    arr = (amb_job * max(len(jobs), 1))(*jobs)
    h = ctypes.c_void_p()
    _check(lib().amb_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(jobs), _stream_handle(stream),
                                  ctypes.byref(h)))
    return h


def amb_batch_run(batch, band_rows_cap=0, autotune=False, use_graph=True, spread_bands=False):
    t = amb_tune(band_rows_cap=int(band_rows_cap), spread_bands=int(bool(spread_bands)), autotune=int(bool(autotune)),
                 use_graph=int(bool(use_graph)))
    ms = ctypes.c_double()
    _check(lib().amb_batch_run(batch, ctypes.byref(t), ctypes.byref(ms)))
    return ms.value


def amb_batch_population(batch, i):
    h = ctypes.c_void_p()
    _check(lib().amb_batch_population(batch, int(i), ctypes.byref(h)))
    return h


def amb_batch_info(batch):
    r = amb_batch_report()
    _check(lib().amb_batch_info(batch, ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in amb_batch_report._fields_}


def amb_batch_destroy(batch):
    _check(lib().amb_batch_destroy(batch))


def amb_job_bytes(job):
    """(resident, transient) device bytes of a job (host arithmetic only)."""
    r, t = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().amb_job_bytes(ctypes.byref(job), ctypes.byref(r), ctypes.byref(t)))
    return r.value, t.value


def _result_dict(r):
    return {"ticket": r.ticket, "status": r.status, "model": r.model, "n": r.n, "steps": r.steps,
            "last": list(r.last), "submit_s": r.submit_s, "admit_s": r.admit_s, "done_s": r.done_s}


def amb_server_create(hbm_budget_bytes, stream, max_active=0, chunk_steps=0, band_rows_cap=0, spread_bands=0,
                      iteration_us=0):
    cfg = amb_server_config(hbm_budget_bytes=int(hbm_budget_bytes), max_active=int(max_active),
                            chunk_steps=int(chunk_steps), band_rows_cap=int(band_rows_cap),
                            spread_bands=int(spread_bands), iteration_us=int(iteration_us))
    h = ctypes.c_void_p()
    _check(lib().amb_server_create(ctypes.byref(cfg), _stream_handle(stream), ctypes.byref(h)))
    return h


def amb_server_submit(server, job, keep_columns=False):
    t = ctypes.c_uint64()
    _check(lib().amb_server_submit(server, ctypes.byref(job), int(bool(keep_columns)), ctypes.byref(t)))
    return t.value


def amb_server_poll(server, ticket):
    """Result dict, or None while the job is queued or running."""
    r = amb_result()
    rc = lib().amb_server_poll(server, int(ticket), ctypes.byref(r))
    if rc == AMB_EBUSY:
        return None
    _check(rc)
    return _result_dict(r)


def amb_server_wait(server, ticket, timeout_s=60.0):
    r = amb_result()
    _check(lib().amb_server_wait(server, int(ticket), float(timeout_s), ctypes.byref(r)))
    return _result_dict(r)


def amb_server_counts(server, ticket, steps):
    out = np.zeros((max(int(steps), 1), 4), dtype=np.int64)
    rows = ctypes.c_size_t()
    _check(lib().amb_server_counts(server, int(ticket), ctypes.c_void_p(out.ctypes.data), int(steps),
                                   ctypes.byref(rows)))
    return out[:rows.value]


def amb_server_read_column(server, ticket, col, n):
    if isinstance(col, str):
        col = COLUMNS[col]
    out = np.zeros(int(n), dtype=np.uint8 if col == AMB_COL_STATE else np.int32)
    _check(lib().amb_server_read_column(server, int(ticket), int(col), ctypes.c_void_p(out.ctypes.data), int(n)))
    return out


def amb_server_release(server, ticket):
    _check(lib().amb_server_release(server, int(ticket)))


def amb_server_drain(server, timeout_s=600.0):
    _check(lib().amb_server_drain(server, float(timeout_s)))


def amb_server_stats(server):
    r = amb_server_report()
    _check(lib().amb_server_stats(server, ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in amb_server_report._fields_}


def amb_server_destroy(server):
    _check(lib().amb_server_destroy(server))


# --------------------------------------------------------------- convenience --
class Population:
    """Owning wrapper around an amb_pop handle (torch tensors for columns)."""

    def __init__(self, model, n, seed, rep=0, L=1, beta=0.0, gamma=0.0, n0=0, w_init=1, variant=0, stream=None):
        self.model = model
        self.n = int(n)
        self.L = int(L)
        self.params = amb_params(n=self.n, grid_side=self.L, beta=float(beta), gamma=float(gamma),
                                 n_init_infected=int(n0), w_init=int(w_init), variant=int(variant))
        self.handle = amb_create(model, self.params, seed, rep, stream)

    def close(self):
        if self.handle is not None and self.handle.value:
            amb_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, k=1):
        amb_step(self.handle, k)
        return self

    @property
    def t(self):
        return amb_step_index(self.handle)

    def set_step(self, t):
        _check(lib().amb_set_step(self.handle, int(t)))

    def column(self, name, device="cuda"):
        import torch
        dt = torch.uint8 if name == "state" else torch.int32
        out = torch.empty(self.n, dtype=dt, device=device)
        amb_read_column(self.handle, name, out)
        return out

    def write(self, name, values):
        amb_write_column(self.handle, name, values)

    def counts(self):
        return amb_counts(self.handle)

    def index(self, device="cuda"):
        import torch
        start = torch.empty(self.L * self.L + 1, dtype=torch.int32, device=device)
        ids = torch.empty(max(self.n, 1), dtype=torch.int32, device=device)[: self.n]
        amb_read_index(self.handle, start, ids)
        return start, ids

    def occupancy(self, device="cuda"):
        import torch
        occ = torch.empty(self.L * self.L, dtype=torch.int32, device=device)
        amb_occupancy(self.handle, occ)
        return occ

    def invariants(self):
        return amb_invariants(self.handle)

    def stats(self, hist_cap=1 << 16):
        return amb_stats_compute(self.handle, hist_cap)

    def synchronize(self):
        amb_synchronize(self.handle)


class PopulationView(Population):
    """Non-owning view of a population that belongs to a batch or server."""

    def __init__(self, handle, model, n, L=1):
        self.model = model
        self.n = int(n)
        self.L = int(L)
        self.handle = handle

    def close(self):
        self.handle = None


class Batch:
    """Owning wrapper around amb_batch: jobs are dicts of make_job keywords."""

    def __init__(self, jobs, stream=None):
        self.specs = [dict(j) for j in jobs]
        self.handle = amb_batch_create([make_job(**j) for j in self.specs], stream)

    def run(self, band_rows_cap=0, autotune=False, use_graph=True, spread_bands=False):
        return amb_batch_run(self.handle, band_rows_cap, autotune, use_graph, spread_bands)

    def info(self):
        return amb_batch_info(self.handle)

    def population(self, i):
        s = self.specs[i]
        return PopulationView(amb_batch_population(self.handle, i), s["model"], s["n"], s.get("L", 1))

    def close(self):
        if self.handle is not None and self.handle.value:
            amb_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owning wrapper around amb_server; jobs are dicts of make_job keywords."""

    def __init__(self, hbm_budget_bytes, stream, **cfg):
        self.handle = amb_server_create(hbm_budget_bytes, stream, **cfg)
        self.specs = {}

    def submit(self, job, keep_columns=False):
        t = amb_server_submit(self.handle, make_job(**job), keep_columns)
        self.specs[t] = dict(job)
        return t

    def poll(self, ticket):
        return amb_server_poll(self.handle, ticket)

    def wait(self, ticket, timeout_s=60.0):
        return amb_server_wait(self.handle, ticket, timeout_s)

    def counts(self, ticket):
        return amb_server_counts(self.handle, ticket, self.specs[ticket]["steps"])

    def column(self, ticket, name):
        return amb_server_read_column(self.handle, ticket, name, self.specs[ticket]["n"])

    def release(self, ticket):
        amb_server_release(self.handle, ticket)
        self.specs.pop(ticket, None)

    def cancel(self, ticket):
        _check(lib().amb_server_cancel(self.handle, int(ticket)))

    def drain(self, timeout_s=600.0):
        amb_server_drain(self.handle, timeout_s)

    def stats(self):
        return amb_server_stats(self.handle)

    def close(self):
        if self.handle is not None and self.handle.value:
            amb_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- view API ----
AMB_DT_I32, AMB_DT_U8 = 0, 1
DTYPES = {"i32": AMB_DT_I32, "int32": AMB_DT_I32, "u8": AMB_DT_U8, "uint8": AMB_DT_U8}
OPS = {"set": 0, "add": 1, "sub": 2, "mul": 3, "min": 4, "max": 5}
CMPS = {"==": 0, "!=": 1, "<": 2, "<=": 3, ">": 4, ">=": 5}


class Table:
    """A device-resident columnar table (amb_table) with named int32 / uint8
    columns; the view API of the paper (Sec. 3.1, 3.3) on top of it."""

    def __init__(self, n, stream=None):
        self.n = int(n)
        h = ctypes.c_void_p()
        _check(lib().amb_table_create(self.n, _stream_handle(stream), ctypes.byref(h)))
        self.handle = h
        self.dtypes = {}

    def add_column(self, name, dtype="i32", fill=0):
        c = ctypes.c_int()
        _check(lib().amb_table_add_column(self.handle, name.encode(), DTYPES[dtype], int(fill), ctypes.byref(c)))
        self.dtypes[name] = DTYPES[dtype]
        return c.value

    def col(self, name):
        c = ctypes.c_int()
        _check(lib().amb_table_find_column(self.handle, name.encode(), ctypes.byref(c)))
        return c.value

    def write(self, name, values):
        p, dev, n, _ = _buffer(values)
        _check(lib().amb_table_write(self.handle, self.col(name), p, n, dev))

    def read(self, name, device="cpu"):
        import torch
        dt = torch.uint8 if self.dtypes[name] == AMB_DT_U8 else torch.int32
        out = torch.empty(self.n, dtype=dt, device=device)
        p, dev, n, _ = _buffer(out)
        _check(lib().amb_table_read(self.handle, self.col(name), p, n, dev))
        return out

    def map(self, name, op, scalar):
        """Full-population view: column OP= scalar."""
        _check(lib().amb_table_map(self.handle, self.col(name), OPS[op], int(scalar)))

    def map_col(self, dst, op, src):
        _check(lib().amb_table_map_col(self.handle, self.col(dst), OPS[op], self.col(src)))

    def where(self, name, cmp, scalar):
        """Filtered view of the ids with column CMP scalar (ascending)."""
        h = ctypes.c_void_p()
        _check(lib().amb_table_where(self.handle, self.col(name), CMPS[cmp], int(scalar), ctypes.byref(h)))
        return View(self, h)

    def at(self, ids):
        """Scatter view of the given ids (repeats allowed)."""
        p, dev, n, _ = _buffer(ids)
        h = ctypes.c_void_p()
        _check(lib().amb_view_from_ids(self.handle, p, n, dev, ctypes.byref(h)))
        return View(self, h)

    def synchronize(self):
        _check(lib().amb_table_synchronize(self.handle))

    def log(self, capacity):
        """A buffered-write log of this table (Log)."""
        return Log(self, capacity)

    def grid_walk(self, cols, sizes, moore=True, torus=True, seed=0, rep=0, step=0, steps=1):
        """`steps` grid-walk steps on the int32 coordinate columns `cols`."""
        d = len(cols)
        c = (ctypes.c_int * d)(*[self.col(x) for x in cols])
        sz = (ctypes.c_uint32 * d)(*[int(v) for v in sizes])
        _check(lib().amb_table_grid_walk(self.handle, c, d, sz, int(bool(moore)), int(bool(torus)), int(seed), int(rep),
                                         int(step), int(steps)))

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().amb_table_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class View:
    """A filtered or scatter view of a Table (amb_view)."""

    def __init__(self, table, handle):
        self.table = table
        self.handle = handle

    def map(self, name, op, scalar):
        _check(lib().amb_view_map(self.handle, self.table.col(name), OPS[op], int(scalar)))
        return self

    def scatter_add(self, name, value):
        """scatter_add with one value for every listed id, or with a device
        int32 tensor of per-entry values."""
        if hasattr(value, "data_ptr"):
            p, dev, k, _ = _buffer(value)
            if not dev:
                raise ValueError("per-entry values must be a device tensor")
            _check(lib().amb_view_scatter_add_values(self.handle, self.table.col(name), p, k))
        else:
            _check(lib().amb_view_scatter_add(self.handle, self.table.col(name), int(value)))
        return self

    def where(self, name, cmp, scalar):
        """The listed ids whose value satisfies name CMP scalar (a view)."""
        h = ctypes.c_void_p()
        _check(lib().amb_view_where(self.handle, self.table.col(name), CMPS[cmp], int(scalar), ctypes.byref(h)))
        return View(self.table, h)

    def draw(self, seed, rep, step, word=0, rng=None, exclude_self=True):
        h = ctypes.c_void_p()
        rng = self.table.n if rng is None else rng
        _check(lib().amb_view_draw(self.handle, int(seed), int(rep), int(step), int(word), int(rng),
                                   int(bool(exclude_self)), ctypes.byref(h)))
        return View(self.table, h)

    def count(self):
        k = ctypes.c_size_t()
        _check(lib().amb_view_count(self.handle, ctypes.byref(k)))
        return k.value

    def ids(self):
        k = self.count()
        out = np.zeros(max(k, 1), dtype=np.int32)
        got = ctypes.c_size_t()
        _check(lib().amb_view_ids(self.handle, ctypes.c_void_p(out.ctypes.data), k, 0, ctypes.byref(got)))
        return out[:got.value]

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().amb_view_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class CPopulation(Population):
    """Continuous-space population ("cwalk" / "csir"): float32 x, y in
    [0, w] x [0, h]; see amb_create_continuous."""

    def __init__(self, model, n, seed, rep=0, w=100.0, h=100.0, s=1.0, r=5.0, p=0.1, rec_steps=14, n0=5,
                 stream=None):
        self.model = model
        self.n = int(n)
        self.L = 0
        self.cparams = amb_cparams(n=self.n, width=float(w), height=float(h), step=float(s), radius=float(r),
                                   p_infect=float(p), recovery_steps=int(rec_steps), n_init_infected=int(n0))
        h_ = ctypes.c_void_p()
        _check(lib().amb_create_continuous(MODELS[model], ctypes.byref(self.cparams), int(seed), int(rep),
                                           _stream_handle(stream), ctypes.byref(h_)))
        self.handle = h_

    def column(self, name, device="cuda"):
        import torch
        dt = {"x": torch.float32, "y": torch.float32, "state": torch.uint8, "days": torch.int32}[name]
        out = torch.empty(self.n, dtype=dt, device=device)
        amb_read_column(self.handle, name, out)
        return out


class Log:
    """Buffered per-agent writes of a Table (amb_log): record, then flush once."""

    def __init__(self, table, capacity):
        self.table = table
        h = ctypes.c_void_p()
        _check(lib().amb_log_create(table.handle, int(capacity), ctypes.byref(h)))
        self.handle = h

    def record(self, name, ids, values):
        if hasattr(ids, "data_ptr"):
            pi, dev, k, _ = _buffer(ids)
            pv, dev2, k2, _ = _buffer(values)
            if dev != dev2 or k != k2:
                raise ValueError("ids and values must have the same length and location")
        else:
            ids = np.ascontiguousarray(ids, dtype=np.int32)
            values = np.ascontiguousarray(values, dtype=np.int64)
            if ids.size != values.size:
                raise ValueError("ids and values must have the same length")
            pi, pv, k, dev = ctypes.c_void_p(ids.ctypes.data), ctypes.c_void_p(values.ctypes.data), ids.size, 0
        _check(lib().amb_log_record(self.handle, self.table.col(name), pi, pv, k, dev))

    def pending(self):
        k = ctypes.c_size_t()
        _check(lib().amb_log_pending(self.handle, ctypes.byref(k)))
        return k.value

    def flush(self):
        _check(lib().amb_log_flush(self.handle))

    def debug_base(self, base):
        """Test hook: the number of the next record (see amb_debug_log_base)."""
        _check(lib().amb_debug_log_base(self.handle, int(base)))

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().amb_log_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def amb_debug_fail_creates(k):
    """Test hook: the next k population creations fail with AMB_ENOMEM."""
    _check(lib().amb_debug_fail_creates(int(k)))
