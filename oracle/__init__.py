"""Parity oracle: ctypes front end of the single-threaded C statement of the
AMBER update rules (oracle/amb_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this package.  The CUDA
library never calls it, and it never calls the CUDA library.

Each function states the passage of the paper it follows:
  * wealth transfer: Sec. 5.1.2 and Listings 2-3 (filtered debit, scatter_add
    credit to a random other agent), invariant of Sec. 5.1.3;
  * random walk: Sec. 5.1.2 (re-cast as Moore moves on an integer torus,
    grid environment of Sec. 4.1);
  * spatial SIR: Sec. 5.1.2 (re-cast as same-cell contacts on the grid),
    invariants of Sec. 5.1.3;
  * synchronous snapshot semantics: Sec. 3.4;
  * counting-sort cell index: grid environment, Sec. 4.1.
"""
import ctypes
import os

import numpy as np

from . import build as _build

S, I, R = 0, 1, 2
INIT_STEP = 0xFFFFFFFF

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u64 = ctypes.c_uint64
        u32 = ctypes.c_uint32
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_init_wealth.argtypes = [u32, ctypes.c_int32, i32p]
        L.orc_init_wealth.restype = None
        L.orc_init_positions.argtypes = [u32, u32, u32, u32, i32p, i32p]
        L.orc_init_positions.restype = None
        L.orc_init_sir_state.argtypes = [u32, u32, u8p]
        L.orc_init_sir_state.restype = None
        L.orc_wealth_step.argtypes = [u32, u32, u32, u32, i32p, i64p]
        L.orc_walk_step.argtypes = [u32, u32, u32, u32, u32, i32p, i32p]
        L.orc_sir_thresholds.argtypes = [ctypes.c_double, ctypes.c_double, u32, u32p, u32p, u32p]
        L.orc_sir_step.argtypes = [u32, u32, u32, u32, u32, u32p, u32, u32, i32p, i32p, u8p, i64p]
        L.orc_cell_index.argtypes = [u32, u32, i32p, i32p, i64p, i32p]
        L.orc_occupancy.argtypes = [u32, u32, i32p, i32p, i32p, i64p, u32]
        L.orc_gini.argtypes = [u32, i32p, ctypes.POINTER(ctypes.c_double), i64p,
                               ctypes.POINTER(u64), i64p]
        L.orc_curve_moments.argtypes = [i64p, u32, i64p, u32p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        L.orc_col_map.argtypes = [ctypes.c_int, vp, u32, ctypes.c_int, i64]
        L.orc_col_map_col.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, u32, ctypes.c_int]
        L.orc_where.argtypes = [ctypes.c_int, vp, u32, ctypes.c_int, i64, i32p, u32p]
        L.orc_view_map.argtypes = [ctypes.c_int, vp, u32, i32p, u32, ctypes.c_int, i64]
        L.orc_view_draw.argtypes = [i32p, u32, u32, u32, u32, u32, u32, ctypes.c_int, i32p]
        f32p, f32 = ctypes.POINTER(ctypes.c_float), ctypes.c_float
        L.orc_cinit_positions.argtypes = [u32, f32, f32, u32, u32, f32p, f32p]
        L.orc_cinit_positions.restype = None
        L.orc_cwalk_step.argtypes = [u32, f32, f32, f32, u32, u32, u32, f32p, f32p]
        L.orc_csir_step.argtypes = [u32, f32, f32, f32, f32, u32, u32, u32, u32p, u32, u32, f32p, f32p, u8p, i32p, i64p]
        L.orc_log_flush.argtypes = [ctypes.c_int, vp, u32, i32p, i64p, u32]
        L.orc_view_where.argtypes = [ctypes.c_int, vp, u32, i32p, u32, ctypes.c_int, i64, i32p, u32p]
        L.orc_view_add_values.argtypes = [ctypes.c_int, vp, u32, i32p, i32p, u32]
        L.orc_grid_walk_step.argtypes = [u32, u32p, ctypes.c_int, ctypes.c_int, u32, ctypes.POINTER(i32p), u32, u32,
                                         u32]
        for f in ("orc_view_where", "orc_view_add_values", "orc_log_flush", "orc_grid_walk_step", "orc_cwalk_step", "orc_csir_step", "orc_col_map", "orc_col_map_col", "orc_where", "orc_view_map", "orc_view_draw",
                  "orc_wealth_step", "orc_walk_step", "orc_sir_thresholds", "orc_sir_step",
                  "orc_cell_index", "orc_occupancy", "orc_gini", "orc_curve_moments"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: counter (4 x uint32), key (2 x uint32) -> 4 x uint32."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def sir_thresholds(beta, gamma, n):
    """(t_inf[0..K], t_rec) for infection probability 1-(1-beta)^k and recovery gamma."""
    cap = max(int(n), 1)
    t_inf = np.zeros(cap + 1, dtype=np.uint32)
    K = np.zeros(1, dtype=np.uint32)
    t_rec = np.zeros(1, dtype=np.uint32)
    _check(lib().orc_sir_thresholds(float(beta), float(gamma), cap, _p(t_inf, ctypes.c_uint32),
                                    _p(K, ctypes.c_uint32), _p(t_rec, ctypes.c_uint32)),
           "sir_thresholds")
    return t_inf[: int(K[0]) + 1].copy(), int(t_rec[0])


def cell_index(x, y, L):
    """Stable counting sort by cell c = y*L + x: (start[C+1] int64, perm[n] int32)."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    n = x.size
    C = int(L) * int(L)
    start = np.zeros(C + 1, dtype=np.int64)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().orc_cell_index(n, int(L), _p(x, ctypes.c_int32), _p(y, ctypes.c_int32),
                                _p(start, ctypes.c_int64), _p(perm, ctypes.c_int32)), "cell_index")
    return start, perm[:n]


def occupancy(x, y, L, hist_len=64):
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    C = int(L) * int(L)
    occ = np.zeros(C, dtype=np.int32)
    hist = np.zeros(hist_len, dtype=np.int64)
    _check(lib().orc_occupancy(x.size, int(L), _p(x, ctypes.c_int32), _p(y, ctypes.c_int32),
                               _p(occ, ctypes.c_int32), _p(hist, ctypes.c_int64), hist_len),
           "occupancy")
    return occ, hist


def gini(w):
    """Gini coefficient and its exact integer numerator / total."""
    w = np.ascontiguousarray(w, dtype=np.int32)
    g = ctypes.c_double()
    hi = np.zeros(1, dtype=np.int64)
    lo = ctypes.c_uint64()
    tot = np.zeros(1, dtype=np.int64)
    _check(lib().orc_gini(w.size, _p(w, ctypes.c_int32), ctypes.byref(g), _p(hi, ctypes.c_int64),
                          ctypes.byref(lo), _p(tot, ctypes.c_int64)), "gini")
    num = (int(hi[0]) << 64) | int(lo.value)
    return g.value, num, int(tot[0])


def curve_moments(infected):
    """(peak, argmax step, mean, variance) of t weighted by I(t), t = 1..T."""
    a = np.ascontiguousarray(infected, dtype=np.int64)
    pk = np.zeros(1, dtype=np.int64)
    am = np.zeros(1, dtype=np.uint32)
    mean = ctypes.c_double()
    var = ctypes.c_double()
    _check(lib().orc_curve_moments(_p(a, ctypes.c_int64), a.size, _p(pk, ctypes.c_int64),
                                   _p(am, ctypes.c_uint32), ctypes.byref(mean), ctypes.byref(var)),
           "curve_moments")
    return int(pk[0]), int(am[0]), mean.value, var.value


class Population:
    """One oracle population: columns in id order, advanced one step at a time.

    model: "wealth" | "walk" | "sir".  Per-step counts are recorded in
    ``series`` (one row of 4 int64 per step): wealth {donors, total wealth},
    SIR {S, I, R, new infections}, walk {agent count}.
    """

    def __init__(self, model, n, seed, rep=0, L=1, beta=0.0, gamma=0.0, n0=0, w_init=1):
        self.model = model
        self.n = int(n)
        self.L = int(L)
        self.seed = int(seed)
        self.rep = int(rep)
        self.t = 0
        self.series = []
        Lb = lib()
        if model == "wealth":
            self.w = np.zeros(self.n, dtype=np.int32)
            Lb.orc_init_wealth(self.n, int(w_init), _p(self.w, ctypes.c_int32))
        elif model in ("walk", "sir"):
            self.x = np.zeros(self.n, dtype=np.int32)
            self.y = np.zeros(self.n, dtype=np.int32)
            Lb.orc_init_positions(self.n, self.L, self.seed, self.rep,
                                  _p(self.x, ctypes.c_int32), _p(self.y, ctypes.c_int32))
            if model == "sir":
                self.state = np.zeros(self.n, dtype=np.uint8)
                Lb.orc_init_sir_state(self.n, int(n0), _p(self.state, ctypes.c_uint8))
                self.t_inf, self.t_rec = sir_thresholds(beta, gamma, self.n)
                self.K = self.t_inf.size - 1
        else:
            raise ValueError("unknown model %r" % (model,))

    def step(self, k=1):
        Lb = lib()
        cnt = np.zeros(4, dtype=np.int64)
        for _ in range(int(k)):
            if self.model == "wealth":
                _check(Lb.orc_wealth_step(self.n, self.seed, self.rep, self.t,
                                          _p(self.w, ctypes.c_int32), _p(cnt, ctypes.c_int64)),
                       "wealth_step")
            elif self.model == "walk":
                _check(Lb.orc_walk_step(self.n, self.L, self.seed, self.rep, self.t,
                                        _p(self.x, ctypes.c_int32), _p(self.y, ctypes.c_int32)),
                       "walk_step")
                # the walk's count row is the agent count, which never changes
                cnt[:] = (self.n, 0, 0, 0)
            else:
                _check(Lb.orc_sir_step(self.n, self.L, self.seed, self.rep, self.t,
                                       _p(self.t_inf, ctypes.c_uint32), self.K, self.t_rec,
                                       _p(self.x, ctypes.c_int32), _p(self.y, ctypes.c_int32),
                                       _p(self.state, ctypes.c_uint8), _p(cnt, ctypes.c_int64)),
                       "sir_step")
            self.series.append(cnt.copy())
            self.t += 1
        return self

    def counts(self):
        return np.array(self.series, dtype=np.int64).reshape(-1, 4)


# ------------------------------------------------------------- view API ----
OPS = {"set": 0, "add": 1, "sub": 2, "mul": 3, "min": 4, "max": 5}
CMPS = {"==": 0, "!=": 1, "<": 2, "<=": 3, ">": 4, ">=": 5}


def _dtype_code(a):
    if a.dtype == np.int32:
        return 0
    if a.dtype == np.uint8:
        return 1
    raise ValueError("columns are int32 or uint8")


def col_map(col, op, s):
    """Full-population view update, in place: col = col OP s."""
    col = np.ascontiguousarray(col)
    _check(lib().orc_col_map(_dtype_code(col), col.ctypes.data, col.size, OPS[op], int(s)), "col_map")
    return col


def col_map_col(dst, op, src):
    """dst = dst OP src, elementwise, in place."""
    _check(lib().orc_col_map_col(_dtype_code(dst), dst.ctypes.data, _dtype_code(src), src.ctypes.data, dst.size,
                                 OPS[op]), "col_map_col")
    return dst


def where(col, cmp, s):
    """Filtered view: ascending ids with col CMP s."""
    ids = np.zeros(max(col.size, 1), dtype=np.int32)
    k = np.zeros(1, dtype=np.uint32)
    _check(lib().orc_where(_dtype_code(col), col.ctypes.data, col.size, CMPS[cmp], int(s), _p(ids, ctypes.c_int32),
                           _p(k, ctypes.c_uint32)), "where")
    return ids[:int(k[0])]


def view_map(col, ids, op, s):
    """Update through a view (ids may repeat; applied once per occurrence)."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    _check(lib().orc_view_map(_dtype_code(col), col.ctypes.data, col.size, _p(ids, ctypes.c_int32), ids.size,
                              OPS[op], int(s)), "view_map")
    return col


def view_draw(ids, seed, rep, step, word, rng, exclude_self):
    """One random id per listed id (counter-based; see orc_view_draw)."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    out = np.zeros(max(ids.size, 1), dtype=np.int32)
    _check(lib().orc_view_draw(_p(ids, ctypes.c_int32), ids.size, int(seed), int(rep), int(step), int(word), int(rng),
                               int(bool(exclude_self)), _p(out, ctypes.c_int32)), "view_draw")
    return out[:ids.size]


# ------------------------------------------------------ continuous space ----
class CPopulation:
    """Oracle population of the continuous-space models ("cwalk", "csir"):
    float32 positions in [0, w] x [0, h]; see orc_cwalk_step / orc_csir_step."""

    def __init__(self, model, n, seed, rep=0, w=100.0, h=100.0, s=1.0, r=5.0, p=0.1, rec_steps=14, n0=5):
        if model not in ("cwalk", "csir"):
            raise ValueError(model)
        self.model, self.n, self.seed, self.rep = model, int(n), int(seed), int(rep)
        self.w, self.h, self.s, self.r = float(w), float(h), float(s), float(r)
        self.rec_steps = int(rec_steps)
        self.t = 0
        self.series = []
        self.x = np.zeros(self.n, dtype=np.float32)
        self.y = np.zeros(self.n, dtype=np.float32)
        lib().orc_cinit_positions(self.n, self.w, self.h, self.seed, self.rep, _p(self.x, ctypes.c_float),
                                  _p(self.y, ctypes.c_float))
        if model == "csir":
            self.state = np.zeros(self.n, dtype=np.uint8)
            lib().orc_init_sir_state(self.n, int(n0), _p(self.state, ctypes.c_uint8))
            self.days = np.zeros(self.n, dtype=np.int32)
            self.t_inf, _ = sir_thresholds(p, 0.0, self.n)
            self.K = self.t_inf.size - 1

    def step(self, k=1):
        cnt = np.zeros(4, dtype=np.int64)
        for _ in range(int(k)):
            if self.model == "cwalk":
                _check(lib().orc_cwalk_step(self.n, self.w, self.h, self.s, self.seed, self.rep, self.t,
                                            _p(self.x, ctypes.c_float), _p(self.y, ctypes.c_float)), "cwalk_step")
                cnt[:] = (self.n, 0, 0, 0)
            else:
                _check(lib().orc_csir_step(self.n, self.w, self.h, self.s, self.r, self.seed, self.rep, self.t,
                                           _p(self.t_inf, ctypes.c_uint32), self.K, self.rec_steps,
                                           _p(self.x, ctypes.c_float), _p(self.y, ctypes.c_float),
                                           _p(self.state, ctypes.c_uint8), _p(self.days, ctypes.c_int32),
                                           _p(cnt, ctypes.c_int64)), "csir_step")
            self.series.append(cnt.copy())
            self.t += 1
        return self

    def counts(self):
        return np.array(self.series, dtype=np.int64).reshape(-1, 4)


# ------------------------------------------------------ buffered writes ----
def log_flush(col, ids, values):
    """Apply recorded writes (ids[j], values[j]) in order: the last per row wins."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    values = np.ascontiguousarray(values, dtype=np.int64)
    _check(lib().orc_log_flush(_dtype_code(col), col.ctypes.data, col.size, _p(ids, ctypes.c_int32),
                               _p(values, ctypes.c_int64), ids.size), "log_flush")
    return col


# ---------------------------------------------------------- grid walks ----
def grid_walk_step(coords, sizes, moore, torus, seed, rep, t):
    """One step of the d-dimensional grid walk on the int32 coordinate arrays
    (modified in place; see orc_grid_walk_step)."""
    d = len(coords)
    sz = np.ascontiguousarray(sizes, dtype=np.uint32)
    arrs = [np.ascontiguousarray(c, dtype=np.int32) for c in coords]
    ptrs = (ctypes.POINTER(ctypes.c_int32) * d)(*[_p(a, ctypes.c_int32) for a in arrs])
    n = arrs[0].size if d else 0
    _check(lib().orc_grid_walk_step(d, _p(sz, ctypes.c_uint32), int(bool(moore)), int(bool(torus)), n, ptrs,
                                    int(seed), int(rep), int(t)), "grid_walk_step")
    for c, a in zip(coords, arrs):
        if c is not a:
            c[:] = a
    return coords


def view_where(col, ids, cmp, s):
    """The listed ids (list order, repeats kept) with col[id] CMP s."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    out = np.zeros(max(ids.size, 1), dtype=np.int32)
    k = np.zeros(1, dtype=np.uint32)
    _check(lib().orc_view_where(_dtype_code(col), col.ctypes.data, col.size, _p(ids, ctypes.c_int32), ids.size,
                                CMPS[cmp], int(s), _p(out, ctypes.c_int32), _p(k, ctypes.c_uint32)), "view_where")
    return out[:int(k[0])]


def view_add_values(col, ids, values):
    """col[ids[j]] += values[j] for every j (repeats accumulate)."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    values = np.ascontiguousarray(values, dtype=np.int32)
    _check(lib().orc_view_add_values(_dtype_code(col), col.ctypes.data, col.size, _p(ids, ctypes.c_int32),
                                     _p(values, ctypes.c_int32), ids.size), "view_add_values")
    return col
