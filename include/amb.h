/*
 * amb.h -- C ABI of the GB300 columnar agent-step engine.
 *
 * The engine runs the per-step population update that AMBER's view API
 * lowers to column operations (paper Sec. 3.1-3.4): full-population maps,
 * predicate-filtered (masked) updates and id-indexed scatter-adds over a
 * struct-of-arrays agent table, for the paper's three benchmark models
 * (Sec. 5.1.2): wealth transfer, random walk (on an integer torus grid) and
 * spatial SIR (same-cell contacts on the grid, with the grid's counting-sort
 * cell index rebuilt every step, Sec. 4.1).
 *
 * Conventions for every call:
 *  - Every function returns an amb_status and never aborts, traps or exits.
 *    On failure amb_last_error() returns a message (thread-local, valid until
 *    the next failing call on the same thread).
 *  - The library owns all device memory it allocates (stream-ordered, on the
 *    population's stream) and frees it in amb_destroy.  Callers own every
 *    buffer they pass; no pointer is kept after a call returns.
 *  - "on_device" buffers are device pointers of the current CUDA device;
 *    otherwise host pointers (pinned or pageable).
 *  - Agents are identified by their id 0..n-1; every column read or written
 *    through this ABI is in id order, whatever the internal layout.
 *  - One population per host thread at a time; the server object is
 *    internally synchronised.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *    (seed, replicate) and counter (agent id, step, 0, 0); seeds are 32-bit.
 *    Initial positions use step 0xFFFFFFFF, so at most 2^32 - 2 steps.
 */
#ifndef AMB_H
#define AMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMB_OK = 0,
    AMB_EINVAL = 1,      /* bad argument; nothing was changed */
    AMB_ENOMEM = 2,      /* device or host allocation failed */
    AMB_ECUDA = 3,       /* a CUDA call failed (message has the CUDA error) */
    AMB_EINVARIANT = 4,  /* an invariant check failed (see the report) */
    AMB_ETIMEOUT = 5,    /* a bounded device-side wait ran out; results invalid */
    AMB_EBUSY = 6,       /* server: job not finished yet */
    AMB_EBUDGET = 7,     /* server: job can never fit in the HBM budget */
    AMB_ENOTFOUND = 8,   /* server: unknown ticket */
    AMB_ECANCELED = 9    /* server: the job was cancelled */
} amb_status;

typedef enum {
    AMB_WEALTH = 0, /* wealth transfer */
    AMB_WALK = 1,   /* random walk on an integer torus grid */
    AMB_SIR = 2,    /* spatial SIR, same-cell contacts on the grid */
    AMB_CWALK = 3,  /* random walk in continuous space (amb_create_continuous) */
    AMB_CSIR = 4    /* SIR in continuous space, radius contacts (amb_create_continuous) */
} amb_model;

typedef enum {
    AMB_COL_WEALTH = 0, /* int32, wealth model */
    AMB_COL_X = 1,      /* int32 in [0, L), walk and SIR */
    AMB_COL_Y = 2,      /* int32 in [0, L), walk and SIR */
    AMB_COL_STATE = 3,  /* uint8: AMB_S, AMB_I or AMB_R, SIR */
    AMB_COL_DAYS = 4    /* int32: steps spent infected, continuous SIR */
} amb_col;

enum { AMB_S = 0, AMB_I = 1, AMB_R = 2 };

/* Execution path of the SIR step (amb_params.variant). */
enum {
    AMB_SIR_AUTO = 0,    /* band path when the grid allows it, else generic */
    AMB_SIR_GENERIC = 1, /* id-ordered columns, global counting sort each step */
    AMB_SIR_BAND = 2,    /* cell-ordered records, one fused kernel per step */
    AMB_SIR_BAND32 = 3,  /* band path with 32-bit per-cell counters in shared memory */
    AMB_SIR_BAND16 = 4   /* band path with 16-bit per-cell counters (bands twice as tall; a band whose counts
                            do not fit is redone with 32-bit counters); L a multiple of 8, at most 8192.
                            AMB_SIR_BAND and AMB_SIR_AUTO take 16-bit counters when that needs fewer waves
                            of bands and rows hold at most 3,072 agents on average */
};

typedef struct {
    uint32_t n;               /* number of agents (0 allowed) */
    uint32_t grid_side;       /* L: the grid is L x L cells (walk, SIR); >= 1 */
    double beta;              /* SIR: per infected cell-mate infection probability, [0,1] */
    double gamma;             /* SIR: per-step recovery probability, [0,1] */
    uint32_t n_init_infected; /* SIR: agents 0 .. n0-1 start infected (n0 <= n) */
    int32_t w_init;           /* wealth: initial wealth of every agent */
    uint32_t variant;         /* SIR execution path, AMB_SIR_*; 0 = automatic */
} amb_params;

typedef struct amb_pop amb_pop;

/*
 * Create a population of p->n agents (paper Sec. 3.3, add_agents: one call
 * creates all agents column by column).  Wealth: every agent holds w_init.
 * Walk / SIR: positions uniform on the torus, x = hi32(u0 * L),
 * y = hi32(u1 * L) with u = Philox(key, (id, 0xFFFFFFFF, 0, 0)); SIR: agents
 * 0 .. n0-1 infected, the rest susceptible.  cuda_stream (a cudaStream_t, may
 * be NULL for the legacy default stream) orders every later operation on the
 * population.  Grid limits: walk L <= 2^31 - 1; SIR L <= 46340 (L*L < 2^31).
 * seed must be < 2^32.  On success *out owns device memory until
 * amb_destroy.
 */
amb_status amb_create(amb_model model, const amb_params *p, uint64_t seed, uint32_t replicate,
                      void *cuda_stream, amb_pop **out);

/*
 * Continuous-space models as the paper states them (Sec. 5.1.2): agents in
 * the box [0, width] x [0, height] with float32 positions (columns X and Y
 * are float32 for these models).
 *  AMB_CWALK: every step dx, dy = step * sunit(u0), step * sunit(u1), then
 *    the position is clamped to the box.
 *  AMB_CSIR: (with step > 0, every agent first moves as in AMB_CWALK); a
 *    susceptible agent with k agents infected at the start of the step within
 *    distance radius becomes infected iff u2 < T_inf[min(k, K)], T_inf the
 *    thresholds of 1 - (1 - p_infect)^k (as for AMB_SIR); an agent infected at
 *    the start of the step counts one more step infected (column DAYS) and
 *    recovers when that count reaches recovery_steps.  Agents 0 .. n0-1 start
 *    infected.
 * Float arithmetic, each operation one IEEE single-precision operation
 * rounded to nearest: unit(u) = (u >> 8) 2^-24, sunit(u) = ((u >> 8) - 2^23)
 * 2^-23; initial x = width * unit(u0), y = height * unit(u1) (step
 * 0xFFFFFFFF); contact iff (xi - xj)^2 + (yi - yj)^2 <= radius * radius,
 * evaluated in that order.  Per-step counts: CWALK {n, 0, 0, 0}; CSIR
 * {S, I, R, new infections}.
 */
typedef struct {
    uint32_t n;
    float width, height;       /* box; >= 0 */
    float step;                /* displacement half-width s >= 0 (0: SIR agents do not move) */
    float radius;              /* CSIR contact radius >= 0 */
    double p_infect;           /* CSIR per-contact infection probability in [0, 1] */
    uint32_t recovery_steps;   /* CSIR: >= 1 */
    uint32_t n_init_infected;  /* CSIR: <= n */
} amb_cparams;

amb_status amb_create_continuous(amb_model model, const amb_cparams *p, uint64_t seed, uint32_t replicate,
                                 void *cuda_stream, amb_pop **out);

/* Set the step index to t (checkpoint / resume): the next amb_step runs step
 * t with the draws of step t.  Because every random draw is keyed by (seed,
 * replicate, agent id, step), a population created with the same seed and
 * replicate, given the columns read from another one after t steps
 * (amb_write_column) and set to step t, continues bit-identically.  Count rows
 * of steps not run by this population read as zeros; the invariant checks
 * start at step t.  Synchronises. */
amb_status amb_set_step(amb_pop *pop, uint64_t t);

/* Free everything the population owns (stream-ordered), then synchronise. */
amb_status amb_destroy(amb_pop *pop);

/*
 * Advance k synchronous steps (paper Sec. 3.4: every agent reads the state
 * of the start of the step).  Asynchronous on the population's stream.
 *  wealth (Sec. 5.1.2, Listings 2-3): donors = agents with wealth > 0; each
 *    gives one unit to r = r' + (r' >= id), r' = hi32(u0 * (n-1)); credits
 *    from several donors add up.  n == 1: nothing happens.
 *  walk: direction d = u0 >> 29 selects one of the 8 Moore neighbours
 *    (dx,dy) = (-1,-1) (0,-1) (1,-1) (-1,0) (1,0) (-1,1) (0,1) (1,1); coordinates
 *    wrap on the torus.
 *  SIR: every agent moves as in the walk; k = number of agents infected at
 *    the start of the step whose new cell is the same; a susceptible agent
 *    becomes infected iff k >= 1 and u1 < T_inf[min(k, K)]; an agent infected
 *    at the start of the step recovers iff u2 < T_rec; the cell index is
 *    rebuilt for the new positions.
 * Per-step counts are recorded on the device (amb_counts).
 */
amb_status amb_step(amb_pop *pop, uint32_t k);

/* Overwrite one column with n == p->n values in id order (host or device).
 * SIR states must be 0, 1 or 2 and positions in [0, L) (checked on the device;
 * violations return AMB_EINVAL and leave the population unchanged). */
amb_status amb_write_column(amb_pop *pop, amb_col col, const void *src, size_t n, int src_on_device);

/* Copy one column (id order) into dst (n == p->n elements).  Synchronises the
 * population's stream; reports a device-side error raised by earlier steps. */
amb_status amb_read_column(amb_pop *pop, amb_col col, void *dst, size_t n, int dst_on_device);

/*
 * Per-step counts, 4 int64 per step, rows 0 .. steps-1 (host buffer):
 *   wealth {donors, total wealth after the step, 0, 0}
 *   walk   {n, 0, 0, 0}
 *   SIR    {S, I, R, new infections} after the step.
 * Copies min(cap_rows, steps) rows; *rows_out = steps done.  Synchronises.
 */
amb_status amb_counts(amb_pop *pop, int64_t *out, size_t cap_rows, size_t *rows_out);

/* Rows first .. first+n_rows-1 of the per-step counts (4 int64 each) into
 * out (host); fails with AMB_EINVAL unless first + n_rows <= steps done.
 * Synchronises. */
amb_status amb_counts_range(amb_pop *pop, uint64_t first, size_t n_rows, int64_t *out);

/* As amb_counts_range, but asynchronous: the copy runs on a side stream of
 * the library, ordered after the work queued so far on the population's
 * stream, and the call returns at once, so later steps do not wait for the
 * copy.  The rows in `out` are final once amb_synchronize (or any call that
 * synchronises the population, or amb_destroy) has returned; the stream
 * itself does not cover the copy.  Use page-locked host memory for a truly
 * asynchronous copy.  Errors: AMB_EINVAL for rows not recorded yet,
 * AMB_ECUDA if the side stream cannot be created. */
amb_status amb_counts_async(amb_pop *pop, uint64_t first, size_t n_rows, int64_t *out);

/*
 * The counting-sort cell index of the current positions (grid environment,
 * paper Sec. 4.1): start[C+1] with C = L*L (start[c] = agents in cells < c,
 * start[C] = n) and ids[n] listing agent ids cell by cell (order inside a
 * cell unspecified).  Walk and SIR.  Synchronises.
 */
amb_status amb_read_index(amb_pop *pop, int32_t *start, int32_t *ids, int dst_on_device);

typedef struct {
    int32_t ok;              /* 1 iff every check below holds */
    int32_t conservation_ok; /* wealth: total wealth = n * w_init after every step */
    int32_t nonnegative_ok;  /* wealth: no negative wealth now */
    int32_t bounds_ok;       /* walk/SIR: every coordinate in [0, L) now */
    int32_t population_ok;   /* SIR: S + I + R = n after every step; n fixed */
    int32_t monotone_ok;     /* SIR: R never decreases */
    int32_t initial_ok;      /* SIR: initial infected count = n_init_infected */
    int32_t index_ok;        /* walk/SIR: start[C] = n, start non-decreasing */
    int64_t first_bad_step;  /* first step whose counts failed, or -1 */
} amb_invariant_report;

/* Check the paper's invariants (Sec. 5.1.3 / 6.2) plus R monotone and index
 * consistency.  Returns AMB_EINVARIANT when any check fails (report filled). */
amb_status amb_invariants(amb_pop *pop, amb_invariant_report *out);

typedef struct {
    /* wealth (R17): G = sum_i (2i - n - 1) w_(i) / (n * sum w), exact integer
     * numerator (hi, lo two's-complement 128-bit), one double division */
    double gini;
    int64_t gini_num_hi;
    uint64_t gini_num_lo;
    int64_t total_wealth;
    int32_t min_wealth, max_wealth;
    /* SIR curve over steps 1..T: peak I, first step at the peak, mean and
     * variance of t weighted by I(t) from exact integer sums */
    int64_t peak_infected;
    uint32_t peak_step;
    double curve_mean, curve_var;
    int64_t final_s, final_i, final_r;
    /* walk/SIR occupancy: the largest number of agents in one cell */
    int32_t max_occupancy;
} amb_stats;

/* End-of-run statistics.  hist (host, optional): wealth model -> hist[v] =
 * agents with wealth min_wealth + v; walk/SIR -> hist[m] = cells holding m
 * agents.  Copies min(hist_cap, bins) entries, *hist_len = bins.  Synchronises. */
amb_status amb_stats_compute(amb_pop *pop, amb_stats *out, int64_t *hist, size_t hist_cap,
                             size_t *hist_len);

/* Per-cell occupancy (C = L*L int32, host or device). Walk and SIR. */
amb_status amb_occupancy(amb_pop *pop, int32_t *occ, int dst_on_device);

/* Steps completed so far. */
uint64_t amb_step_index(const amb_pop *pop);

/* Number of CUDA kernels the step calls of this population have launched
 * so far (amb_step only; set-up, read-back and statistics are not counted). */
uint64_t amb_launch_count(const amb_pop *pop);

/* Block until the population's queued work is done; reports device errors. */
amb_status amb_synchronize(amb_pop *pop);

/* Message of the last failure on this thread ("" if none). */
const char *amb_last_error(void);

/* SIR thresholds as the library computes them (host only, no GPU needed):
 * t_inf[k] = min(floor((1 - (1-beta)^k) 2^32), 2^32-1), (1-beta)^k built by k
 * IEEE double products; t_inf[0] = 0; the table ends at K (entries beyond K
 * equal t_inf[K]), K <= cap; t_rec = min(floor(gamma 2^32), 2^32-1).
 * t_inf needs cap+1 entries. */
amb_status amb_sir_thresholds(double beta, double gamma, uint32_t cap, uint32_t *t_inf,
                              uint32_t *K, uint32_t *t_rec);

/*
 * Stateless counting-sort cell index over caller buffers (grid environment,
 * paper Sec. 4.1): x, y (n int32 each, device, values in [0, L)) -> start
 * (C+1 int32, device, 16-byte aligned) and ids (n int32, device),
 * C = L*L < 2^31.  Scratch
 * (2 C int32 + look-back state) is allocated and freed on the stream.
 * Asynchronous when sync == 0.  Agents with a coordinate outside [0, L) are
 * left out of the index (start[C] then counts only the others, and ids
 * beyond start[C] are unspecified); with sync != 0 the call waits for the
 * result and returns AMB_EINVAL if any agent was left out.
 */
amb_status amb_cell_index(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L,
                          int32_t *start, int32_t *ids, void *cuda_stream, int sync);

/* ------------------------------------------------------------ batches ----
 * Many independent jobs advanced together on one GPU (the paper's Experiment
 * with replications and ParallelRunner, Sec. 4.2, re-cast for one device):
 * at most three persistent kernel launches (the SIR jobs; the wealth jobs
 * whose column fits one CTA's shared memory; the other wealth and the walk
 * jobs), each draining a device work queue of all of its jobs' steps (one
 * CTA per SM; a job's steps follow one another, different jobs' steps
 * overlap).  The run is captured into one CUDA graph and launched once
 * (use_graph = 1, the default).  Results are bit-identical to stepping each
 * job alone with amb_step.
 */
typedef struct {
    amb_model model;
    amb_params params;   /* SIR jobs run on the band path (variant GENERIC is rejected) */
    uint64_t seed;
    uint32_t replicate;
    uint32_t steps;      /* steps this job advances in amb_batch_run */
} amb_job;

typedef struct {
    uint32_t band_rows_cap; /* tallest SIR band in rows (1..32); 0 = 32 */
    int32_t spread_bands;   /* 0: each SIR job in the fewest bands (many jobs share the GPU);
                               1: each job's bands spread over every SM */
    int32_t autotune;       /* 1: time the shapes {8, 16, 32 rows} x {fewest, spread} on
                               throwaway copies of up to eight of the largest SIR jobs and
                               keep the fastest (overrides the two fields above) */
    int32_t use_graph;      /* 1: one CUDA graph for the whole run */
} amb_tune;

typedef struct {
    size_t n_jobs;
    uint32_t band_rows_cap; /* the band shape used */
    int32_t spread_bands;
    uint64_t launches;      /* kernel launches of the run */
    uint64_t agent_steps;   /* sum over jobs of n * steps */
    double ms;              /* device time of the run (events around the graph launch) */
} amb_batch_report;

typedef struct amb_batch amb_batch;

/* Create the populations of n jobs (device memory on cuda_stream, which must
 * not be the legacy default stream when graphs are used). */
amb_status amb_batch_create(const amb_job *jobs, size_t n, void *cuda_stream, amb_batch **out);

/* Advance every job by its steps (once per batch); tune may be NULL (cap 32,
 * no autotune, graph).  *ms_out (optional): device time of the run. */
amb_status amb_batch_run(amb_batch *b, const amb_tune *tune, double *ms_out);

/* Borrow job i's population (read columns, counts, statistics through the
 * single-population calls; the batch keeps ownership). */
amb_status amb_batch_population(amb_batch *b, size_t i, amb_pop **pop);

amb_status amb_batch_info(amb_batch *b, amb_batch_report *info);

/* Free every population of the batch. */
amb_status amb_batch_destroy(amb_batch *b);

/* Device memory one job needs (host-only arithmetic, no GPU call):
 * *resident = what its population holds while it exists (columns or
 * cell-ordered records, cell index, thresholds, count rows, look-back words),
 * *transient = what its creation holds on top for a moment (initial columns,
 * the cell-ordered id list and counting-sort scratch).  Stream-ordered pool rounding is not included. */
amb_status amb_job_bytes(const amb_job *job, size_t *resident, size_t *transient);

/* ------------------------------------------------------------ serving ----
 * A request loop for simulation jobs (the paper's Experiment runs, re-cast as
 * a service; the paper has no server).  Jobs are submitted at any time from
 * any thread.  A worker thread admits them in arrival order while their device
 * memory (amb_job_bytes) fits the budget, keeps every admitted job's state on
 * the device, and advances all admitted jobs together, chunk_steps steps at a
 * time, with the batched launches (continuous batching: jobs that arrive
 * while others run join at the next chunk; finished jobs leave and free their
 * memory).  An iteration also ends at the step where the first of its jobs
 * finishes (it takes at least min(8, chunk_steps) steps), so a finished job's
 * result does not wait for the others' chunks.  A job's results are
 * bit-identical to stepping it alone.
 */
typedef struct {
    size_t hbm_budget_bytes; /* device memory for job state (resident + the creation
                                transient of the job being admitted) */
    uint32_t max_active;     /* jobs on the device at once; 0 = 4096 */
    uint32_t chunk_steps;    /* steps per job per iteration; 0 = 32 */
    uint32_t band_rows_cap;  /* SIR band height cap (as in amb_tune); 0 = 16 */
    int32_t spread_bands;    /* 0: per iteration, spread the bands over every SM when
                                the active SIR jobs' fewest bands would leave SMs idle;
                                1: always spread; -1: always the fewest bands */
    uint32_t iteration_us;   /* 0: no time target; otherwise an iteration takes at most
                                as many steps as the previous iteration's device time per
                                step says fit in this many microseconds (at least
                                min(8, chunk_steps)), so that jobs arriving meanwhile
                                join sooner */
} amb_server_config;

typedef struct {
    uint64_t ticket;
    amb_status status;     /* AMB_OK, or the error that ended the job */
    amb_model model;
    uint32_t n;
    uint32_t steps;        /* steps completed */
    int64_t last[4];       /* the job's last per-step count row (zeros when steps = 0) */
    double submit_s;       /* host times in seconds since amb_server_create */
    double admit_s;        /* state created on the device */
    double done_s;         /* result readable */
} amb_result;

typedef struct {
    uint64_t submitted, admitted, completed, failed, cancelled;
    uint64_t agent_steps;  /* of completed jobs */
    uint64_t iterations, launches;
    size_t hbm_in_use, hbm_peak; /* by amb_job_bytes accounting */
    uint32_t active, pending;
    double busy_s;         /* worker time spent advancing jobs */
} amb_server_report;

typedef struct amb_server amb_server;

/* Start a server on cuda_stream (not the legacy default stream) of the
 * current device.  cfg may not be NULL; hbm_budget_bytes > 0. */
amb_status amb_server_create(const amb_server_config *cfg, void *cuda_stream, amb_server **out);

/* Queue a job; *ticket identifies it.  keep_columns != 0 keeps the final
 * columns on the host for amb_server_read_column.  AMB_EBUDGET when the job
 * alone can never fit the budget; AMB_EINVAL for parameters amb_create would
 * reject (SIR variant GENERIC included). */
amb_status amb_server_submit(amb_server *s, const amb_job *job, int keep_columns, uint64_t *ticket);

/* AMB_OK and *out filled once the job is done (out->status tells whether it
 * succeeded); AMB_EBUSY while it is queued or running; AMB_ENOTFOUND for an
 * unknown or released ticket. */
amb_status amb_server_poll(amb_server *s, uint64_t ticket, amb_result *out);

/* As poll, but waits up to timeout_s seconds (AMB_ETIMEOUT if still running). */
amb_status amb_server_wait(amb_server *s, uint64_t ticket, double timeout_s, amb_result *out);

/* The finished job's per-step count rows (host copy; as amb_counts). */
amb_status amb_server_counts(amb_server *s, uint64_t ticket, int64_t *out, size_t cap_rows, size_t *rows_out);

/* A kept final column of a finished job, in id order, into host memory dst
 * (n = the job's n elements; int32, or uint8 for the state). */
amb_status amb_server_read_column(amb_server *s, uint64_t ticket, amb_col col, void *dst, size_t n);

/* Cancel a job: a queued job ends at once, a running one after the current
 * iteration (its device memory is freed then); its result reports
 * AMB_ECANCELED.  A finished job is left as it is. */
amb_status amb_server_cancel(amb_server *s, uint64_t ticket);

/* Forget a finished job's result (its ticket becomes unknown). */
amb_status amb_server_release(amb_server *s, uint64_t ticket);

/* Wait until every submitted job is done (AMB_ETIMEOUT after timeout_s). */
amb_status amb_server_drain(amb_server *s, double timeout_s);

amb_status amb_server_stats(amb_server *s, amb_server_report *out);

/* Stop the worker after its current iteration, cancel queued jobs, free every
 * job's device memory and the server. */
amb_status amb_server_destroy(amb_server *s);

/* ------------------------------------------------------------- view API ----
 * The paper's view API (Sec. 3.1, 3.3) over a device-resident columnar table
 * of n rows (row = agent id):
 *  - full-population views: amb_table_map / amb_table_map_col update every
 *    row of a column ("agents.wealth += 10");
 *  - filtered views: amb_table_where(col, cmp, s) lists, in ascending order,
 *    the ids whose value satisfies the predicate at the moment of the call
 *    ("agents.where(agents.wealth > 0)"); updates through it touch exactly
 *    those rows;
 *  - scatter views: id lists in which ids may repeat (amb_view_from_ids,
 *    amb_view_draw); an update through a scatter view is applied once per
 *    occurrence, so amb_view_scatter_add accumulates duplicates
 *    ("agents.at[recipients].scatter_add(wealth=1)").
 * Columns are int32 or uint8.  Operations: v = v OP s with wrapping
 * arithmetic in the column's type (the scalar is reduced to that type by
 * two's-complement truncation); MIN / MAX compare signed int32 or unsigned
 * uint8 values.  Through a view with repeated ids every operation with one
 * scalar gives the same result in any order (SET stores s; MUL multiplies
 * once per occurrence).  Predicates compare the value, as a 64-bit integer,
 * with the 64-bit scalar.
 * A view's length stays on the device: view operations are asynchronous on
 * the table's stream and never wait for the host; amb_view_count and
 * amb_view_ids synchronise.  Views belong to their table and must be
 * destroyed before it (amb_table_destroy returns AMB_EBUSY otherwise).
 */
typedef enum { AMB_DT_I32 = 0, AMB_DT_U8 = 1 } amb_dtype;
typedef enum { AMB_OP_SET = 0, AMB_OP_ADD = 1, AMB_OP_SUB = 2, AMB_OP_MUL = 3, AMB_OP_MIN = 4, AMB_OP_MAX = 5 } amb_op;
typedef enum { AMB_CMP_EQ = 0, AMB_CMP_NE = 1, AMB_CMP_LT = 2, AMB_CMP_LE = 3, AMB_CMP_GT = 4, AMB_CMP_GE = 5 } amb_cmp;

typedef struct amb_table amb_table;
typedef struct amb_view amb_view;

/* A table of n rows (no columns yet) on cuda_stream; n < 2^31. */
amb_status amb_table_create(uint32_t n, void *cuda_stream, amb_table **out);
/* Frees the columns; AMB_EBUSY while views of the table exist. */
amb_status amb_table_destroy(amb_table *t);
/* Add a column, every row set to fill (bulk creation, paper Sec. 3.3
 * add_agents with a scalar broadcast); *col_out = its index.  Names are unique. */
amb_status amb_table_add_column(amb_table *t, const char *name, amb_dtype dtype, int64_t fill, int *col_out);
/* Index of a named column (AMB_ENOTFOUND if absent). */
amb_status amb_table_find_column(amb_table *t, const char *name, int *col_out);
amb_status amb_table_rows(amb_table *t, uint32_t *n);
/* Replace / read a whole column (n == rows; int32 or uint8 elements). */
amb_status amb_table_write(amb_table *t, int col, const void *src, size_t n, int src_on_device);
amb_status amb_table_read(amb_table *t, int col, void *dst, size_t n, int dst_on_device);
/* Full-population view: col = col OP scalar. */
amb_status amb_table_map(amb_table *t, int col, amb_op op, int64_t scalar);
/* Full-population view with a column operand: dst = dst OP src, row by row
 * (src's value taken as an integer, then reduced to dst's type). */
amb_status amb_table_map_col(amb_table *t, int dst, amb_op op, int src);
/* Filtered view: ascending ids with col CMP scalar (order-preserving stream
 * compaction).  The view holds up to n ids. */
amb_status amb_table_where(amb_table *t, int col, amb_cmp cmp, int64_t scalar, amb_view **out);
/* Scatter view from k caller ids (repeats allowed; every id in [0, n),
 * else AMB_EINVAL).  Synchronises. */
amb_status amb_view_from_ids(amb_table *t, const int32_t *ids, size_t k, int ids_on_device, amb_view **out);
/* Scatter view of random ids, one per id i of v, in v's order: u = Philox
 * (key (seed, replicate), counter (i, step, 0, 0)), r' = hi32(u[word] * m);
 * exclude_self: m = range - 1 and r = r' + (r' >= i) (a uniformly chosen other
 * id, range >= 2); otherwise m = range and r = r' (range >= 1).  The drawn ids
 * address rows of the table: range <= n, else AMB_EINVAL. */
amb_status amb_view_draw(amb_view *v, uint64_t seed, uint32_t replicate, uint32_t step, uint32_t word, uint32_t range,
                         int exclude_self, amb_view **out);
/* A view of a view: the ids v lists (in v's order, repeats kept) whose value
 * satisfies col CMP scalar, so where(A) followed by amb_view_where(B) is the
 * conjunction of A and B.  Asynchronous; the length stays on the device. */
amb_status amb_view_where(amb_view *v, int col, amb_cmp cmp, int64_t scalar, amb_view **out);
/* scatter_add with one value per listed id: col[id_j] += values[j] for the
 * view's entries j (device int32 array of n_values >= the view's length;
 * shorter arrays are reported by amb_table_synchronize). */
amb_status amb_view_scatter_add_values(amb_view *v, int col, const int32_t *values, size_t n_values);
/* Update the rows a view lists: col[id] = col[id] OP scalar per listed id. */
amb_status amb_view_map(amb_view *v, int col, amb_op op, int64_t scalar);
/* amb_view_map with AMB_OP_ADD: duplicate ids accumulate. */
amb_status amb_view_scatter_add(amb_view *v, int col, int64_t value);
/* Number of ids in the view (synchronises). */
amb_status amb_view_count(amb_view *v, size_t *count);
/* The view's ids (min(count, cap) of them) into dst; *count (optional) =
 * the view's length.  Synchronises. */
amb_status amb_view_ids(amb_view *v, int32_t *dst, size_t cap, int dst_on_device, size_t *count);
amb_status amb_view_destroy(amb_view *v);
/* Wait for the table's stream; report device-side errors of view operations. */
amb_status amb_table_synchronize(amb_table *t);

/* Buffered per-agent writes (paper Sec. 3.2.1: per-agent record() calls are
 * buffered and flushed by one id-keyed update per step).  A log belongs to a
 * table (destroy it before the table).  amb_log_record appends k writes
 * "column col of row ids[j] := values[j]" in order (values reduced to the
 * column's type by two's-complement truncation; ids in [0, n), else
 * AMB_EINVAL and nothing is appended); the log holds `capacity` writes.
 * amb_log_flush applies every pending write so that, for each (row, column),
 * the last recorded write wins, and empties the log (asynchronous). */
typedef struct amb_log amb_log;
amb_status amb_log_create(amb_table *t, uint32_t capacity, amb_log **out);
amb_status amb_log_record(amb_log *l, int col, const int32_t *ids, const int64_t *values, size_t k, int on_device);
amb_status amb_log_pending(amb_log *l, size_t *k);
amb_status amb_log_flush(amb_log *l);
amb_status amb_log_destroy(amb_log *l);

/* Grid environments (paper Sec. 4.1): `steps` steps of a random walk on a
 * d-dimensional lattice (d = 1..4; sizes[q] cells along axis q; positions in
 * the int32 columns cols[0..d-1], each in [0, sizes[q])).  Each step every
 * agent moves to a neighbour chosen uniformly, m = hi32(u0 * count) with u
 * the agent's Philox draw for the step (key (seed, replicate), counter (id,
 * step)), the m-th neighbour in this order: Moore (moore != 0): offsets in
 * {-1, 0, 1}^d without zero, enumerated as base-3 numbers with axis 0 the
 * fastest digit; von Neumann: (axis 0, -1), (axis 0, +1), (axis 1, -1), ...
 * On a torus (torus != 0) coordinates wrap; otherwise only neighbours inside
 * the box count, in the same order, and an agent with none stays.  d = 2,
 * Moore, torus is the walk of amb_step.  Coordinates outside the box are left
 * unchanged and reported by amb_table_synchronize. */
amb_status amb_table_grid_walk(amb_table *t, const int *cols, uint32_t d, const uint32_t *sizes, int moore, int torus,
                               uint64_t seed, uint32_t replicate, uint32_t step, uint32_t steps);

/*
 * amb_cell_index without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory while they run, for example a process whose device memory is
 * all handed out by another allocator up front (a fixed HBM budget), or code
 * that must not call cudaMalloc / cudaFree because those can synchronise the
 * whole device.  The caller passes inputs and outputs exactly as for
 * amb_cell_index; the scratch (cell counts, cursors, look-back words, error
 * word) is a file-scope device array of about 8 MiB, for grids of at most
 * 1,048,576 cells (L <= 1024); larger grids return AMB_EINVAL.  Every GPU that
 * loads the library keeps that array until the process exits.
 *  - The first call on a device, with that device current, looks up the
 *    array's device address (cudaGetSymbolAddress); make that first call
 *    before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents;
 *    the call clears what has to start at zero.  Calls that overlap on the
 *    GPU (other streams, other threads) race on it: serialise them.
 *  - Each call starts by clearing, in stream order, the look-back words,
 *    ticket counters and error word in that array, so no call depends on
 *    what an earlier one left there.
 *  - sync != 0 waits for the result and reports coordinates outside [0, L)
 *    as AMB_EINVAL, as amb_cell_index does, and a look-back wait that ran out
 *    as AMB_ETIMEOUT.  sync == 0 returns once the work is queued and reports
 *    no device-side error at all (the next call clears the error word): such
 *    a caller learns of left-out agents by checking start[L*L] == n after
 *    synchronising the stream.
 */
amb_status amb_cell_index_noalloc(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *start,
                                  int32_t *ids, void *cuda_stream, int sync);

/* Failure-handling self-check (no counterpart in the paper): one warp waits
 * in the library's decoupled look-back for a predecessor whose status word
 * nothing ever sets.  The wait is bounded (2 s), so the kernel gives up, sets
 * the error word and returns; the call returns AMB_ETIMEOUT, the expected
 * outcome, with *waited_s the time waited, and the device stays usable.  Any
 * other status means the bound did not work. */
amb_status amb_selfcheck_wait_timeout(void *cuda_stream, double *waited_s);

/* Fault-injection hook for tests (no counterpart in the paper): the next k
 * population creations (amb_create, amb_create_continuous, batch and server
 * admissions included) fail with AMB_ENOMEM before touching the device.
 * k = 0 turns it off.  Process-wide. */
amb_status amb_debug_fail_creates(uint32_t k);

/* Test hook (no counterpart in the paper): the number the log gives its next
 * record.  A flush numbers its records from this value on and restarts from 0,
 * with the winner words cleared, when the numbers would reach 2^31 - 1; the
 * hook lets a test reach that restart without 2^31 records.  Fails with
 * AMB_EINVAL while records are pending or for base >= 2^31. */
amb_status amb_debug_log_base(amb_log *l, uint32_t base);

/* Version string of the library build. */
const char *amb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AMB_H */
