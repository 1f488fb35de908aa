// server.cu -- a request loop for simulation jobs with continuous batching.
//
// Jobs arrive through amb_server_submit (any thread) and wait in arrival
// order.  One worker thread owns the GPU work: it admits waiting jobs while
// their device memory fits the budget (strict arrival order, so a large job is
// never overtaken indefinitely), creates their populations on the device, and
// then repeatedly advances every admitted job by up to chunk_steps steps with
// the batched launches (one shared band launch per SIR step over all SIR jobs,
// one launch for all small wealth jobs, shared launches for the large ones,
// one per walk job).  After each iteration, jobs that reached their step count
// leave: their count rows (and, on request, final columns) are copied to the
// host, their device memory is freed and their result becomes readable.  Jobs
// that arrive meanwhile join at the next iteration.
//
// Memory accounting uses amb_job_bytes (host arithmetic), plus a fixed reserve
// for the per-iteration launch tables and wide band counters.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "amb_internal.cuh"

using namespace amb;

namespace {

constexpr size_t kIterationReserve = size_t(512) << 20;  // launch tables, wide band counters
constexpr size_t kPoolSlack = size_t(64) << 10;          // per population: pool rounding, small buffers
constexpr uint32_t kMinChunk = 8;                        // fewest steps of an iteration (unless chunk_steps is lower)

size_t series_bytes(uint32_t steps)
{
    size_t cap = 64;
    while (cap < steps) cap *= 2;
    return cap * 4u * sizeof(int64_t);
}

struct ServerJob {
    uint64_t ticket = 0;
    amb_job job{};
    bool keep = false;
    size_t resident = 0, transient = 0;
    double t_submit = 0, t_admit = -1, t_done = -1;
    amb_pop *pop = nullptr;
    uint32_t done_steps = 0;
    amb_status status = AMB_OK;
    bool finished = false;
    std::atomic<bool> cancel{false};  // set by amb_server_cancel while the job runs
    std::vector<int64_t> series;
    std::vector<int32_t> col_a, col_b;  // wealth, or x and y
    std::vector<uint8_t> col_state;
};

}  // namespace

struct amb_server {
    amb_server_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::chrono::steady_clock::time_point origin;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerJob *> pending;
    std::unordered_map<uint64_t, ServerJob *> jobs;  // every job not released
    std::vector<ServerJob *> active;                 // worker thread only
    uint64_t next_ticket = 1;
    uint64_t cancelled_running = 0;  // jobs cancelled after admission
    size_t in_use = 0, peak = 0;
    amb_server_report rep{};
    bool stop = false;
    std::thread worker;

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - origin).count(); }
};

extern "C" amb_status amb_job_bytes(const amb_job *job, size_t *resident, size_t *transient)
{
    if (!job || !resident || !transient) return fail(AMB_EINVAL, "null pointer");
    AMB_TRY(check_params(job->model, &job->params, job->seed));
    const uint64_t n = job->params.n, L = job->params.grid_side, C = L * L;
    uint64_t r = series_bytes(job->steps) + sizeof(uint32_t), t = 0;
    switch (job->model) {
    case AMB_WEALTH:
        r += 4 * n + (wealth_uses_smem((uint32_t)n) ? 0 : 4 * n);
        break;
    case AMB_WALK:
        r += 8 * n;
        break;
    case AMB_SIR: {
        // records (id + word, two buffers), row starts, cell index, thresholds,
        // look-back words of the cell-index scan and of the bands
        const uint64_t tiles = std::max<uint64_t>(scan_tiles((uint32_t)C), L);
        r += 16 * (n + 4) + 8 * (L + 1) + 4 * (C + 1) + 4 * (n + 2) + 8 * std::max<uint64_t>(tiles, 1024) + 16;
        // initial columns (x, y, state), the cell-ordered id list and the
        // counting sort's counters
        t = 13 * n + 8 * C;
        break;
    }
    case AMB_CWALK:
    case AMB_CSIR:  // rejected by check_params: continuous models are not batched or served
        return fail(AMB_EINVAL, "continuous-space models are not served");
    }
    *resident = (size_t)r + kPoolSlack;
    *transient = (size_t)t;
    return AMB_OK;
}

namespace {

void finish_job(amb_server *S, ServerJob *j, amb_status st)
{
    // device side first (worker thread, no lock held)
    if (j->pop) {
        if (st == AMB_OK) {
            j->series.resize((size_t)j->done_steps * 4u);
            size_t rows = 0;
            st = amb_counts(j->pop, j->series.data(), j->done_steps, &rows);
            if (st == AMB_OK && j->keep) {
                const size_t n = j->job.params.n;
                if (j->job.model == AMB_WEALTH) {
                    j->col_a.resize(n);
                    st = amb_read_column(j->pop, AMB_COL_WEALTH, j->col_a.data(), n, 0);
                } else {
                    j->col_a.resize(n);
                    j->col_b.resize(n);
                    st = amb_read_column(j->pop, AMB_COL_X, j->col_a.data(), n, 0);
                    if (st == AMB_OK) st = amb_read_column(j->pop, AMB_COL_Y, j->col_b.data(), n, 0);
                    if (st == AMB_OK && j->job.model == AMB_SIR) {
                        j->col_state.resize(n);
                        st = amb_read_column(j->pop, AMB_COL_STATE, j->col_state.data(), n, 0);
                    }
                }
            }
        }
        amb_destroy(j->pop);
        j->pop = nullptr;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use -= j->resident;
    j->status = st;
    j->t_done = S->now();
    j->finished = true;
    if (st == AMB_OK) {
        S->rep.completed += 1;
        S->rep.agent_steps += (uint64_t)j->job.params.n * j->done_steps;
    } else if (st == AMB_ECANCELED) {
        S->rep.cancelled += 1;
        S->cancelled_running += 1;
    } else {
        S->rep.failed += 1;
    }
    S->cv_done.notify_all();
}

void worker_loop(amb_server *S)
{
    cudaSetDevice(S->device);
    const uint32_t max_active = S->cfg.max_active ? S->cfg.max_active : 4096u;
    const uint32_t chunk = S->cfg.chunk_steps ? S->cfg.chunk_steps : 32u;
    BandShape shape;
    shape.rows_cap = S->cfg.band_rows_cap ? std::min<uint32_t>(S->cfg.band_rows_cap, 32u) : 16u;
    shape.spread = S->cfg.spread_bands > 0;
    shape.adaptive = S->cfg.spread_bands == 0;
    double step_us = 0.0;  // device time per step of the last iteration
    for (;;) {
        std::vector<ServerJob *> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->active.empty())
                S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
            if (S->stop) break;
            // admission: arrival order, while memory and slots allow
            while (!S->pending.empty() && S->active.size() + admit.size() < max_active) {
                ServerJob *j = S->pending.front();
                if (S->in_use + j->resident + j->transient + kIterationReserve > S->cfg.hbm_budget_bytes) break;
                S->in_use += j->resident;
                S->peak = std::max(S->peak, S->in_use + j->transient + kIterationReserve);
                S->pending.pop_front();
                admit.push_back(j);
            }
            S->rep.admitted += admit.size();
        }
        for (ServerJob *j : admit) {
            amb_params p = j->job.params;
            if (j->job.model == AMB_SIR) p.variant = AMB_SIR_BAND;
            const amb_status st = amb_create(j->job.model, &p, j->job.seed, j->job.replicate, S->stream, &j->pop);
            if (st != AMB_OK) {
                j->pop = nullptr;
                finish_job(S, j, st);
                continue;
            }
            j->t_admit = S->now();
            if (j->job.steps == 0) {
                finish_job(S, j, AMB_OK);
                continue;
            }
            S->active.push_back(j);
        }
        if (S->active.empty()) continue;

        // one iteration: every active job advances by up to `k_it` steps: at
        // most `chunk`, no further than the step where the first active job
        // finishes, and (with a time target) no more steps than the previous
        // iteration's device time per step says fit in the target; at least
        // min(kMinChunk, chunk)
        AMB_TRACE("amb_server_iteration");
        const double t0 = S->now();
        std::vector<amb_pop *> pops;
        std::vector<uint32_t> ks;
        uint32_t k_it = chunk;
        for (ServerJob *j : S->active) k_it = std::min<uint32_t>(k_it, j->job.steps - j->done_steps);
        if (S->cfg.iteration_us && step_us > 0.0)
            k_it = std::min<uint32_t>(k_it, (uint32_t)std::max(1.0, (double)S->cfg.iteration_us / step_us));
        k_it = std::max<uint32_t>(k_it, std::min<uint32_t>(kMinChunk, chunk));
        for (ServerJob *j : S->active) {
            pops.push_back(j->pop);
            ks.push_back(std::min<uint32_t>(k_it, j->job.steps - j->done_steps));
        }
        uint64_t launches = 0;
        float ms = 0.f;
        amb_status st = advance(pops, ks, shape, S->stream, false, &launches, &ms);
        if (st == AMB_OK && ms > 0.f) step_us = 1000.0 * (double)ms / (double)k_it;
        std::vector<uint32_t> words;
        if (st == AMB_OK) st = read_errors(pops, S->stream, words);
        std::vector<ServerJob *> still;
        for (size_t q = 0; q < S->active.size(); ++q) {
            ServerJob *j = S->active[q];
            if (st != AMB_OK) {
                finish_job(S, j, st);  // the iteration as a whole failed
                continue;
            }
            j->done_steps += ks[q];
            if (j->cancel.load()) {
                finish_job(S, j, AMB_ECANCELED);
            } else if (words[q]) {
                finish_job(S, j, (words[q] & ERR_TIMEOUT) ? AMB_ETIMEOUT : AMB_EINVARIANT);
            } else if (j->done_steps == j->job.steps) {
                finish_job(S, j, AMB_OK);
            } else {
                still.push_back(j);
            }
        }
        S->active.swap(still);
        std::lock_guard<std::mutex> lk(S->mu);
        S->rep.iterations += 1;
        S->rep.launches += launches;
        S->rep.busy_s += S->now() - t0;
    }
    // stopping: free what is still on the device
    for (ServerJob *j : S->active) {
        if (j->pop) amb_destroy(j->pop);
        j->pop = nullptr;
    }
    S->active.clear();
}

ServerJob *find_locked(amb_server *S, uint64_t ticket)
{
    auto it = S->jobs.find(ticket);
    return it == S->jobs.end() ? nullptr : it->second;
}

void fill_result(const ServerJob *j, amb_result *out)
{
    out->ticket = j->ticket;
    out->status = j->status;
    out->model = j->job.model;
    out->n = j->job.params.n;
    out->steps = j->done_steps;
    for (int c = 0; c < 4; ++c)
        out->last[c] = (j->status == AMB_OK && j->done_steps) ? j->series[(size_t)(j->done_steps - 1) * 4u + c] : 0;
    out->submit_s = j->t_submit;
    out->admit_s = j->t_admit;
    out->done_s = j->t_done;
}

}  // namespace

extern "C" {

amb_status amb_server_create(const amb_server_config *cfg, void *cuda_stream, amb_server **out)
{
    if (!cfg || !out) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    if (cfg->hbm_budget_bytes == 0) return fail(AMB_EINVAL, "hbm_budget_bytes must be > 0");
    if (cuda_stream == nullptr) return fail(AMB_EINVAL, "the server needs a created stream, not the legacy default stream");
    amb_server *S = new (std::nothrow) amb_server();
    if (!S) return fail(AMB_ENOMEM, "host allocation failed");
    S->cfg = *cfg;
    S->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return fail(AMB_ECUDA, "no current device");
    }
    S->origin = std::chrono::steady_clock::now();
    try {
        S->worker = std::thread(worker_loop, S);
    } catch (...) {
        delete S;
        return fail(AMB_ENOMEM, "could not start the worker thread");
    }
    *out = S;
    return AMB_OK;
}

amb_status amb_server_submit(amb_server *S, const amb_job *job, int keep_columns, uint64_t *ticket)
{
    AMB_TRACE("amb_server_submit");
    if (!S || !job || !ticket) return fail(AMB_EINVAL, "null pointer");
    if (job->model == AMB_SIR && job->params.variant == AMB_SIR_GENERIC)
        return fail(AMB_EINVAL, "the server runs SIR on the band path");
    if (job->steps >= kInitStep) return fail(AMB_EINVAL, "too many steps");
    size_t resident = 0, transient = 0;
    AMB_TRY(amb_job_bytes(job, &resident, &transient));
    if (resident + transient + kIterationReserve > S->cfg.hbm_budget_bytes)
        return fail(AMB_EBUDGET, "the job needs %zu + %zu bytes, over the %zu-byte budget", resident, transient,
                    S->cfg.hbm_budget_bytes);
    ServerJob *j = new (std::nothrow) ServerJob();
    if (!j) return fail(AMB_ENOMEM, "host allocation failed");
    j->job = *job;
    j->keep = keep_columns != 0;
    j->resident = resident;
    j->transient = transient;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete j;
            return fail(AMB_EINVAL, "server is stopping");
        }
        j->ticket = S->next_ticket++;
        j->t_submit = S->now();
        S->jobs[j->ticket] = j;
        S->pending.push_back(j);
        S->rep.submitted += 1;
        *ticket = j->ticket;
    }
    S->cv_work.notify_one();
    return AMB_OK;
}

amb_status amb_server_poll(amb_server *S, uint64_t ticket, amb_result *out)
{
    if (!S || !out) return fail(AMB_EINVAL, "null pointer");
    std::lock_guard<std::mutex> lk(S->mu);
    ServerJob *j = find_locked(S, ticket);
    if (!j) return fail(AMB_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (!j->finished) return AMB_EBUSY;
    fill_result(j, out);
    return AMB_OK;
}

amb_status amb_server_wait(amb_server *S, uint64_t ticket, double timeout_s, amb_result *out)
{
    if (!S || !out) return fail(AMB_EINVAL, "null pointer");
    std::unique_lock<std::mutex> lk(S->mu);
    ServerJob *j = find_locked(S, ticket);
    if (!j) return fail(AMB_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(std::max(timeout_s, 0.0));
    if (!S->cv_done.wait_until(lk, until, [&] { return j->finished; }))
        return fail(AMB_ETIMEOUT, "job %llu still running", (unsigned long long)ticket);
    fill_result(j, out);
    return AMB_OK;
}

amb_status amb_server_counts(amb_server *S, uint64_t ticket, int64_t *out, size_t cap_rows, size_t *rows_out)
{
    if (!S || (!out && cap_rows)) return fail(AMB_EINVAL, "null pointer");
    std::lock_guard<std::mutex> lk(S->mu);
    ServerJob *j = find_locked(S, ticket);
    if (!j) return fail(AMB_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (!j->finished) return AMB_EBUSY;
    if (j->status != AMB_OK) return fail(j->status, "job %llu failed", (unsigned long long)ticket);
    const size_t rows = j->series.size() / 4u;
    if (rows_out) *rows_out = rows;
    std::copy_n(j->series.begin(), std::min(rows, cap_rows) * 4u, out);
    return AMB_OK;
}

amb_status amb_server_read_column(amb_server *S, uint64_t ticket, amb_col col, void *dst, size_t n)
{
    AMB_TRACE("amb_server_read_column");
    if (!S || (!dst && n)) return fail(AMB_EINVAL, "null pointer");
    std::lock_guard<std::mutex> lk(S->mu);
    ServerJob *j = find_locked(S, ticket);
    if (!j) return fail(AMB_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (!j->finished) return AMB_EBUSY;
    if (j->status != AMB_OK) return fail(j->status, "job %llu failed", (unsigned long long)ticket);
    if (!j->keep) return fail(AMB_EINVAL, "job %llu was submitted without keep_columns", (unsigned long long)ticket);
    if (n != j->job.params.n) return fail(AMB_EINVAL, "column length %zu != n = %u", n, j->job.params.n);
    const amb_model m = j->job.model;
    if (m == AMB_WEALTH && col == AMB_COL_WEALTH) {
        std::copy_n(j->col_a.begin(), n, static_cast<int32_t *>(dst));
    } else if (m != AMB_WEALTH && col == AMB_COL_X) {
        std::copy_n(j->col_a.begin(), n, static_cast<int32_t *>(dst));
    } else if (m != AMB_WEALTH && col == AMB_COL_Y) {
        std::copy_n(j->col_b.begin(), n, static_cast<int32_t *>(dst));
    } else if (m == AMB_SIR && col == AMB_COL_STATE) {
        std::copy_n(j->col_state.begin(), n, static_cast<uint8_t *>(dst));
    } else {
        return fail(AMB_EINVAL, "column %d does not belong to this model", (int)col);
    }
    return AMB_OK;
}

amb_status amb_server_cancel(amb_server *S, uint64_t ticket)
{
    if (!S) return fail(AMB_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    ServerJob *j = find_locked(S, ticket);
    if (!j) return fail(AMB_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (j->finished) return AMB_OK;
    auto it = std::find(S->pending.begin(), S->pending.end(), j);
    if (it != S->pending.end()) {  // still queued: ends now
        S->pending.erase(it);
        j->status = AMB_ECANCELED;
        j->t_done = S->now();
        j->finished = true;
        S->rep.cancelled += 1;
        S->cv_done.notify_all();
        return AMB_OK;
    }
    j->cancel.store(true);  // admitted: ends after the current iteration
    return AMB_OK;
}

amb_status amb_server_release(amb_server *S, uint64_t ticket)
{
    if (!S) return fail(AMB_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    ServerJob *j = find_locked(S, ticket);
    if (!j) return fail(AMB_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (!j->finished) return fail(AMB_EBUSY, "job %llu is still running", (unsigned long long)ticket);
    S->jobs.erase(ticket);
    delete j;
    return AMB_OK;
}

amb_status amb_server_drain(amb_server *S, double timeout_s)
{
    if (!S) return fail(AMB_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(std::max(timeout_s, 0.0));
    const bool ok = S->cv_done.wait_until(lk, until, [&] {
        return S->rep.completed + S->rep.failed + S->rep.cancelled == S->rep.submitted;
    });
    return ok ? AMB_OK
              : fail(AMB_ETIMEOUT, "%llu jobs still queued or running",
                     (unsigned long long)(S->rep.submitted - S->rep.completed - S->rep.failed - S->rep.cancelled));
}

amb_status amb_server_stats(amb_server *S, amb_server_report *out)
{
    if (!S || !out) return fail(AMB_EINVAL, "null pointer");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->rep;
    out->hbm_in_use = S->in_use;
    out->hbm_peak = S->peak;
    out->pending = (uint32_t)S->pending.size();
    out->active = (uint32_t)(S->rep.admitted - S->rep.completed - S->rep.failed - S->cancelled_running);
    return AMB_OK;
}

amb_status amb_server_destroy(amb_server *S)
{
    if (!S) return AMB_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaStreamSynchronize(S->stream);
    for (auto &kv : S->jobs) delete kv.second;
    S->jobs.clear();
    delete S;
    return AMB_OK;
}

}  // extern "C"
