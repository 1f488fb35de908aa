// batch.cu -- many independent simulation jobs advanced together (the
// paper's Experiment / ParallelRunner, Sec. 4.2, re-cast for one GPU): every
// SIR step of every job is one shared launch over all their bands, the small
// wealth jobs run in one launch (one CTA each, all steps), the large ones take
// three shared launches per step, walk jobs one launch each; the whole run is
// captured into one CUDA graph and launched once.  An autotuner picks the
// band-height cap of the SIR launches by timing candidates on throwaway copies
// of a sample of the jobs (results do not depend on it).
#include <algorithm>
#include <new>
#include <vector>

#include "amb_internal.cuh"

namespace amb {
amb_status walk_steps(amb_pop *pop, uint32_t k);
}

using namespace amb;

struct amb_batch {
    cudaStream_t stream = nullptr;
    std::vector<amb_job> jobs;
    std::vector<amb_pop *> pops;
    bool ran = false;
    BandShape shape;
    uint64_t launches = 0;
    double ms = 0.0;
};

namespace amb {

// Advance every population by its own number of steps (ks[i] for pops[i]):
// one shared band launch per SIR step over all SIR populations, one launch for
// all small wealth populations (all their steps), three shared launches per
// step for the large ones, one launch per walk population.  With graph, the
// launches are captured into one CUDA graph and launched once.  *ms: device
// time of the launches (events on s).  Returns after the work is done.
amb_status advance(const std::vector<amb_pop *> &pops, const std::vector<uint32_t> &ks, BandShape shape,
                   cudaStream_t s, bool graph, uint64_t *launches_out, float *ms_out)
{
    std::vector<amb_pop *> sir, wealth, walk;
    std::vector<uint32_t> sir_steps, wealth_steps, walk_steps_v;
    uint32_t max_large = 0, max_sir = 0;
    for (size_t i = 0; i < pops.size(); ++i) {
        amb_pop *p = pops[i];
        const uint32_t k = ks[i];
        if (p->t + k >= (uint64_t)kInitStep) return fail(AMB_EINVAL, "job %zu: too many steps", i);
        AMB_TRY(band_sync_records(p));
        AMB_TRY(ensure_series(p, p->t + k));
        if (k) AMB_TRY_CUDA(cudaMemsetAsync(p->series + (size_t)p->t * 4u, 0, (size_t)k * 4u * sizeof(int64_t), s));
        if (p->model == AMB_SIR) {
            sir.push_back(p);
            sir_steps.push_back(k);
            max_sir = std::max(max_sir, k);
        } else if (p->model == AMB_WEALTH) {
            wealth.push_back(p);
            wealth_steps.push_back(k);
            if (!wealth_uses_smem(p->p.n) && p->p.n) max_large = std::max(max_large, k);
        } else {
            walk.push_back(p);
            walk_steps_v.push_back(k);
        }
    }
    SirBatch sb;
    WealthBatch wb;
    amb_status r = sir_batch_build(sb, sir.data(), sir_steps.data(), (uint32_t)sir.size(), shape, s);
    if (r == AMB_OK) r = wealth_batch_build(wb, wealth.data(), wealth_steps.data(), (uint32_t)wealth.size(), s);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint64_t launches = 0;
    if (r == AMB_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        r = fail(AMB_ECUDA, "event creation failed");
    auto issue = [&]() -> amb_status {
        AMB_TRY(wealth_batch_small(wb, s, &launches));
        for (size_t q = 0; q < walk.size(); ++q) {
            if (walk_steps_v[q] == 0) continue;
            AMB_TRY(walk_steps(walk[q], walk_steps_v[q]));
            launches += 1;
        }
        const uint32_t steps = std::max(max_sir, max_large);
        for (uint32_t k = 0; k < steps; ++k) {
            if (k < max_sir) AMB_TRY(sir_batch_step(sb, s, &launches));
            if (k < max_large) AMB_TRY(wealth_batch_large_step(wb, s, &launches));
        }
        return AMB_OK;
    };
    if (r == AMB_OK && graph) {
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            r = fail(AMB_ECUDA, "stream capture failed to begin (is the stream the legacy default stream?)");
        } else {
            r = issue();
            const cudaError_t ec = cudaStreamEndCapture(s, &g);
            if (r == AMB_OK && ec != cudaSuccess) r = fail(AMB_ECUDA, "capture: %s", cudaGetErrorString(ec));
            if (r == AMB_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) r = fail(AMB_ECUDA, "graph instantiate failed");
        }
        if (r == AMB_OK) {
            cudaEventRecord(e0, s);
            if (cudaGraphLaunch(ge, s) != cudaSuccess) r = fail(AMB_ECUDA, "graph launch failed");
            cudaEventRecord(e1, s);
        }
    } else if (r == AMB_OK) {
        cudaEventRecord(e0, s);
        r = issue();
        cudaEventRecord(e1, s);
    }
    if (r == AMB_OK) {
        const cudaError_t es = cudaEventSynchronize(e1);
        if (es != cudaSuccess) r = fail(AMB_ECUDA, "batched steps: %s", cudaGetErrorString(es));
        float ms = 0.f;
        if (r == AMB_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out) *ms_out = ms;
        sir_batch_finish(sb, sir.data(), sir_steps.data(), (uint32_t)sir.size());
        for (size_t q = 0; q < wealth.size(); ++q) {
            wealth[q]->t += wealth_steps[q];
            wealth[q]->launches += wealth_steps[q];
        }
        for (size_t q = 0; q < walk.size(); ++q) {
            walk[q]->t += walk_steps_v[q];
            walk[q]->index_valid = false;
        }
        if (launches_out) *launches_out += launches;
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    sir_batch_release(sb, s);
    wealth_batch_release(wb, s);
    cudaStreamSynchronize(s);
    return r;
}

// The error words of every population (one synchronisation).
amb_status read_errors(const std::vector<amb_pop *> &pops, cudaStream_t s, std::vector<uint32_t> &words)
{
    words.assign(pops.size(), 0u);
    for (size_t i = 0; i < pops.size(); ++i)
        AMB_TRY_CUDA(cudaMemcpyAsync(&words[i], pops[i]->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    AMB_TRY_CUDA(cudaStreamSynchronize(s));
    return AMB_OK;
}

amb_status check_errors(const std::vector<amb_pop *> &pops, cudaStream_t s)
{
    std::vector<uint32_t> h;
    AMB_TRY(read_errors(pops, s, h));
    for (size_t i = 0; i < pops.size(); ++i) {
        if (h[i] & ERR_TIMEOUT) return fail(AMB_ETIMEOUT, "job %zu: a bounded device-side wait ran out (0x%x)", i, h[i]);
        if (h[i]) return fail(AMB_EINVARIANT, "job %zu: device reported an out-of-range value (0x%x)", i, h[i]);
    }
    return AMB_OK;
}

}  // namespace amb


namespace {

void destroy_pops(std::vector<amb_pop *> &pops)
{
    for (amb_pop *p : pops)
        if (p) amb_destroy(p);
    pops.clear();
}

amb_status create_pops(const amb_job *jobs, size_t n, cudaStream_t s, std::vector<amb_pop *> &pops)
{
    pops.assign(n, nullptr);
    for (size_t i = 0; i < n; ++i) {
        amb_params p = jobs[i].params;
        if (jobs[i].model == AMB_SIR) p.variant = AMB_SIR_BAND;
        const amb_status st = amb_create(jobs[i].model, &p, jobs[i].seed, jobs[i].replicate, s, &pops[i]);
        if (st != AMB_OK) {
            destroy_pops(pops);
            return st;
        }
    }
    return AMB_OK;
}

// Batched SIR steps of `pops` with the given band shape: `steps` steps, timed on s.
amb_status time_sir(std::vector<amb_pop *> &pops, uint32_t steps, BandShape shape, cudaStream_t s, float *ms)
{
    std::vector<uint32_t> st(pops.size(), steps);
    SirBatch sb;
    uint64_t launches = 0;
    amb_status r = sir_batch_build(sb, pops.data(), st.data(), (uint32_t)pops.size(), shape, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (r == AMB_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        r = fail(AMB_ECUDA, "event creation failed");
    if (r == AMB_OK) {
        cudaEventRecord(e0, s);
        for (uint32_t k = 0; k < steps && r == AMB_OK; ++k) r = sir_batch_step(sb, s, &launches);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) r = fail(AMB_ECUDA, "timing failed");
        if (r == AMB_OK) cudaEventElapsedTime(ms, e0, e1);
        sir_batch_finish(sb, pops.data(), st.data(), (uint32_t)pops.size());
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    sir_batch_release(sb, s);
    return r;
}

// Band shape with the shortest batched SIR step on throwaway copies of (up
// to) the eight largest SIR jobs: caps of 8, 16 and 32 rows, fewest or spread
// bands.
amb_status autotune_shape(const std::vector<amb_job> &jobs, cudaStream_t s, BandShape *best_shape)
{
    std::vector<size_t> sir;
    for (size_t i = 0; i < jobs.size(); ++i)
        if (jobs[i].model == AMB_SIR && jobs[i].params.n > 0 && jobs[i].steps > 0) sir.push_back(i);
    *best_shape = BandShape{};
    if (sir.empty()) return AMB_OK;
    std::sort(sir.begin(), sir.end(), [&](size_t a, size_t b) { return jobs[a].params.n > jobs[b].params.n; });
    if (sir.size() > 8) sir.resize(8);
    std::vector<amb_job> sample;
    for (size_t i : sir) sample.push_back(jobs[i]);
    float best = 1e30f;
    for (int spread = 0; spread < 2; ++spread) {
        for (uint32_t c : {8u, 16u, 32u}) {
            BandShape shape;
            shape.rows_cap = c;
            shape.spread = spread != 0;
            std::vector<amb_pop *> pops;
            AMB_TRY(create_pops(sample.data(), sample.size(), s, pops));
            float warm = 0.f, ms = 0.f;
            amb_status r = time_sir(pops, 1, shape, s, &warm);
            if (r == AMB_OK) r = time_sir(pops, 3, shape, s, &ms);
            if (r == AMB_OK) r = check_errors(pops, s);
            destroy_pops(pops);
            AMB_TRY(r);
            if (ms < best) {
                best = ms;
                *best_shape = shape;
            }
        }
    }
    return AMB_OK;
}

}  // namespace

extern "C" {

amb_status amb_batch_create(const amb_job *jobs, size_t n, void *cuda_stream, amb_batch **out)
{
    AMB_TRACE("amb_batch_create");
    if (!out || (!jobs && n)) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    for (size_t i = 0; i < n; ++i)
        if (jobs[i].model == AMB_SIR && jobs[i].params.variant == AMB_SIR_GENERIC)
            return fail(AMB_EINVAL, "job %zu: batches run SIR on the band path", i);
    amb_batch *b = new (std::nothrow) amb_batch();
    if (!b) return fail(AMB_ENOMEM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    b->jobs.assign(jobs, jobs + n);
    const amb_status st = create_pops(jobs, n, b->stream, b->pops);
    if (st != AMB_OK) {
        delete b;
        return st;
    }
    *out = b;
    return AMB_OK;
}

amb_status amb_batch_run(amb_batch *b, const amb_tune *tune, double *ms_out)
{
    AMB_TRACE("amb_batch_run");
    if (!b) return fail(AMB_EINVAL, "null batch");
    if (b->ran) return fail(AMB_EINVAL, "a batch runs once");
    cudaStream_t s = b->stream;
    BandShape shape;
    if (tune && tune->band_rows_cap) shape.rows_cap = std::min<uint32_t>(tune->band_rows_cap, 32u);
    shape.spread = tune && tune->spread_bands;
    const bool graph = !tune || tune->use_graph;
    if (tune && tune->autotune) AMB_TRY(autotune_shape(b->jobs, s, &shape));
    b->shape = shape;
    std::vector<uint32_t> ks(b->jobs.size());
    for (size_t i = 0; i < ks.size(); ++i) ks[i] = b->jobs[i].steps;
    uint64_t launches = 0;
    float ms = 0.f;
    AMB_TRY(advance(b->pops, ks, shape, s, graph, &launches, &ms));
    b->ms = ms;
    if (ms_out) *ms_out = ms;
    b->launches = launches;
    b->ran = true;
    return check_errors(b->pops, s);
}

amb_status amb_batch_population(amb_batch *b, size_t i, amb_pop **pop)
{
    if (!b || !pop) return fail(AMB_EINVAL, "null pointer");
    if (i >= b->pops.size()) return fail(AMB_EINVAL, "job %zu out of range", i);
    *pop = b->pops[i];
    return AMB_OK;
}

amb_status amb_batch_info(amb_batch *b, amb_batch_report *info)
{
    if (!b || !info) return fail(AMB_EINVAL, "null pointer");
    info->n_jobs = b->pops.size();
    info->band_rows_cap = b->shape.rows_cap;
    info->spread_bands = b->shape.spread ? 1 : 0;
    info->launches = b->launches;
    info->ms = b->ms;
    uint64_t as = 0;
    for (size_t i = 0; i < b->jobs.size(); ++i) as += (uint64_t)b->jobs[i].params.n * b->jobs[i].steps;
    info->agent_steps = as;
    return AMB_OK;
}

amb_status amb_batch_destroy(amb_batch *b)
{
    if (!b) return AMB_OK;
    destroy_pops(b->pops);
    delete b;
    return AMB_OK;
}

}  // extern "C"
