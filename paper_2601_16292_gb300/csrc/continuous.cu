// continuous.cu -- the paper's continuous-space models (Sec. 5.1.2 as the
// paper states them): agents in the box [0, w] x [0, h] with float32
// positions.
//   random walk: dx, dy uniform in [-s, s), the position clamped to the box;
//   SIR: a susceptible agent with k infected agents within distance r
//     becomes infected iff u2 < T_inf[min(k, K)] (thresholds of 1 - (1-p)^k);
//     an infected agent recovers after rec_steps steps; with s > 0 agents
//     first move as in the walk.
// Every float operation is one IEEE-754 single-precision operation rounded to
// nearest, written out with the _rn intrinsics so none is fused or reordered:
//   unit(u) = (u >> 8) * 2^-24, sunit(u) = ((u >> 8) - 2^23) * 2^-23 (exact);
//   x0 = w * unit(u0); x' = clamp(x + s * sunit(u0), 0, w);
//   contact iff (xi - xj)^2 + (yi - yj)^2 <= r * r, in that order.
// The infection step finds contacts through a uniform grid of cells a little
// wider than r (cell size r * 1.001): a pair at float distance <= r is at most
// one cell apart on each axis, so the 3 x 3 cells around a susceptible agent
// hold every infected agent it can touch (the quadratic all-pairs test of the
// paper's cross join, restricted to those cells).
#include <algorithm>
#include <cmath>

#include "amb_internal.cuh"

namespace amb {

amb_status host_thresholds(double beta, double gamma, uint32_t cap, uint32_t *t_inf, uint32_t *K, uint32_t *t_rec);
amb_status check_cparams(amb_model model, const amb_cparams *p, uint64_t seed);

namespace {

__device__ __forceinline__ float unit24(uint32_t u) { return __fmul_rn((float)(u >> 8), 5.9604644775390625e-8f); }

__device__ __forceinline__ float sunit24(uint32_t u)
{
    return __fmul_rn((float)((int32_t)(u >> 8) - 8388608), 1.1920928955078125e-7f);
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ void cmove(float w, float h, float s, const U4 &u, float &x, float &y)
{
    x = clampf(__fadd_rn(x, __fmul_rn(s, sunit24(u.w0))), 0.0f, w);
    y = clampf(__fadd_rn(y, __fmul_rn(s, sunit24(u.w1))), 0.0f, h);
}

struct Grid {
    float size;       // cell edge
    float inv;        // 1 / size: cell lookups multiply (monotone; the margin in size absorbs the rounding)
    uint32_t gx, gy;  // cells per axis
};

__device__ __forceinline__ uint32_t cell_coord(float v, float inv, uint32_t g)
{
    const float q = floorf(__fmul_rn(v, inv));
    const uint32_t c = q <= 0.0f ? 0u : (uint32_t)q;
    return c < g ? c : g - 1u;
}

__global__ void cinit_kernel(float *__restrict__ x, float *__restrict__ y, uint8_t *__restrict__ state,
                             int32_t *__restrict__ days, uint32_t n, float w, float h, uint32_t n0, uint32_t k0,
                             uint32_t k1)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const U4 u = philox(i, kInitStep, k0, k1);
        x[i] = __fmul_rn(w, unit24(u.w0));
        y[i] = __fmul_rn(h, unit24(u.w1));
        if (state) {
            state[i] = (i < n0) ? (uint8_t)AMB_I : (uint8_t)AMB_S;
            days[i] = 0;
        }
    }
}

// k walk steps per agent in registers; block 0 writes the count rows {n, 0, 0, 0}
__global__ void cwalk_kernel(float *__restrict__ x, float *__restrict__ y, uint32_t n, float w, float h, float s,
                             uint32_t k0, uint32_t k1, uint32_t t0, uint32_t k, int64_t *__restrict__ rows)
{
    if (blockIdx.x == 0)
        for (uint32_t j = threadIdx.x; j < k; j += blockDim.x) {
            rows[j * 4u] = n;
            rows[j * 4u + 1] = rows[j * 4u + 2] = rows[j * 4u + 3] = 0;
        }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float xi = x[i], yi = y[i];
        for (uint32_t j = 0; j < k; ++j) cmove(w, h, s, philox(i, t0 + j, k0, k1), xi, yi);
        x[i] = xi;
        y[i] = yi;
    }
}

// SIR step, launch 1: moves (s > 0); start-of-step infected agents counted per cell
__global__ void csir_move_kernel(float *__restrict__ x, float *__restrict__ y, const uint8_t *__restrict__ state,
                                 uint32_t n, float w, float h, float s, uint32_t k0, uint32_t k1, uint32_t t, Grid g,
                                 int32_t *__restrict__ cell, int32_t *__restrict__ cnt)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float xi = x[i], yi = y[i];
        if (s > 0.0f) {
            cmove(w, h, s, philox(i, t, k0, k1), xi, yi);
            x[i] = xi;
            y[i] = yi;
        }
        if (state[i] == AMB_I) {
            const uint32_t c = cell_coord(yi, g.inv, g.gy) * g.gx + cell_coord(xi, g.inv, g.gx);
            cell[i] = (int32_t)c;
            atomicAdd(&cnt[c], 1);
        }
    }
}

// launch 3: the infected agents' positions in cell order
__global__ void csir_scatter_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                    const uint8_t *__restrict__ state, const int32_t *__restrict__ cell, uint32_t n,
                                    int32_t *__restrict__ cursor, float2 *__restrict__ inf_pos)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] != AMB_I) continue;
        const int32_t slot = atomicAdd(&cursor[cell[i]], 1);
        inf_pos[slot] = make_float2(x[i], y[i]);
    }
}

// launch 4: infection (susceptible agents count infected contacts in the 3 x 3
// cells around them) and recovery; S / I / R / new-infection counts
__global__ void csir_contact_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                    uint8_t *__restrict__ state, int32_t *__restrict__ days, uint32_t n, Grid g,
                                    const int32_t *__restrict__ start, const float2 *__restrict__ inf_pos, float r2,
                                    uint32_t k0, uint32_t k1, uint32_t t, const uint32_t *__restrict__ t_inf,
                                    uint32_t K, uint32_t rec_steps, int64_t *__restrict__ row)
{
    uint32_t cs = 0, ci = 0, cr = 0, fresh = 0;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        uint32_t st = state[j];
        if (st == AMB_S) {
            const float xj = x[j], yj = y[j];
            const uint32_t cx = cell_coord(xj, g.inv, g.gx), cy = cell_coord(yj, g.inv, g.gy);
            uint32_t k = 0;
            const uint32_t y0 = cy ? cy - 1u : 0u, y1 = min(cy + 1u, g.gy - 1u);
            const uint32_t x0 = cx ? cx - 1u : 0u, x1 = min(cx + 1u, g.gx - 1u);
            for (uint32_t yy = y0; yy <= y1; ++yy) {
                const int32_t b = start[yy * g.gx + x0], e = start[yy * g.gx + x1 + 1u];
                for (int32_t q = b; q < e; ++q) {
                    const float2 p = inf_pos[q];
                    const float dx = __fsub_rn(p.x, xj), dy = __fsub_rn(p.y, yj);
                    const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                    k += (d2 <= r2) ? 1u : 0u;
                }
            }
            if (k) {
                const U4 u = philox(j, t, k0, k1);
                if (u.w2 < t_inf[k < K ? k : K]) {
                    st = AMB_I;
                    state[j] = (uint8_t)AMB_I;
                    days[j] = 0;
                    ++fresh;
                }
            }
        } else if (st == AMB_I) {
            const int32_t d = days[j] + 1;
            days[j] = d;
            if ((uint32_t)d >= rec_steps) {
                st = AMB_R;
                state[j] = (uint8_t)AMB_R;
            }
        }
        cs += (st == AMB_S);
        ci += (st == AMB_I);
        cr += (st == AMB_R);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cs += __shfl_down_sync(0xffffffffu, cs, o);
        ci += __shfl_down_sync(0xffffffffu, ci, o);
        cr += __shfl_down_sync(0xffffffffu, cr, o);
        fresh += __shfl_down_sync(0xffffffffu, fresh, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        unsigned long long *r = reinterpret_cast<unsigned long long *>(row);
        if (cs) atomicAdd(&r[0], (unsigned long long)cs);
        if (ci) atomicAdd(&r[1], (unsigned long long)ci);
        if (cr) atomicAdd(&r[2], (unsigned long long)cr);
        if (fresh) atomicAdd(&r[3], (unsigned long long)fresh);
    }
}

// Small populations: one CTA runs all k steps with positions, per-cell counts
// and the infected agents' positions in shared memory (the same arithmetic as
// the four-launch path; no launch per step).
constexpr int kSmallNT = 1024;
constexpr uint32_t kSmallMaxN = 8192;
constexpr uint32_t kSmallMaxCells = 4096;

__global__ void __launch_bounds__(kSmallNT) csir_small_kernel(float *__restrict__ gx_, float *__restrict__ gy_,
                                                              uint8_t *__restrict__ state, int32_t *__restrict__ days,
                                                              uint32_t n, float w, float h, float s, Grid g, float r2,
                                                              uint32_t k0, uint32_t k1, uint32_t t0, uint32_t k,
                                                              const uint32_t *__restrict__ t_inf, uint32_t K,
                                                              uint32_t rec_steps, int64_t *__restrict__ rows)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *x = reinterpret_cast<float *>(smem_raw);
    float *y = x + kSmallMaxN;
    float2 *inf = reinterpret_cast<float2 *>(y + kSmallMaxN);
    int32_t *start = reinterpret_cast<int32_t *>(inf + kSmallMaxN);  // kSmallMaxCells + 1
    int32_t *cursor = start + kSmallMaxCells + 1;                     // kSmallMaxCells
    __shared__ uint32_t s_warp[kSmallNT / 32 + 1];
    __shared__ unsigned long long s_cnt[4];
    const uint32_t tid = threadIdx.x, C = g.gx * g.gy;
    for (uint32_t i = tid; i < n; i += kSmallNT) {
        x[i] = gx_[i];
        y[i] = gy_[i];
    }
    for (uint32_t j = 0; j < k; ++j) {
        const uint32_t t = t0 + j;
        for (uint32_t c = tid; c < C; c += kSmallNT) cursor[c] = 0;
        if (tid < 4) s_cnt[tid] = 0ull;
        __syncthreads();
        // moves; start-of-step infected agents per cell
        for (uint32_t i = tid; i < n; i += kSmallNT) {
            float xi = x[i], yi = y[i];
            if (s > 0.0f) {
                cmove(w, h, s, philox(i, t, k0, k1), xi, yi);
                x[i] = xi;
                y[i] = yi;
            }
            if (state[i] == AMB_I)
                atomicAdd(&cursor[cell_coord(yi, g.inv, g.gy) * g.gx + cell_coord(xi, g.inv, g.gx)], 1);
        }
        __syncthreads();
        // exclusive scan of the counts: four cells per thread
        {
            uint32_t c4[4], sum = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t c = tid * 4u + (uint32_t)e;
                c4[e] = c < C ? (uint32_t)cursor[c] : 0u;
                sum += c4[e];
            }
            uint32_t total;
            uint32_t off = block_exclusive_scan<kSmallNT>(sum, s_warp, &total);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t c = tid * 4u + (uint32_t)e;
                if (c < C) {
                    start[c] = (int32_t)off;
                    cursor[c] = (int32_t)off;
                }
                off += c4[e];
            }
            if (tid == 0) start[C] = (int32_t)total;
        }
        __syncthreads();
        for (uint32_t i = tid; i < n; i += kSmallNT) {
            if (state[i] != AMB_I) continue;
            const float xi = x[i], yi = y[i];
            const int32_t slot = atomicAdd(&cursor[cell_coord(yi, g.inv, g.gy) * g.gx + cell_coord(xi, g.inv, g.gx)], 1);
            inf[slot] = make_float2(xi, yi);
        }
        __syncthreads();
        // infection and recovery against the start-of-step infected set
        uint32_t cs = 0, ci = 0, cr = 0, fresh = 0;
        for (uint32_t i = tid; i < n; i += kSmallNT) {
            uint32_t st = state[i];
            if (st == AMB_S) {
                const float xj = x[i], yj = y[i];
                const uint32_t cx = cell_coord(xj, g.inv, g.gx), cy = cell_coord(yj, g.inv, g.gy);
                const uint32_t ya = cy ? cy - 1u : 0u, yb = min(cy + 1u, g.gy - 1u);
                const uint32_t xa = cx ? cx - 1u : 0u, xb = min(cx + 1u, g.gx - 1u);
                uint32_t kk = 0;
                for (uint32_t yy = ya; yy <= yb; ++yy) {
                    const int32_t b = start[yy * g.gx + xa], e = start[yy * g.gx + xb + 1u];
                    for (int32_t q = b; q < e; ++q) {
                        const float2 p = inf[q];
                        const float dx = __fsub_rn(p.x, xj), dy = __fsub_rn(p.y, yj);
                        kk += (__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) <= r2) ? 1u : 0u;
                    }
                }
                if (kk) {
                    const U4 u = philox(i, t, k0, k1);
                    if (u.w2 < t_inf[kk < K ? kk : K]) {
                        st = AMB_I;
                        state[i] = (uint8_t)AMB_I;
                        days[i] = 0;
                        ++fresh;
                    }
                }
            } else if (st == AMB_I) {
                const int32_t d = days[i] + 1;
                days[i] = d;
                if ((uint32_t)d >= rec_steps) {
                    st = AMB_R;
                    state[i] = (uint8_t)AMB_R;
                }
            }
            cs += (st == AMB_S);
            ci += (st == AMB_I);
            cr += (st == AMB_R);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cs += __shfl_down_sync(0xffffffffu, cs, o);
            ci += __shfl_down_sync(0xffffffffu, ci, o);
            cr += __shfl_down_sync(0xffffffffu, cr, o);
            fresh += __shfl_down_sync(0xffffffffu, fresh, o);
        }
        if ((tid & 31u) == 0) {
            if (cs) atomicAdd(&s_cnt[0], (unsigned long long)cs);
            if (ci) atomicAdd(&s_cnt[1], (unsigned long long)ci);
            if (cr) atomicAdd(&s_cnt[2], (unsigned long long)cr);
            if (fresh) atomicAdd(&s_cnt[3], (unsigned long long)fresh);
        }
        __syncthreads();
        if (tid < 4) rows[(size_t)j * 4u + tid] = (int64_t)s_cnt[tid];
        __syncthreads();
    }
    for (uint32_t i = tid; i < n; i += kSmallNT) {
        gx_[i] = x[i];
        gy_[i] = y[i];
    }
}

constexpr size_t kSmallSmem =
    (size_t)kSmallMaxN * (4u + 4u + 8u) + ((size_t)kSmallMaxCells * 2u + 1u) * 4u;

// coordinates outside the box (or NaN)
__global__ void cbounds_kernel(const float *__restrict__ v, uint32_t n, float hi, unsigned long long *bad)
{
    uint32_t b = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        b += !(v[i] >= 0.0f && v[i] <= hi);
    if (b) atomicAdd(bad, (unsigned long long)b);
}

__global__ void cdays_check_kernel(const int32_t *__restrict__ v, uint32_t n, unsigned long long *bad)
{
    uint32_t b = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b += v[i] < 0;
    if (b) atomicAdd(bad, (unsigned long long)b);
}

__global__ void cstate_check_kernel(const uint8_t *__restrict__ v, uint32_t n, unsigned long long *bad)
{
    uint32_t b = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b += v[i] > 2u;
    if (b) atomicAdd(bad, (unsigned long long)b);
}

Grid grid_of(const amb_cparams &p)
{
    // cells a little wider than r, at most 1024 per axis
    const float ext = std::max(p.width, p.height);
    float size = std::max(p.radius * 1.001f, ext / 1024.0f);
    if (!(size > 0.0f)) size = 1.0f;  // empty box: one cell
    Grid g;
    g.size = size;
    g.inv = 1.0f / size;
    g.gx = (uint32_t)std::min(1024.0f, std::max(1.0f, std::ceil(p.width / size)));
    g.gy = (uint32_t)std::min(1024.0f, std::max(1.0f, std::ceil(p.height / size)));
    return g;
}

}  // namespace

bool is_continuous(const amb_pop *pop) { return pop->model == AMB_CWALK || pop->model == AMB_CSIR; }

amb_status cont_init(amb_pop *pop)
{
    cudaStream_t s = pop->stream;
    const uint32_t n = pop->cp.n;
    AMB_TRY(dalloc(&pop->fx, n, s));
    AMB_TRY(dalloc(&pop->fy, n, s));
    if (pop->model == AMB_CSIR) {
        AMB_TRY(dalloc(&pop->state, n, s));
        AMB_TRY(dalloc(&pop->days, n, s));
        const uint32_t cap = n > 0 ? n : 1;
        pop->t_inf_h.assign((size_t)cap + 1, 0u);
        AMB_TRY(host_thresholds(pop->cp.p_infect, 0.0, cap, pop->t_inf_h.data(), &pop->K, &pop->t_rec));
        pop->t_inf_h.resize((size_t)pop->K + 1);
        AMB_TRY(dalloc(&pop->t_inf_d, pop->t_inf_h.size(), s));
        AMB_TRY_CUDA(cudaMemcpyAsync(pop->t_inf_d, pop->t_inf_h.data(), pop->t_inf_h.size() * sizeof(uint32_t),
                                     cudaMemcpyHostToDevice, s));
        const Grid g = grid_of(pop->cp);
        const uint32_t C = g.gx * g.gy;
        AMB_TRY(dalloc(&pop->cell, n, s));
        AMB_TRY(dalloc(&pop->cnt, C, s));
        AMB_TRY(dalloc(&pop->start, (size_t)C + 1, s));
        AMB_TRY(dalloc(&pop->cursor, (size_t)C + 1, s));
        AMB_TRY(dalloc(&pop->inf_pos, n, s));
        pop->init_infected = pop->cp.n_init_infected;
    }
    if (n)
        cinit_kernel<<<grid_for(n, 256, 16u), 256, 0, s>>>(pop->fx, pop->fy, pop->state, pop->days, n,
                                                                  pop->cp.width, pop->cp.height,
                                                                  pop->cp.n_init_infected, pop->key0, pop->key1);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status cont_steps(amb_pop *pop, uint32_t k)
{
    cudaStream_t s = pop->stream;
    const amb_cparams &p = pop->cp;
    const uint32_t n = p.n;
    int64_t *rows = pop->series + (size_t)pop->t * 4u;
    if (pop->model == AMB_CWALK) {
        cwalk_kernel<<<grid_for(n, 256, 32u), 256, 0, s>>>(pop->fx, pop->fy, n, p.width, p.height, p.step,
                                                                  pop->key0, pop->key1, (uint32_t)pop->t, k, rows);
        AMB_TRY_CUDA(cudaGetLastError());
        pop->launches += 1;
        return AMB_OK;
    }
    const Grid g = grid_of(p);
    const uint32_t C = g.gx * g.gy;
    const float r2 = p.radius * p.radius;
    if (n <= kSmallMaxN && C <= kSmallMaxCells) {
        // the whole run in one CTA (rows are written for every step)
        AMB_TRY_CUDA(cudaFuncSetAttribute(csir_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kSmallSmem));
        csir_small_kernel<<<1, kSmallNT, kSmallSmem, s>>>(pop->fx, pop->fy, pop->state, pop->days, n, p.width,
                                                           p.height, p.step, g, r2, pop->key0, pop->key1,
                                                           (uint32_t)pop->t, k, pop->t_inf_d, pop->K,
                                                           p.recovery_steps, rows);
        AMB_TRY_CUDA(cudaGetLastError());
        pop->launches += 1;
        return AMB_OK;
    }
    AMB_TRY_CUDA(cudaMemsetAsync(rows, 0, (size_t)k * 4u * sizeof(int64_t), s));
    const unsigned grid = grid_for(n, 256, 16u);
    for (uint32_t j = 0; j < k; ++j) {
        const uint32_t t = (uint32_t)(pop->t + j);
        AMB_TRY_CUDA(cudaMemsetAsync(pop->cnt, 0, (size_t)C * sizeof(int32_t), s));
        csir_move_kernel<<<grid, 256, 0, s>>>(pop->fx, pop->fy, pop->state, n, p.width, p.height, p.step, pop->key0,
                                              pop->key1, t, g, pop->cell, pop->cnt);
        AMB_TRY_CUDA(cudaGetLastError());
        AMB_TRY(launch_scan(pop->cnt, pop->start, pop->cursor, C, pop->lb, pop->err, s));
        csir_scatter_kernel<<<grid, 256, 0, s>>>(pop->fx, pop->fy, pop->state, pop->cell, n, pop->cursor,
                                                 pop->inf_pos);
        csir_contact_kernel<<<grid, 256, 0, s>>>(pop->fx, pop->fy, pop->state, pop->days, n, g, pop->start,
                                                 pop->inf_pos, r2, pop->key0, pop->key1, t, pop->t_inf_d, pop->K,
                                                 p.recovery_steps, rows + (size_t)j * 4u);
        AMB_TRY_CUDA(cudaGetLastError());
        pop->launches += 4;
    }
    return AMB_OK;
}

static bool cont_col_ok(const amb_pop *pop, amb_col col)
{
    if (col == AMB_COL_X || col == AMB_COL_Y) return true;
    return pop->model == AMB_CSIR && (col == AMB_COL_STATE || col == AMB_COL_DAYS);
}

static void *cont_col_ptr(amb_pop *pop, amb_col col)
{
    switch (col) {
    case AMB_COL_X: return pop->fx;
    case AMB_COL_Y: return pop->fy;
    case AMB_COL_STATE: return pop->state;
    default: return pop->days;
    }
}

amb_status cont_read_column(amb_pop *pop, amb_col col, void *dst, size_t n, int dst_on_device)
{
    if (!cont_col_ok(pop, col)) return fail(AMB_EINVAL, "column %d does not belong to this model", (int)col);
    const size_t esz = (col == AMB_COL_STATE) ? 1 : 4;
    if (n)
        AMB_TRY_CUDA(cudaMemcpyAsync(dst, cont_col_ptr(pop, col), n * esz,
                                     dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, pop->stream));
    AMB_TRY_CUDA(cudaStreamSynchronize(pop->stream));
    return AMB_OK;
}

amb_status cont_write_column(amb_pop *pop, amb_col col, const void *src, size_t n, int src_on_device)
{
    if (!cont_col_ok(pop, col)) return fail(AMB_EINVAL, "column %d does not belong to this model", (int)col);
    cudaStream_t s = pop->stream;
    const size_t esz = (col == AMB_COL_STATE) ? 1 : 4;
    unsigned char *tmp = nullptr;
    unsigned long long *bad = nullptr;
    AMB_TRY(dalloc(&tmp, n * esz, s));
    amb_status st = dalloc(&bad, 1, s);
    if (st == AMB_OK && cudaMemsetAsync(bad, 0, sizeof(*bad), s) != cudaSuccess) st = fail(AMB_ECUDA, "memset failed");
    if (st == AMB_OK && n &&
        cudaMemcpyAsync(tmp, src, n * esz, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        st = fail(AMB_ECUDA, "column upload failed");
    if (st == AMB_OK && n) {
        const unsigned g = grid_for(n, 256, 8u);
        if (col == AMB_COL_X || col == AMB_COL_Y)
            cbounds_kernel<<<g, 256, 0, s>>>(reinterpret_cast<const float *>(tmp), (uint32_t)n,
                                             col == AMB_COL_X ? pop->cp.width : pop->cp.height, bad);
        else if (col == AMB_COL_STATE)
            cstate_check_kernel<<<g, 256, 0, s>>>(tmp, (uint32_t)n, bad);
        else
            cdays_check_kernel<<<g, 256, 0, s>>>(reinterpret_cast<const int32_t *>(tmp), (uint32_t)n, bad);
        unsigned long long h = 0;
        if (cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = fail(AMB_ECUDA, "column check failed");
        else if (h)
            st = fail(AMB_EINVAL, "%llu values out of range", h);
    }
    if (st == AMB_OK && n &&
        cudaMemcpyAsync(cont_col_ptr(pop, col), tmp, n * esz, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        st = fail(AMB_ECUDA, "column copy failed");
    if (st == AMB_OK && pop->model == AMB_CSIR && col == AMB_COL_STATE) pop->monotone_from = pop->t;
    dfree(tmp, s);
    dfree(bad, s);
    cudaStreamSynchronize(s);
    return st;
}

// coordinates inside the box (bounds_ok)
amb_status cont_bounds(amb_pop *pop, bool *ok)
{
    cudaStream_t s = pop->stream;
    unsigned long long *bad = nullptr;
    AMB_TRY(dalloc(&bad, 1, s));
    AMB_TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(*bad), s));
    const uint32_t n = pop->cp.n;
    if (n) {
        const unsigned g = grid_for(n, 256, 8u);
        cbounds_kernel<<<g, 256, 0, s>>>(pop->fx, n, pop->cp.width, bad);
        cbounds_kernel<<<g, 256, 0, s>>>(pop->fy, n, pop->cp.height, bad);
    }
    unsigned long long h = 0;
    AMB_TRY_CUDA(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s));
    AMB_TRY_CUDA(cudaStreamSynchronize(s));
    dfree(bad, s);
    *ok = (h == 0);
    return AMB_OK;
}

void cont_release(amb_pop *pop)
{
    cudaStream_t s = pop->stream;
    dfree(pop->fx, s);
    dfree(pop->fy, s);
    dfree(pop->days, s);
    dfree(pop->cell, s);
    dfree(pop->inf_pos, s);
}

}  // namespace amb

using namespace amb;

extern "C" amb_status amb_create_continuous(amb_model model, const amb_cparams *p, uint64_t seed, uint32_t replicate,
                                            void *cuda_stream, amb_pop **out)
{
    AMB_TRACE("amb_create_continuous");
    if (!p || !out) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    AMB_TRY(check_cparams(model, p, seed));
    if (injected_create_failure()) return fail(AMB_ENOMEM, "injected creation failure");
    amb_pop *pop = new (std::nothrow) amb_pop();
    if (!pop) return fail(AMB_ENOMEM, "host allocation failed");
    pop->model = model;
    pop->cp = *p;
    memset(&pop->p, 0, sizeof(pop->p));
    pop->p.n = p->n;
    pop->p.n_init_infected = p->n_init_infected;
    pop->key0 = (uint32_t)seed;
    pop->key1 = replicate;
    pop->stream = (cudaStream_t)cuda_stream;
    amb_status st = dalloc(&pop->err, 1, pop->stream);
    if (st == AMB_OK && cudaMemsetAsync(pop->err, 0, sizeof(uint32_t), pop->stream) != cudaSuccess)
        st = fail(AMB_ECUDA, "memset failed");
    if (st == AMB_OK) st = ensure_series(pop, 64);
    if (st == AMB_OK) st = cont_init(pop);
    if (st == AMB_OK && cudaStreamSynchronize(pop->stream) != cudaSuccess) st = fail(AMB_ECUDA, "initialisation failed");
    if (st != AMB_OK) {
        amb_destroy(pop);
        return st;
    }
    *out = pop;
    return AMB_OK;
}
