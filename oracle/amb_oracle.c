/*
 * amb_oracle.c -- plain, slow, single-threaded CPU statement of the AMBER
 * per-step population update (wealth transfer, random walk on a torus grid,
 * spatial SIR on a grid), used as the parity oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs
 * of bench.py load it.  It shares no source with the CUDA library (its own
 * Philox, its own threshold tables, its own index and statistics).
 *
 * Every loop runs over agents in id order on plain arrays.  Synchronous
 * (snapshot-then-apply) semantics throughout (paper Sec. 3.4): every agent
 * reads the state as it was at the start of the step.
 *
 * Where the paper is silent, the reading taken is stated next to the code
 * that implements it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -shared -fPIC (oracle/build.py).
 * -ffp-contract=off matters: the threshold tables are defined by individual
 * IEEE-754 double operations and must not be fused into FMAs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

#define ST_S 0
#define ST_I 1
#define ST_R 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Written from the published round function:    */
/* two 32x32->64 products per round, the high halves xor-ed with the other  */
/* two words and the round key, the key bumped by the Weyl constants        */
/* between rounds, ten rounds.                                              */
/* ------------------------------------------------------------------------ */
static const uint32_t PH_MUL_A = 0xD2511F53u; /* multiplies word 0 */
static const uint32_t PH_MUL_B = 0xCD9E8D57u; /* multiplies word 2 */
static const uint32_t PH_WEYL_0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PH_WEYL_1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t w0 = ctr[0], w1 = ctr[1], w2 = ctr[2], w3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t pa = (uint64_t)PH_MUL_A * (uint64_t)w0;
        uint64_t pb = (uint64_t)PH_MUL_B * (uint64_t)w2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ w1 ^ k0;
        uint32_t n1 = (uint32_t)pb;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ w3 ^ k1;
        uint32_t n3 = (uint32_t)pa;
        w0 = n0; w1 = n1; w2 = n2; w3 = n3;
        k0 += PH_WEYL_0;
        k1 += PH_WEYL_1;
    }
    out[0] = w0; out[1] = w1; out[2] = w2; out[3] = w3;
}

/* The draw of one agent at one step: key = (seed, replicate), counter =
 * (agent id, step, 0, 0).  Initial positions use step = 0xFFFFFFFF. */
static void draw(uint32_t seed, uint32_t rep, uint32_t id, uint32_t step, uint32_t u[4])
{
    uint32_t c[4] = {id, step, 0u, 0u};
    uint32_t k[2] = {seed, rep};
    orc_philox4x32_10(c, k, u);
}

#define INIT_STEP 0xFFFFFFFFu

/* Uniform integer in [0, n): the high word of u * n (no rejection). */
static uint32_t uniform_below(uint32_t u, uint32_t n)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* Moore neighbourhood, direction d = top three bits of the move word. */
static const int MOORE_DX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
static const int MOORE_DY[8] = {-1, -1, -1, 0, 0, 1, 1, 1};

/* Non-negative residue of (v + d) on a ring of L sites, v in [0, L). */
static int32_t wrap_add(int32_t v, int d, uint32_t L)
{
    int64_t s = (int64_t)v + d;
    int64_t m = (int64_t)L;
    s %= m;
    if (s < 0) s += m;
    return (int32_t)s;
}

/* ------------------------------------------------------------------------ */
/* Initialisation (paper Sec. 3.3, add_agents: one call creates n agents).  */
/* ------------------------------------------------------------------------ */
void orc_init_wealth(uint32_t n, int32_t w_init, int32_t *w)
{
    for (uint32_t i = 0; i < n; ++i) w[i] = w_init;
}

/* Positions uniform on the L x L torus: x from word 0, y from word 1 of the
 * agent's initial draw. */
void orc_init_positions(uint32_t n, uint32_t L, uint32_t seed, uint32_t rep,
                        int32_t *x, int32_t *y)
{
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u[4];
        draw(seed, rep, i, INIT_STEP, u);
        x[i] = (int32_t)uniform_below(u[0], L);
        y[i] = (int32_t)uniform_below(u[1], L);
    }
}

/* Initial infected: agents 0 .. n0-1 (their positions are independent
 * uniform draws, so they form a uniformly random spatial sample); the count
 * equals the configured parameter exactly (paper Sec. 5.1.3). */
void orc_init_sir_state(uint32_t n, uint32_t n0, uint8_t *state)
{
    for (uint32_t i = 0; i < n; ++i) state[i] = (i < n0) ? ST_I : ST_S;
}

/* ------------------------------------------------------------------------ */
/* Wealth transfer (paper Sec. 5.1.2; Listings 2-3).                        */
/* Every agent with positive wealth (on the snapshot) gives one unit to a   */
/* uniformly chosen OTHER agent: r' = uniform_below(u0, n-1), r = r' + (r'  */
/* >= i).  Duplicate recipients accumulate (scatter_add).  n == 1: no agent */
/* has another agent to give to, so nothing happens.                        */
/* counts[0] = donors this step, counts[1] = total wealth after the step.   */
/* Arithmetic on wealth wraps modulo 2^32.                                  */
/* ------------------------------------------------------------------------ */
int orc_wealth_step(uint32_t n, uint32_t seed, uint32_t rep, uint32_t t,
                    int32_t *w, int64_t counts[4])
{
    counts[0] = counts[1] = counts[2] = counts[3] = 0;
    if (n >= 2) {
        int32_t *snap = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (!snap) return ORC_ENOMEM;
        memcpy(snap, w, sizeof(int32_t) * (size_t)n);
        for (uint32_t i = 0; i < n; ++i) {
            if (snap[i] > 0) {
                uint32_t u[4];
                draw(seed, rep, i, t, u);
                uint32_t r = uniform_below(u[0], n - 1);
                if (r >= i) r += 1;
                w[i] = (int32_t)((uint32_t)w[i] - 1u);
                w[r] = (int32_t)((uint32_t)w[r] + 1u);
                counts[0] += 1;
            }
        }
        free(snap);
    }
    for (uint32_t i = 0; i < n; ++i) counts[1] += w[i];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Random walk (paper Sec. 5.1.2, re-cast on an integer torus): every agent */
/* steps to one of its 8 Moore neighbours, direction = u0 >> 29.            */
/* ------------------------------------------------------------------------ */
int orc_walk_step(uint32_t n, uint32_t L, uint32_t seed, uint32_t rep, uint32_t t,
                  int32_t *x, int32_t *y)
{
    if (L == 0) return ORC_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u[4];
        draw(seed, rep, i, t, u);
        uint32_t d = u[0] >> 29;
        x[i] = wrap_add(x[i], MOORE_DX[d], L);
        y[i] = wrap_add(y[i], MOORE_DY[d], L);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SIR probabilities as uint32 thresholds; an event with probability p      */
/* happens iff the uniform word u < T(p), T(p) = min(floor(p 2^32), 2^32-1).*/
/* Infection with k infected cell-mates: p_k = 1 - (1-beta)^k, where        */
/* (1-beta)^k is built by k successive IEEE double products (no pow()).     */
/* t_inf[0] = 0.  The table ends at K: the first k whose entry is the       */
/* largest uint32, or after which the power no longer changes, or k = cap;  */
/* every entry beyond K equals t_inf[K], so lookups use min(k, K).          */
/* ------------------------------------------------------------------------ */
static uint32_t prob_to_threshold(double p)
{
    double v = p * 4294967296.0; /* exact scaling by 2^32 */
    if (!(v > 0.0)) return 0u;
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)v; /* truncation == floor for v >= 0 */
}

int orc_sir_thresholds(double beta, double gamma, uint32_t cap,
                       uint32_t *t_inf, uint32_t *K_out, uint32_t *t_rec)
{
    if (!(beta >= 0.0 && beta <= 1.0) || !(gamma >= 0.0 && gamma <= 1.0)) return ORC_EINVAL;
    if (cap < 1) cap = 1;
    double keep = 1.0 - beta; /* survival factor for one infected cell-mate */
    double q = 1.0;           /* probability of escaping k infected */
    t_inf[0] = 0u;
    uint32_t K = cap;
    for (uint32_t k = 1; k <= cap; ++k) {
        double q_next = q * keep;
        double p = 1.0 - q_next;
        t_inf[k] = prob_to_threshold(p);
        if (t_inf[k] == 0xFFFFFFFFu) { K = k; break; }
        if (q_next == q) { K = (k > 1) ? k - 1 : 1; break; }
        q = q_next;
    }
    *K_out = K;
    *t_rec = prob_to_threshold(gamma);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Spatial SIR on the grid (paper Sec. 5.1.2, re-cast with same-cell         */
/* contacts).  One step t:                                                   */
/*  1. every agent (S, I and R) makes its Moore move as in the random walk;  */
/*  2. with the states of the start of the step, k[c] = number of infected   */
/*     agents whose NEW cell is c;                                           */
/*  3. S agent in cell c with k[c] >= 1 becomes I iff u1 < t_inf[min(k,K)];  */
/*     I agent (start-of-step state) becomes R iff u2 < t_rec; R stays R.    */
/*     An agent infected in this step does not recover in this step.        */
/* counts = {S, I, R, new infections} after the step.                       */
/* ------------------------------------------------------------------------ */
int orc_sir_step(uint32_t n, uint32_t L, uint32_t seed, uint32_t rep, uint32_t t,
                 const uint32_t *t_inf, uint32_t K, uint32_t t_rec,
                 int32_t *x, int32_t *y, uint8_t *state, int64_t counts[4])
{
    if (L == 0) return ORC_EINVAL;
    uint64_t C = (uint64_t)L * (uint64_t)L;
    uint32_t *u1 = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t *u2 = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t *kc = (uint32_t *)calloc((size_t)C, sizeof(uint32_t));
    if (!u1 || !u2 || !kc) { free(u1); free(u2); free(kc); return ORC_ENOMEM; }

    /* 1. moves */
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u[4];
        draw(seed, rep, i, t, u);
        uint32_t d = u[0] >> 29;
        x[i] = wrap_add(x[i], MOORE_DX[d], L);
        y[i] = wrap_add(y[i], MOORE_DY[d], L);
        u1[i] = u[1];
        u2[i] = u[2];
    }
    /* 2. infected per new cell, start-of-step states */
    for (uint32_t i = 0; i < n; ++i)
        if (state[i] == ST_I) kc[(uint64_t)y[i] * L + (uint64_t)x[i]] += 1;
    /* 3. transitions against the snapshot */
    int64_t newinf = 0;
    for (uint32_t i = 0; i < n; ++i) {
        uint8_t s = state[i];
        if (s == ST_S) {
            uint32_t k = kc[(uint64_t)y[i] * L + (uint64_t)x[i]];
            if (k >= 1) {
                uint32_t kk = (k < K) ? k : K;
                if (u1[i] < t_inf[kk]) { state[i] = ST_I; newinf += 1; }
            }
        } else if (s == ST_I) {
            if (u2[i] < t_rec) state[i] = ST_R;
        }
    }
    counts[0] = counts[1] = counts[2] = 0;
    for (uint32_t i = 0; i < n; ++i) counts[state[i]] += 1; /* states are 0, 1, 2 */
    counts[3] = newinf;
    free(u1); free(u2); free(kc);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Counting-sort cell index (paper Sec. 4.1, grid environment): cell id     */
/* c = y * L + x; start[c] = number of agents in cells < c; start[C] = n;   */
/* perm lists agent ids cell by cell, ascending id inside a cell (a stable  */
/* counting sort).                                                          */
/* ------------------------------------------------------------------------ */
int orc_cell_index(uint32_t n, uint32_t L, const int32_t *x, const int32_t *y,
                   int64_t *start, int32_t *perm)
{
    if (L == 0) return ORC_EINVAL;
    uint64_t C = (uint64_t)L * (uint64_t)L;
    int64_t *cursor = (int64_t *)calloc((size_t)C, sizeof(int64_t));
    if (!cursor) return ORC_ENOMEM;
    for (uint64_t c = 0; c <= C; ++c) start[c] = 0;
    for (uint32_t i = 0; i < n; ++i) start[(uint64_t)y[i] * L + (uint64_t)x[i] + 1] += 1;
    for (uint64_t c = 0; c < C; ++c) start[c + 1] += start[c];
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t c = (uint64_t)y[i] * L + (uint64_t)x[i];
        perm[start[c] + cursor[c]] = (int32_t)i;
        cursor[c] += 1;
    }
    free(cursor);
    return ORC_OK;
}

/* Occupancy per cell (occ[C]) and the histogram of occupancies
 * (hist[m] = number of cells holding m agents, m < hist_len). */
int orc_occupancy(uint32_t n, uint32_t L, const int32_t *x, const int32_t *y,
                  int32_t *occ, int64_t *hist, uint32_t hist_len)
{
    if (L == 0) return ORC_EINVAL;
    uint64_t C = (uint64_t)L * (uint64_t)L;
    for (uint64_t c = 0; c < C; ++c) occ[c] = 0;
    for (uint32_t i = 0; i < n; ++i) occ[(uint64_t)y[i] * L + (uint64_t)x[i]] += 1;
    for (uint32_t m = 0; m < hist_len; ++m) hist[m] = 0;
    for (uint64_t c = 0; c < C; ++c)
        if ((uint32_t)occ[c] < hist_len) hist[occ[c]] += 1;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Gini coefficient of the wealth column, from the ascending order          */
/* statistics w_(1) <= ... <= w_(n):                                        */
/*   G = sum_i (2i - n - 1) w_(i) / (n * sum_i w_i),                         */
/* numerator and denominator as exact integers, then one double division.   */
/* sum w == 0 gives G = 0.                                                  */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int orc_gini(uint32_t n, const int32_t *w, double *gini, int64_t *num_hi, uint64_t *num_lo,
             int64_t *total)
{
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!s) return ORC_ENOMEM;
    memcpy(s, w, sizeof(int32_t) * (size_t)n);
    qsort(s, n, sizeof(int32_t), cmp_i32);
    __int128 num = 0;
    int64_t tot = 0;
    for (uint32_t i = 0; i < n; ++i) {
        int64_t coef = 2 * (int64_t)(i + 1) - (int64_t)n - 1;
        num += (__int128)coef * (__int128)s[i];
        tot += s[i];
    }
    free(s);
    __int128 den = (__int128)n * (__int128)tot;
    *gini = (tot == 0) ? 0.0 : (double)num / (double)den;
    *num_hi = (int64_t)(num >> 64);
    *num_lo = (uint64_t)num;
    *total = tot;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Epidemic curve moments from the per-step infected series I(1..T):        */
/* peak, first step reaching the peak, and the mean and variance of t under */
/* the weights I(t): mean = S1/S0, var = (S0 S2 - S1^2) / S0^2 with         */
/* S_j = sum_t t^j I(t) as exact integers (one double division each).       */
/* ------------------------------------------------------------------------ */
int orc_curve_moments(const int64_t *infected, uint32_t T, int64_t *peak, uint32_t *argmax,
                      double *mean, double *var)
{
    unsigned __int128 s0 = 0, s1 = 0, s2 = 0;
    int64_t pk = -1;
    uint32_t am = 0;
    for (uint32_t j = 0; j < T; ++j) {
        uint64_t t = (uint64_t)j + 1;
        uint64_t v = (uint64_t)infected[j];
        if ((int64_t)v > pk) { pk = (int64_t)v; am = (uint32_t)t; }
        s0 += v;
        s1 += (unsigned __int128)v * t;
        s2 += (unsigned __int128)v * t * t;
    }
    *peak = (T == 0) ? 0 : pk;
    *argmax = am;
    if (s0 == 0) { *mean = 0.0; *var = 0.0; return ORC_OK; }
    *mean = (double)s1 / (double)s0;
    unsigned __int128 a = s0 * s2, b = s1 * s1; /* a >= b by Cauchy-Schwarz */
    *var = (double)(a - b) / ((double)s0 * (double)s0);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* View primitives (paper Sec. 3.1 and 3.3, the view API): a column of a    */
/* population is int32 (dtype 0) or uint8 (dtype 1), indexed by agent id.   */
/*  - full-population view: every row gets  v = v OP s;                     */
/*  - filtered view: where(column CMP s) = the ids whose value satisfies    */
/*    the predicate on the column as it is at that moment, ascending;       */
/*  - scatter view: a list of ids in which ids may repeat; an update is     */
/*    applied once per occurrence, so additions accumulate (scatter_add).   */
/* OP: 0 set, 1 add, 2 sub, 3 mul, 4 min, 5 max.  Arithmetic wraps modulo   */
/* 2^32 (int32) or 2^8 (uint8); min / max compare signed int32 or unsigned  */
/* uint8 values; the scalar is reduced to the column's type first (two's    */
/* complement truncation).  CMP: 0 ==, 1 !=, 2 <, 3 <=, 4 >, 5 >=, comparing */
/* the value (sign-extended int32 or zero-extended uint8) with the 64-bit   */
/* scalar as integers.                                                      */
/* ------------------------------------------------------------------------ */
#define DT_I32 0
#define DT_U8 1

static int64_t col_get(int dtype, const void *col, uint32_t i)
{
    return dtype == DT_I32 ? (int64_t)((const int32_t *)col)[i] : (int64_t)((const uint8_t *)col)[i];
}

/* v OP s in the column's type */
static int64_t apply_op(int dtype, int64_t v, int op, int64_t s)
{
    if (dtype == DT_I32) {
        uint32_t a = (uint32_t)v, b = (uint32_t)s, r;
        int32_t sa = (int32_t)a, sb = (int32_t)b;
        switch (op) {
        case 0: r = b; break;
        case 1: r = a + b; break;
        case 2: r = a - b; break;
        case 3: r = a * b; break;
        case 4: r = (uint32_t)(sa < sb ? sa : sb); break;
        default: r = (uint32_t)(sa > sb ? sa : sb); break;
        }
        return (int64_t)(int32_t)r;
    } else {
        uint8_t a = (uint8_t)v, b = (uint8_t)s, r;
        switch (op) {
        case 0: r = b; break;
        case 1: r = (uint8_t)(a + b); break;
        case 2: r = (uint8_t)(a - b); break;
        case 3: r = (uint8_t)(a * b); break;
        case 4: r = a < b ? a : b; break;
        default: r = a > b ? a : b; break;
        }
        return (int64_t)r;
    }
}

static void col_set(int dtype, void *col, uint32_t i, int64_t v)
{
    if (dtype == DT_I32)
        ((int32_t *)col)[i] = (int32_t)v;
    else
        ((uint8_t *)col)[i] = (uint8_t)v;
}

static int valid_dtype_op(int dtype, int op) { return (dtype == DT_I32 || dtype == DT_U8) && op >= 0 && op <= 5; }

/* Full-population view: col[i] = col[i] OP s for every row. */
int orc_col_map(int dtype, void *col, uint32_t n, int op, int64_t s)
{
    if (!valid_dtype_op(dtype, op) || (!col && n)) return ORC_EINVAL;
    for (uint32_t i = 0; i < n; ++i) col_set(dtype, col, i, apply_op(dtype, col_get(dtype, col, i), op, s));
    return ORC_OK;
}

/* Full-population view with a column operand: dst[i] = dst[i] OP src[i]
 * (src's value taken as an integer, then reduced to dst's type). */
int orc_col_map_col(int dtype_dst, void *dst, int dtype_src, const void *src, uint32_t n, int op)
{
    if (!valid_dtype_op(dtype_dst, op) || (dtype_src != DT_I32 && dtype_src != DT_U8) || (n && (!dst || !src)))
        return ORC_EINVAL;
    for (uint32_t i = 0; i < n; ++i)
        col_set(dtype_dst, dst, i, apply_op(dtype_dst, col_get(dtype_dst, dst, i), op, col_get(dtype_src, src, i)));
    return ORC_OK;
}

static int compare(int64_t v, int cmp, int64_t s)
{
    switch (cmp) {
    case 0: return v == s;
    case 1: return v != s;
    case 2: return v < s;
    case 3: return v <= s;
    case 4: return v > s;
    default: return v >= s;
    }
}

/* Filtered view: the ids i (ascending) with col[i] CMP s. */
int orc_where(int dtype, const void *col, uint32_t n, int cmp, int64_t s, int32_t *ids, uint32_t *count)
{
    if ((dtype != DT_I32 && dtype != DT_U8) || cmp < 0 || cmp > 5 || (n && (!col || !ids)) || !count)
        return ORC_EINVAL;
    uint32_t k = 0;
    for (uint32_t i = 0; i < n; ++i)
        if (compare(col_get(dtype, col, i), cmp, s)) ids[k++] = (int32_t)i;
    *count = k;
    return ORC_OK;
}

/* Update through a view: for every listed id, in list order,
 * col[id] = col[id] OP s.  Ids must lie in [0, n). */
int orc_view_map(int dtype, void *col, uint32_t n, const int32_t *ids, uint32_t k, int op, int64_t s)
{
    if (!valid_dtype_op(dtype, op) || (k && (!col || !ids))) return ORC_EINVAL;
    for (uint32_t j = 0; j < k; ++j)
        if (ids[j] < 0 || (uint32_t)ids[j] >= n) return ORC_EINVAL;
    for (uint32_t j = 0; j < k; ++j) {
        uint32_t i = (uint32_t)ids[j];
        col_set(dtype, col, i, apply_op(dtype, col_get(dtype, col, i), op, s));
    }
    return ORC_OK;
}

/* Random ids, one per listed id (the paper's random recipient choice, in
 * the counter-based form): for listed agent i, u = the agent's draw for
 * `step`, r' = uniform_below(u[word], m) with m = range - 1 when
 * exclude_self (then r = r' + (r' >= i)) and m = range otherwise (r = r').
 * exclude_self needs range >= 2; range >= 1 otherwise. */
int orc_view_draw(const int32_t *ids, uint32_t k, uint32_t seed, uint32_t rep, uint32_t step, uint32_t word,
                  uint32_t range, int exclude_self, int32_t *out)
{
    if (word > 3 || (k && (!ids || !out)) || range < (exclude_self ? 2u : 1u) || range > 0x80000000u)
        return ORC_EINVAL;
    for (uint32_t j = 0; j < k; ++j) {
        uint32_t i = (uint32_t)ids[j], u[4];
        draw(seed, rep, i, step, u);
        uint32_t r = uniform_below(u[word], exclude_self ? range - 1u : range);
        if (exclude_self && r >= i) r += 1;
        out[j] = (int32_t)r;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Continuous-space models as the paper states them (Sec. 5.1.2): agents in */
/* the box [0, w] x [0, h] with float32 positions.                          */
/*  - random walk: independent uniform x and y displacements, clamped to    */
/*    the box: dx = s * sunit(u0), dy = s * sunit(u1);                       */
/*  - SIR: an infected agent infects susceptible agents within distance r;  */
/*    a susceptible agent with k infected contacts becomes infected iff      */
/*    u2 < t_inf[min(k, K)] (the thresholds of 1 - (1-p)^k, as for the grid  */
/*    SIR); an agent recovers after rec_steps steps as infected; with        */
/*    s > 0 every agent first moves as in the walk.                          */
/* Every float operation below is one IEEE-754 single-precision operation   */
/* rounded to nearest (-ffp-contract=off: no fused multiply-add):           */
/*  unit(u)  = (u >> 8) * 2^-24           in [0, 1), exact;                  */
/*  sunit(u) = ((u >> 8) - 2^23) * 2^-23  in [-1, 1), exact;                 */
/*  x0 = w * unit(u0), y0 = h * unit(u1) with the initial draw (step         */
/*  0xFFFFFFFF); x' = clamp(x + dx, 0, w);                                   */
/*  contact iff (xi - xj)^2 + (yi - yj)^2 <= r*r, evaluated as written.      */
/* ------------------------------------------------------------------------ */
static float unit24(uint32_t u) { return (float)(u >> 8) * 5.9604644775390625e-8f; }
static float sunit24(uint32_t u) { return (float)((int32_t)(u >> 8) - 8388608) * 1.1920928955078125e-7f; }
static float clampf(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }

void orc_cinit_positions(uint32_t n, float w, float h, uint32_t seed, uint32_t rep, float *x, float *y)
{
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u[4];
        draw(seed, rep, i, INIT_STEP, u);
        x[i] = w * unit24(u[0]);
        y[i] = h * unit24(u[1]);
    }
}

static void cmove(float w, float h, float s, const uint32_t u[4], float *x, float *y)
{
    float dx = s * sunit24(u[0]);
    float dy = s * sunit24(u[1]);
    *x = clampf(*x + dx, 0.0f, w);
    *y = clampf(*y + dy, 0.0f, h);
}

int orc_cwalk_step(uint32_t n, float w, float h, float s, uint32_t seed, uint32_t rep, uint32_t t, float *x, float *y)
{
    if (!(w >= 0.0f) || !(h >= 0.0f) || !(s >= 0.0f)) return ORC_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u[4];
        draw(seed, rep, i, t, u);
        cmove(w, h, s, u, &x[i], &y[i]);
    }
    return ORC_OK;
}

int orc_csir_step(uint32_t n, float w, float h, float s, float r, uint32_t seed, uint32_t rep, uint32_t t,
                  const uint32_t *t_inf, uint32_t K, uint32_t rec_steps, float *x, float *y, uint8_t *state,
                  int32_t *days, int64_t counts[4])
{
    if (!(w >= 0.0f) || !(h >= 0.0f) || !(s >= 0.0f) || !(r >= 0.0f) || rec_steps < 1) return ORC_EINVAL;
    uint32_t *u2 = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint8_t *snap = (uint8_t *)malloc((size_t)n + 1);
    if (!u2 || !snap) { free(u2); free(snap); return ORC_ENOMEM; }
    /* 1. draws; moves (all agents) when s > 0 */
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u[4];
        draw(seed, rep, i, t, u);
        if (s > 0.0f) cmove(w, h, s, u, &x[i], &y[i]);
        u2[i] = u[2];
        snap[i] = state[i];
    }
    /* 2. transitions against the start-of-step states, all pairs */
    const float r2 = r * r;
    int64_t newinf = 0;
    for (uint32_t j = 0; j < n; ++j) {
        if (snap[j] == ST_S) {
            uint32_t k = 0;
            for (uint32_t i = 0; i < n; ++i) {
                if (i == j || snap[i] != ST_I) continue;
                float dx = x[i] - x[j];
                float dy = y[i] - y[j];
                float d2 = dx * dx + dy * dy;
                if (d2 <= r2) k += 1;
            }
            if (k >= 1) {
                uint32_t kk = (k < K) ? k : K;
                if (u2[j] < t_inf[kk]) { state[j] = ST_I; days[j] = 0; newinf += 1; }
            }
        } else if (snap[j] == ST_I) {
            days[j] += 1;
            if ((uint32_t)days[j] >= rec_steps) state[j] = ST_R;
        }
    }
    counts[0] = counts[1] = counts[2] = 0;
    for (uint32_t i = 0; i < n; ++i) counts[state[i]] += 1;
    counts[3] = newinf;
    free(u2);
    free(snap);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Buffered per-agent writes (paper Sec. 3.2.1: per-agent record() calls go */
/* into a pending-writes buffer flushed by one id-keyed update per step):   */
/* applying k recorded writes (id, value) to a column in record order, so   */
/* for every row the last recorded value wins.                              */
/* ------------------------------------------------------------------------ */
int orc_log_flush(int dtype, void *col, uint32_t n, const int32_t *ids, const int64_t *values, uint32_t k)
{
    if ((dtype != DT_I32 && dtype != DT_U8) || (k && (!col || !ids || !values))) return ORC_EINVAL;
    for (uint32_t j = 0; j < k; ++j)
        if (ids[j] < 0 || (uint32_t)ids[j] >= n) return ORC_EINVAL;
    for (uint32_t j = 0; j < k; ++j) col_set(dtype, col, (uint32_t)ids[j], apply_op(dtype, 0, 0, values[j]));
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Grid environments (paper Sec. 4.1): d-dimensional lattices (d = 1..4)    */
/* with Moore or von Neumann neighbourhoods, on a torus or in a bounded box. */
/* One step: every agent moves to a neighbour chosen uniformly among its    */
/* neighbours: m = hi32(u0 * count), the m-th neighbour in this order:      */
/*  - Moore: offsets in {-1, 0, 1}^d without the zero offset, enumerated as */
/*    base-3 numbers with dimension 0 the fastest digit (digit - 1 = offset);*/
/*  - von Neumann: (dim 0, -1), (dim 0, +1), (dim 1, -1), (dim 1, +1), ...; */
/* on a torus every neighbour exists (coordinates wrap); in a bounded box    */
/* only neighbours inside the box count, in the same order (an agent with  */
/* none stays).  For d = 2, Moore, torus this is the random walk above.    */
/* ------------------------------------------------------------------------ */
int orc_grid_walk_step(uint32_t d, const uint32_t *sizes, int moore, int torus, uint32_t n, int32_t **coords,
                       uint32_t seed, uint32_t rep, uint32_t t)
{
    if (d < 1 || d > 4) return ORC_EINVAL;
    for (uint32_t a = 0; a < d; ++a)
        if (sizes[a] < 1 || sizes[a] > 0x7FFFFFFFu) return ORC_EINVAL;
    uint32_t full = 1;
    for (uint32_t a = 0; a < d; ++a) full *= 3u;
    for (uint32_t i = 0; i < n; ++i) {
        int32_t c[4] = {0, 0, 0, 0};
        for (uint32_t a = 0; a < d; ++a) {
            c[a] = coords[a][i];
            if (c[a] < 0 || (uint32_t)c[a] >= sizes[a]) return ORC_EINVAL;
        }
        /* list this agent's neighbours in order */
        int32_t off[81][4];
        uint32_t cnt = 0;
        if (moore) {
            for (uint32_t m = 0; m < full; ++m) {
                uint32_t r = m, zero = 1, inside = 1;
                int32_t o[4] = {0, 0, 0, 0};
                for (uint32_t a = 0; a < d; ++a) {
                    o[a] = (int32_t)(r % 3u) - 1;
                    r /= 3u;
                    if (o[a] != 0) zero = 0;
                    int64_t v = (int64_t)c[a] + o[a];
                    if (v < 0 || v >= (int64_t)sizes[a]) inside = 0;
                }
                if (zero || (!torus && !inside)) continue;
                for (uint32_t a = 0; a < 4; ++a) off[cnt][a] = o[a];
                ++cnt;
            }
        } else {
            for (uint32_t a = 0; a < d; ++a)
                for (int s = -1; s <= 1; s += 2) {
                    int64_t v = (int64_t)c[a] + s;
                    if (!torus && (v < 0 || v >= (int64_t)sizes[a])) continue;
                    for (uint32_t b = 0; b < 4; ++b) off[cnt][b] = 0;
                    off[cnt][a] = s;
                    ++cnt;
                }
        }
        if (cnt == 0) continue;
        uint32_t u[4];
        draw(seed, rep, i, t, u);
        uint32_t m = uniform_below(u[0], cnt);
        for (uint32_t a = 0; a < d; ++a) coords[a][i] = wrap_add(c[a], off[m][a], sizes[a]);
    }
    return ORC_OK;
}

/* Filtered view of a view: the listed ids (in list order, repeats kept) whose
 * value satisfies col CMP s -- where(A).where(B) is the conjunction A and B. */
int orc_view_where(int dtype, const void *col, uint32_t n, const int32_t *ids, uint32_t k, int cmp, int64_t s,
                   int32_t *out, uint32_t *count)
{
    if ((dtype != DT_I32 && dtype != DT_U8) || cmp < 0 || cmp > 5 || (k && (!col || !ids || !out)) || !count)
        return ORC_EINVAL;
    uint32_t m = 0;
    for (uint32_t j = 0; j < k; ++j) {
        if (ids[j] < 0 || (uint32_t)ids[j] >= n) return ORC_EINVAL;
        if (compare(col_get(dtype, col, (uint32_t)ids[j]), cmp, s)) out[m++] = ids[j];
    }
    *count = m;
    return ORC_OK;
}

/* scatter_add with one value per listed id: col[ids[j]] += values[j] (in the
 * column's wrapping arithmetic; repeated ids accumulate). */
int orc_view_add_values(int dtype, void *col, uint32_t n, const int32_t *ids, const int32_t *values, uint32_t k)
{
    if ((dtype != DT_I32 && dtype != DT_U8) || (k && (!col || !ids || !values))) return ORC_EINVAL;
    for (uint32_t j = 0; j < k; ++j)
        if (ids[j] < 0 || (uint32_t)ids[j] >= n) return ORC_EINVAL;
    for (uint32_t j = 0; j < k; ++j) {
        uint32_t i = (uint32_t)ids[j];
        col_set(dtype, col, i, apply_op(dtype, col_get(dtype, col, i), 1, values[j]));
    }
    return ORC_OK;
}
