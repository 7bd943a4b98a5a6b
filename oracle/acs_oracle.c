/*
 * acs_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * synchronous-step Ant Colony System of Skinderowicz, "The GPU-based
 * Parallel Ant Colony System" (JPDC 2016).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and
 * the cpu_baseline / reference legs of bench.py, never by the product. It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   Alg. 1 (Sec. 3)   : random first node per ant, n-1 construction steps with
 *                       local updates, the closing-edge local update, the
 *                       iteration best, the best-so-far, the global update.
 *   Alg. 2 / Eq. 1-2  : candidate set from the cl nearest neighbours, q < q0
 *                       greedy argmax of tau*eta^beta, else proportional
 *                       (roulette) choice, else greedy over all unvisited.
 *   Eq. 3             : local update tau <- (1-xi)*tau + xi*tau0.
 *   global update eq. : tau <- (1-rho)*tau + rho/L_gb on the best-so-far edges.
 *   Sec. 3.2, Alg. 3  : selective pheromone memory (per-node circular buffer
 *                       of s (node, trail) slots; absent edges read tau_min).
 *
 * Readings of the paper fixed here (where it is silent, garbled or ambiguous):
 *   - Synchronous steps (the ACS-GPU model of Sec. 3.1.2): every ant picks its
 *     step-s node from the pheromone state left by step s-1; then the local
 *     updates of step s are applied. An undirected edge taken by k ants in one
 *     step gets ONE update with (1-xi)^k, written tau0 + P[k]*(tau - tau0) with
 *     the FP32 table P[0]=1, P[k]=P[k-1]*(1-xi).
 *   - Exploit iff q < q0 (Eq. 1 writes <=, the text <; with q in [0,1) on a
 *     2^-24 grid, q0=1 always exploits and q0=0 always explores).
 *   - eta = 1/max(d,1); w = 1/(x^beta), x=(float)max(d,1), x^beta by repeated
 *     multiplication from the left.
 *   - Roulette (Eq. 2): inclusive Hillis-Steele scan over 32 positions
 *     (offsets 1,2,4,8,16), t = r*P[31]; pick the first unvisited position k
 *     with v_k > 0 and P_k > t; else the last unvisited k with v_k > 0; else
 *     the first unvisited k.
 *   - Ties: greedy over candidates -> lowest rank k; full scan -> lowest node j.
 *   - tau0 = (float)(1/((double)n*L_nn)), L_nn the nearest-neighbour tour from
 *     node 0 (ties -> lowest index).
 *   - The global update touches only the n edges of the best-so-far tour, every
 *     iteration, both matrix halves; on the SPM in tour order, record of t_i
 *     then record of t_{i+1}.
 *   - SPM: idx=-1 marks an empty slot; tail starts at s-1 so the first insert
 *     lands in slot 0; a miss inserts f(tau0) even when that equals tau0.
 *     Within a step, distinct edges are applied in the order of the lowest ant
 *     that took them, record of the ant's from-node first.
 *   - EUC_2D: d = nint(sqrt(dx^2+dy^2)), computed exactly with an integer
 *     square root here.
 *   - Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 *     (seed lo, seed hi), counter = (iteration, ant, step, instance); word 0
 *     -> q, word 1 -> r, word 2 -> first node (step 0); u = (x>>8)*2^-24,
 *     first node = (x2*n)>>32.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (no FMA contraction, IEEE single precision, no flush-to-zero).
 */
#include "acs_oracle.h"

#include <stdlib.h>
#include <string.h>

#define COORD_LIMIT (1 << 20)

struct acsref_colony {
    int32_t n, cl, m, beta, memory, s, period, instance, flags;
    float q0, rho, xi, tau0;
    uint64_t seed;
    int32_t* xy;        /* 2n */
    int32_t* nn;        /* n*cl */
    float* w;           /* n*cl */
    float* P;           /* m+1 */
    float* tau;         /* n*n (matrix) */
    int32_t* spm_idx;   /* n*s */
    float* spm_val;     /* n*s */
    int32_t* spm_tail;  /* n */
    int32_t* tours;     /* m*n */
    int64_t* lens;      /* m */
    int32_t* best;      /* n */
    int64_t best_len;
    int has_best;
    int64_t L_nn;
    int64_t iteration;
    uint8_t* visited;   /* m*n */
    int64_t fallback_steps, select_steps, spm_hits, spm_misses;
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the published definition (Salmon et al., SC'11,
 * "Parallel random numbers: as easy as 1, 2, 3", Sec. 4 and Table 2):
 * ten rounds of the Philox S-box on a 4-word counter, the 2-word key bumped
 * by the Weyl constants between rounds. */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void acsref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static float unit_float(uint32_t x)
{
    /* 24 random bits onto the 2^-24 grid of [0,1): exact in FP32 */
    return (float)(x >> 8) * (1.0f / 16777216.0f);
}

/* ------------------------------------------------------------------ */
/* EUC_2D distance: nint of the Euclidean distance (TSP on a complete graph,
 * cost d_ij, Sec. 3). Exact: floor square root by bisection in integers, then
 * round half up, which is never a tie for an integer radicand. */
static int64_t isqrt_floor(int64_t s)
{
    int64_t lo = 0, hi = 3037000499LL; /* floor(sqrt(2^63-1)) */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (mid <= s / mid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

int32_t acsref_dist(const int32_t* xy, int32_t i, int32_t j)
{
    int64_t dx = (int64_t)xy[2 * i] - (int64_t)xy[2 * j];
    int64_t dy = (int64_t)xy[2 * i + 1] - (int64_t)xy[2 * j + 1];
    int64_t s = dx * dx + dy * dy;
    int64_t r = isqrt_floor(s);
    /* sqrt(s) >= r + 1/2  <=>  s - r^2 > r  (both sides integers) */
    return (int32_t)(r + ((s - r * r) > r ? 1 : 0));
}

/* w = eta^beta with eta = 1/max(d,1) (Eq. 1), evaluated as 1/(x^beta). */
float acsref_heuristic(int32_t d, int32_t beta)
{
    float x = (float)(d > 1 ? d : 1);
    float p = 1.0f;
    for (int32_t i = 0; i < beta; i++) p = (i == 0) ? x : p * x;
    return 1.0f / p;
}

/* ------------------------------------------------------------------ */
/* Roulette of Eq. 2 on a warp-sized candidate set (Sec. 3.1.1): inclusive
 * Hillis-Steele scan over 32 positions. */
void acsref_scan32(const float* v, float* P)
{
    float x[32], y[32];
    for (int k = 0; k < 32; k++) x[k] = v[k];
    for (int off = 1; off < 32; off *= 2) {
        for (int k = 0; k < 32; k++) y[k] = (k >= off) ? x[k] + x[k - off] : x[k];
        for (int k = 0; k < 32; k++) x[k] = y[k];
    }
    for (int k = 0; k < 32; k++) P[k] = x[k];
}

/* Pseudo-random-proportional rule over a non-empty candidate set (Eq. 1-2,
 * Alg. 2): v[k] = tau*w for unvisited k, 0 otherwise. Returns the rank k. */
int32_t acsref_pick(const float* v, const int32_t* unv, float q, float q0, float r)
{
    if (q < q0) {
        int32_t bk = -1;
        for (int k = 0; k < 32; k++)
            if (unv[k] && (bk < 0 || v[k] > v[bk])) bk = k;
        return bk;
    }
    float P[32];
    float vv[32];
    for (int k = 0; k < 32; k++) vv[k] = unv[k] ? v[k] : 0.0f;
    acsref_scan32(vv, P);
    float t = r * P[31];
    for (int k = 0; k < 32; k++)
        if (unv[k] && vv[k] > 0.0f && P[k] > t) return k;
    for (int k = 31; k >= 0; k--)
        if (unv[k] && vv[k] > 0.0f) return k;
    for (int k = 0; k < 32; k++)
        if (unv[k]) return k;
    return -1;
}

/* Local update (Eq. 3) folded over k same-step visits: tau0 + P[k]*(tau-tau0). */
float acsref_local_value(float tau, float tau0, float Pk)
{
    float d = tau - tau0;
    float e = Pk * d;
    return tau0 + e;
}

/* Global update (eq. global_update): tau + rho*(Delta - tau). */
float acsref_global_value(float tau, float delta, float rho)
{
    float d = delta - tau;
    float e = rho * d;
    return tau + e;
}

void acsref_decay_table(float xi, int32_t kmax, float* P)
{
    float f = 1.0f - xi;
    P[0] = 1.0f;
    for (int32_t k = 1; k <= kmax; k++) P[k] = P[k - 1] * f;
}

/* ------------------------------------------------------------------ */
/* Candidate lists: the cl nearest neighbours of each node (Sec. 3, Alg. 2),
 * sorted by (distance, index). */
typedef struct { int32_t d, j; } dj_pair;

static int cmp_dj(const void* a, const void* b)
{
    const dj_pair* x = (const dj_pair*)a;
    const dj_pair* y = (const dj_pair*)b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    return (x->j > y->j) - (x->j < y->j);
}

int acsref_knn(const int32_t* xy, int32_t n, int32_t cl, int32_t* nn)
{
    dj_pair* buf = (dj_pair*)malloc(sizeof(dj_pair) * (size_t)n);
    if (!buf) return 2;
    for (int32_t c = 0; c < n; c++) {
        int32_t cnt = 0;
        for (int32_t j = 0; j < n; j++) {
            if (j == c) continue;
            buf[cnt].d = acsref_dist(xy, c, j);
            buf[cnt].j = j;
            cnt++;
        }
        qsort(buf, (size_t)cnt, sizeof(dj_pair), cmp_dj);
        for (int32_t k = 0; k < cl; k++) nn[(size_t)c * cl + k] = buf[k].j;
    }
    free(buf);
    return 0;
}

/* Nearest-neighbour tour from node 0, ties to the lowest index; its length
 * sets tau0 = 1/(n*L_nn). */
int64_t acsref_nn_tour_length(const int32_t* xy, int32_t n)
{
    uint8_t* vis = (uint8_t*)calloc((size_t)n, 1);
    if (!vis) return -1;
    int32_t cur = 0;
    int64_t L = 0;
    vis[0] = 1;
    for (int32_t step = 1; step < n; step++) {
        int32_t bj = -1, bd = 0;
        for (int32_t j = 0; j < n; j++) {
            if (vis[j]) continue;
            int32_t d = acsref_dist(xy, cur, j);
            if (bj < 0 || d < bd) { bj = j; bd = d; }
        }
        vis[bj] = 1;
        L += bd;
        cur = bj;
    }
    L += acsref_dist(xy, cur, 0);
    free(vis);
    return L;
}

/* ------------------------------------------------------------------ */
/* Selective pheromone memory update, Alg. 3. mode 0: local update with
 * coef = P[k]; mode 1: global update with coef = rho, target = Delta. */
static float apply_update(float t, float tau0, int32_t mode, float coef, float target)
{
    return mode == 0 ? acsref_local_value(t, tau0, coef)
                     : acsref_global_value(t, target, coef);
}

void acsref_spm_update(int32_t* idx, float* val, int32_t* tail, int32_t s,
                       int32_t nb, float tau0, int32_t mode, float coef,
                       float target, int64_t* hits, int64_t* misses)
{
    for (int32_t i = 0; i < s; i++) {
        if (idx[i] == nb) {
            val[i] = apply_update(val[i], tau0, mode, coef, target);
            if (hits) (*hits)++;
            return;
        }
    }
    if (misses) (*misses)++;
    *tail = (*tail + 1) % s;
    idx[*tail] = nb;
    val[*tail] = apply_update(tau0, tau0, mode, coef, target);
}

/* ------------------------------------------------------------------ */
static float tau_read(const acsref_colony* C, int32_t c, int32_t j)
{
    if (C->memory == 0) return C->tau[(size_t)c * C->n + j];
    const int32_t* idx = C->spm_idx + (size_t)c * C->s;
    const float* val = C->spm_val + (size_t)c * C->s;
    for (int32_t i = 0; i < C->s; i++)
        if (idx[i] == j) return val[i];
    return C->tau0;
}

static void edge_update(acsref_colony* C, int32_t u, int32_t v, int32_t mode,
                        float coef, float target)
{
    if (C->memory == 0) {
        float t = C->tau[(size_t)u * C->n + v];
        float t2 = apply_update(t, C->tau0, mode, coef, target);
        C->tau[(size_t)u * C->n + v] = t2;
        C->tau[(size_t)v * C->n + u] = t2;
    } else {
        int32_t s = C->s;
        for (int side = 0; side < 2; side++) {
            const int32_t r = side ? v : u, nb = side ? u : v;
            int32_t* idx = C->spm_idx + (size_t)r * s;
            if (mode == 0 && (C->flags & ACSREF_FLAG_SPM_SKIP_DEFAULT)) {
                /* variant: an absent edge keeps tau0 without an insert */
                int present = 0;
                for (int32_t i = 0; i < s; i++)
                    if (idx[i] == nb) present = 1;
                if (!present) {
                    C->spm_misses++;
                    continue;
                }
            }
            acsref_spm_update(idx, C->spm_val + (size_t)r * s, C->spm_tail + r, s, nb,
                              C->tau0, mode, coef, target, &C->spm_hits, &C->spm_misses);
        }
    }
}

static int validate(const int32_t* xy, int32_t n, const acsref_params* p)
{
    if (!xy || !p || n < 3) return 1;
    if (p->m < 1 || p->m > 4096) return 1;
    if (p->cl < 1 || p->cl > 32) return 1;
    if (p->beta < 0 || p->beta > 8) return 1;
    if (!(p->q0 >= 0.0f && p->q0 <= 1.0f)) return 1;
    if (!(p->rho > 0.0f && p->rho < 1.0f)) return 1;
    if (!(p->xi > 0.0f && p->xi < 1.0f)) return 1;
    if (p->memory != 0 && p->memory != 1) return 1;
    if (p->memory == 1 && (p->spm_slots < 1 || p->spm_slots > 32)) return 1;
    if (p->local_period < 1 || (p->flags & ~ACSREF_FLAG_SPM_SKIP_DEFAULT) != 0) return 1;
    for (int32_t i = 0; i < 2 * n; i++)
        if (xy[i] < 0 || xy[i] >= COORD_LIMIT) return 1;
    return 0;
}

static int colony_alloc(const int32_t* xy, int32_t n, int32_t cl,
                        const acsref_params* p, int32_t instance,
                        acsref_colony** out)
{
    acsref_colony* C = (acsref_colony*)calloc(1, sizeof(acsref_colony));
    if (!C) return 2;
    C->n = n; C->cl = cl; C->m = p->m; C->beta = p->beta;
    C->memory = p->memory; C->s = p->memory == 1 ? p->spm_slots : 0;
    C->period = p->local_period; C->instance = instance; C->flags = p->flags;
    C->q0 = p->q0; C->rho = p->rho; C->xi = p->xi; C->seed = p->seed;
    size_t nn_sz = (size_t)n * cl;
    C->xy = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)n);
    C->nn = (int32_t*)malloc(sizeof(int32_t) * nn_sz);
    C->w = (float*)malloc(sizeof(float) * nn_sz);
    C->P = (float*)malloc(sizeof(float) * ((size_t)p->m + 1));
    C->tours = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->m * n);
    C->lens = (int64_t*)calloc((size_t)p->m, sizeof(int64_t));
    C->best = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    C->visited = (uint8_t*)malloc((size_t)p->m * n);
    if (C->memory == 0) {
        C->tau = (float*)malloc(sizeof(float) * (size_t)n * n);
    } else {
        C->spm_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * C->s);
        C->spm_val = (float*)malloc(sizeof(float) * (size_t)n * C->s);
        C->spm_tail = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    }
    if (!C->xy || !C->nn || !C->w || !C->P || !C->tours || !C->lens || !C->best ||
        !C->visited || (C->memory == 0 && !C->tau) ||
        (C->memory == 1 && (!C->spm_idx || !C->spm_val || !C->spm_tail))) {
        acsref_destroy(C);
        return 2;
    }
    memcpy(C->xy, xy, sizeof(int32_t) * 2 * (size_t)n);
    acsref_decay_table(p->xi, p->m, C->P);
    C->L_nn = acsref_nn_tour_length(xy, n);
    if (C->L_nn < 0) { acsref_destroy(C); return 2; }
    C->tau0 = (float)(1.0 / ((double)n * (double)C->L_nn));
    if (C->memory == 0) {
        for (size_t i = 0; i < (size_t)n * n; i++) C->tau[i] = C->tau0;
    } else {
        for (size_t i = 0; i < (size_t)n * C->s; i++) {
            C->spm_idx[i] = -1;
            C->spm_val[i] = 0.0f;
        }
        for (int32_t i = 0; i < n; i++) C->spm_tail[i] = C->s - 1;
    }
    *out = C;
    return 0;
}

int acsref_create(const int32_t* xy, int32_t n, const acsref_params* p,
                  int32_t instance, acsref_colony** out)
{
    if (!out) return 1;
    int rc = validate(xy, n, p);
    if (rc) return rc;
    int32_t cl = p->cl < n - 1 ? p->cl : n - 1;
    acsref_colony* C = NULL;
    rc = colony_alloc(xy, n, cl, p, instance, &C);
    if (rc) return rc;
    rc = acsref_knn(xy, n, cl, C->nn);
    if (rc) { acsref_destroy(C); return rc; }
    for (int32_t c = 0; c < n; c++)
        for (int32_t k = 0; k < cl; k++) {
            size_t e = (size_t)c * cl + k;
            C->w[e] = acsref_heuristic(acsref_dist(xy, c, C->nn[e]), p->beta);
        }
    *out = C;
    return 0;
}

int acsref_create_tables(const int32_t* xy, int32_t n, const int32_t* nn,
                         const float* w, int32_t cl, const acsref_params* p,
                         int32_t instance, acsref_colony** out)
{
    if (!out || !nn || !w) return 1;
    int rc = validate(xy, n, p);
    if (rc) return rc;
    if (cl < 1 || cl > 32 || cl > n - 1) return 1;
    for (size_t e = 0; e < (size_t)n * cl; e++) {
        int32_t c = (int32_t)(e / (size_t)cl);
        if (nn[e] < 0 || nn[e] >= n || nn[e] == c || !(w[e] >= 0.0f)) return 1;
    }
    acsref_colony* C = NULL;
    rc = colony_alloc(xy, n, cl, p, instance, &C);
    if (rc) return rc;
    memcpy(C->nn, nn, sizeof(int32_t) * (size_t)n * cl);
    memcpy(C->w, w, sizeof(float) * (size_t)n * cl);
    *out = C;
    return 0;
}

/* Next node of ant a at step s from node c (Alg. 2). */
static int32_t select_next(acsref_colony* C, int32_t a, int32_t s, int32_t c,
                           const uint32_t key[2])
{
    const int32_t n = C->n, cl = C->cl;
    const uint8_t* vis = C->visited + (size_t)a * n;
    float v[32];
    int32_t unv[32];
    int any = 0;
    for (int k = 0; k < 32; k++) { v[k] = 0.0f; unv[k] = 0; }
    for (int32_t k = 0; k < cl; k++) {
        int32_t j = C->nn[(size_t)c * cl + k];
        if (!vis[j]) {
            unv[k] = 1;
            any = 1;
            v[k] = tau_read(C, c, j) * C->w[(size_t)c * cl + k];
        }
    }
    C->select_steps++;
    if (any) {
        uint32_t ctr[4] = {(uint32_t)C->iteration, (uint32_t)a, (uint32_t)s,
                           (uint32_t)C->instance};
        uint32_t x[4];
        acsref_philox4x32_10(ctr, key, x);
        float q = unit_float(x[0]);
        float r = unit_float(x[1]);
        int32_t k = acsref_pick(v, unv, q, C->q0, r);
        return C->nn[(size_t)c * cl + k];
    }
    /* candidate set exhausted: greedy over every unvisited node */
    C->fallback_steps++;
    float best = -1.0f;
    int32_t bj = -1;
    for (int32_t j = 0; j < n; j++) {
        if (vis[j]) continue;
        float p = tau_read(C, c, j) * acsref_heuristic(acsref_dist(C->xy, c, j), C->beta);
        if (p > best) { best = p; bj = j; }
    }
    return bj;
}

/* Local updates of one synchronous step: edges (from[a], to[a]) of all ants. */
static void local_update_step(acsref_colony* C, const int32_t* from, const int32_t* to)
{
    const int32_t m = C->m;
    for (int32_t a = 0; a < m; a++) {
        int32_t u = from[a], v = to[a];
        int dup = 0;
        for (int32_t b = 0; b < a && !dup; b++)
            if ((from[b] == u && to[b] == v) || (from[b] == v && to[b] == u)) dup = 1;
        if (dup) continue;
        int32_t k = 0;
        for (int32_t b = a; b < m; b++)
            if ((from[b] == u && to[b] == v) || (from[b] == v && to[b] == u)) k++;
        edge_update(C, u, v, 0, C->P[k], 0.0f);
    }
}

int acsref_local_step(acsref_colony* C, const int32_t* from, const int32_t* to)
{
    if (!C || !from || !to) return 1;
    for (int32_t a = 0; a < C->m; a++)
        if (from[a] < 0 || from[a] >= C->n || to[a] < 0 || to[a] >= C->n || from[a] == to[a])
            return 1;
    local_update_step(C, from, to);
    return 0;
}

static void one_iteration(acsref_colony* C)
{
    const int32_t n = C->n, m = C->m;
    const uint32_t key[2] = {(uint32_t)C->seed, (uint32_t)(C->seed >> 32)};
    int32_t* from = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    int32_t* to = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    memset(C->visited, 0, (size_t)m * n);
    for (int32_t a = 0; a < m; a++) {
        uint32_t ctr[4] = {(uint32_t)C->iteration, (uint32_t)a, 0u, (uint32_t)C->instance};
        uint32_t x[4];
        acsref_philox4x32_10(ctr, key, x);
        int32_t start = (int32_t)(((uint64_t)x[2] * (uint64_t)n) >> 32);
        C->tours[(size_t)a * n] = start;
        C->visited[(size_t)a * n + start] = 1;
    }
    for (int32_t s = 1; s < n; s++) {
        for (int32_t a = 0; a < m; a++)
            to[a] = select_next(C, a, s, C->tours[(size_t)a * n + s - 1], key);
        for (int32_t a = 0; a < m; a++) {
            from[a] = C->tours[(size_t)a * n + s - 1];
            C->tours[(size_t)a * n + s] = to[a];
            C->visited[(size_t)a * n + to[a]] = 1;
        }
        if (s % C->period == 0) local_update_step(C, from, to);
    }
    /* closing edges count as step n */
    for (int32_t a = 0; a < m; a++) {
        from[a] = C->tours[(size_t)a * n + n - 1];
        to[a] = C->tours[(size_t)a * n];
    }
    if (n % C->period == 0) local_update_step(C, from, to);
    free(from);
    free(to);

    int32_t ib = 0;
    for (int32_t a = 0; a < m; a++) {
        const int32_t* t = C->tours + (size_t)a * n;
        int64_t L = 0;
        for (int32_t i = 0; i < n; i++) L += acsref_dist(C->xy, t[i], t[(i + 1) % n]);
        C->lens[a] = L;
        if (L < C->lens[ib]) ib = a;
    }
    if (!C->has_best || C->lens[ib] < C->best_len) {
        C->has_best = 1;
        C->best_len = C->lens[ib];
        memcpy(C->best, C->tours + (size_t)ib * n, sizeof(int32_t) * (size_t)n);
    }
    float delta = (float)(1.0 / (double)C->best_len);
    for (int32_t i = 0; i < n; i++)
        edge_update(C, C->best[i], C->best[(i + 1) % n], 1, C->rho, delta);
    C->iteration++;
}

int acsref_run(acsref_colony* C, int32_t iters)
{
    if (!C || iters < 0) return 1;
    for (int32_t i = 0; i < iters; i++) one_iteration(C);
    return 0;
}

int acsref_get_tours(const acsref_colony* C, int32_t* tours, int64_t* lens)
{
    if (!C) return 1;
    if (tours) memcpy(tours, C->tours, sizeof(int32_t) * (size_t)C->m * C->n);
    if (lens) memcpy(lens, C->lens, sizeof(int64_t) * (size_t)C->m);
    return 0;
}

int acsref_best(const acsref_colony* C, int32_t* tour, int64_t* len)
{
    if (!C || !C->has_best) return 1;
    if (tour) memcpy(tour, C->best, sizeof(int32_t) * (size_t)C->n);
    if (len) *len = C->best_len;
    return 0;
}

int acsref_offer_best(acsref_colony* C, const int32_t* tour)
{
    if (!C || !tour) return 1;
    const int32_t n = C->n;
    uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
    if (!seen) return 1;
    int ok = 1;
    for (int32_t i = 0; i < n && ok; i++) {
        if (tour[i] < 0 || tour[i] >= n || seen[tour[i]]) ok = 0;
        else seen[tour[i]] = 1;
    }
    free(seen);
    if (!ok) return 1;
    int64_t L = 0;
    for (int32_t i = 0; i < n; i++) L += acsref_dist(C->xy, tour[i], tour[(i + 1) % n]);
    if (!C->has_best || L < C->best_len) {
        memcpy(C->best, tour, sizeof(int32_t) * (size_t)n);
        C->best_len = L;
        C->has_best = 1;
    }
    return 0;
}

int acsref_get_pheromone(const acsref_colony* C, float* tau_or_val,
                         int32_t* spm_idx, int32_t* spm_tail)
{
    if (!C) return 1;
    if (C->memory == 0) {
        if (tau_or_val) memcpy(tau_or_val, C->tau, sizeof(float) * (size_t)C->n * C->n);
        return 0;
    }
    size_t ns = (size_t)C->n * C->s;
    if (tau_or_val) memcpy(tau_or_val, C->spm_val, sizeof(float) * ns);
    if (spm_idx) memcpy(spm_idx, C->spm_idx, sizeof(int32_t) * ns);
    if (spm_tail) memcpy(spm_tail, C->spm_tail, sizeof(int32_t) * (size_t)C->n);
    return 0;
}

int acsref_get_setup(const acsref_colony* C, int32_t* nn, float* w, float* tau0,
                     int64_t* L_nn, int32_t* cl_eff)
{
    if (!C) return 1;
    if (nn) memcpy(nn, C->nn, sizeof(int32_t) * (size_t)C->n * C->cl);
    if (w) memcpy(w, C->w, sizeof(float) * (size_t)C->n * C->cl);
    if (tau0) *tau0 = C->tau0;
    if (L_nn) *L_nn = C->L_nn;
    if (cl_eff) *cl_eff = C->cl;
    return 0;
}

int64_t acsref_iteration(const acsref_colony* C) { return C ? C->iteration : -1; }

void acsref_stats(const acsref_colony* C, int64_t out[4])
{
    out[0] = C->fallback_steps;
    out[1] = C->select_steps;
    out[2] = C->spm_hits;
    out[3] = C->spm_misses;
}

void acsref_destroy(acsref_colony* C)
{
    if (!C) return;
    free(C->xy); free(C->nn); free(C->w); free(C->P); free(C->tau);
    free(C->spm_idx); free(C->spm_val); free(C->spm_tail);
    free(C->tours); free(C->lens); free(C->best); free(C->visited);
    free(C);
}
