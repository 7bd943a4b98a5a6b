/*
 * acs_oracle.h -- interface of the plain CPU oracle for the synchronous-step
 * Ant Colony System (Skinderowicz, "The GPU-based Parallel Ant Colony
 * System", JPDC 2016, Sec. 3, Sec. 3.1, Sec. 3.2).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library. The product
 * (the CUDA library under paper_1605_02669_gb300/) never includes, links or
 * calls it, and the two share no code: this header is not the product's
 * header and the parameter struct below is declared independently.
 *
 * Status codes: 0 ok, 1 invalid argument, 2 out of memory.
 */
#ifndef ACS_ORACLE_H
#define ACS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t  m;            /* ants */
    int32_t  cl;           /* candidate-list width, 1..32, clamped to n-1 */
    int32_t  beta;         /* integer heuristic exponent, 0..8 */
    float    q0;           /* exploitation threshold, [0,1] */
    float    rho;          /* global evaporation (the paper's alpha) */
    float    xi;           /* local evaporation (the paper's rho, Eq. 3) */
    int32_t  memory;       /* 0 = n x n matrix, 1 = selective pheromone memory */
    int32_t  spm_slots;    /* s, slots per record, 1..32 */
    int32_t  local_period; /* local update on every k-th step, >= 1 */
    int32_t  flags;        /* 0, or ACSREF_FLAG_SPM_SKIP_DEFAULT */
    uint64_t seed;         /* Philox key */
} acsref_params;

/* SPM variant: a local update (Eq. 3) of an edge absent from a record leaves
 * the default value tau0, so it is not inserted (no eviction); it still
 * counts as a miss. Alg. 3 as printed inserts it (the default, flag off). */
#define ACSREF_FLAG_SPM_SKIP_DEFAULT 2

typedef struct acsref_colony acsref_colony;

/* ---- building blocks, exposed so tests can pin each one ---- */
void    acsref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int32_t acsref_dist(const int32_t* xy, int32_t i, int32_t j);
float   acsref_heuristic(int32_t d, int32_t beta);
void    acsref_scan32(const float* v, float* P);
int32_t acsref_pick(const float* v, const int32_t* unvisited, float q, float q0, float r);
float   acsref_local_value(float tau, float tau0, float Pk);
float   acsref_global_value(float tau, float delta, float rho);
void    acsref_decay_table(float xi, int32_t kmax, float* P);
int     acsref_knn(const int32_t* xy, int32_t n, int32_t cl, int32_t* nn);
int64_t acsref_nn_tour_length(const int32_t* xy, int32_t n);
void    acsref_spm_update(int32_t* idx, float* val, int32_t* tail, int32_t s,
                          int32_t neighbour, float tau0, int32_t mode,
                          float coef, float target, int64_t* hits, int64_t* misses);

/* ---- whole colony ---- */
int     acsref_create(const int32_t* xy, int32_t n, const acsref_params* p,
                      int32_t instance, acsref_colony** out);
int     acsref_create_tables(const int32_t* xy, int32_t n, const int32_t* nn,
                             const float* w, int32_t cl, const acsref_params* p,
                             int32_t instance, acsref_colony** out);
int     acsref_run(acsref_colony* c, int32_t iters);
/* The local updates of ONE synchronous step (Alg. 1, Eq. 3 folded over the
 * ants that share an undirected edge; Alg. 3 on the SPM), applied to the
 * colony's pheromone memory exactly as a run applies them: from[a] -> to[a]
 * (m entries) is the edge ant a took. Exposed so tests can pin the order and
 * multiplicity rules on hand-made steps. Returns 0, or 1 for a node out of
 * range or a self-loop (nothing changed). */
int     acsref_local_step(acsref_colony* c, const int32_t* from, const int32_t* to);
int     acsref_get_tours(const acsref_colony* c, int32_t* tours, int64_t* lens);
int     acsref_best(const acsref_colony* c, int32_t* tour, int64_t* len);
/* Offer a tour from elsewhere (another colony: multi-colony exchange). It
 * replaces the best-so-far only if it is a permutation and strictly shorter
 * (Alg. 1's replacement rule); returns 0, or 1 for a bad tour. */
int     acsref_offer_best(acsref_colony* c, const int32_t* tour);
int     acsref_get_pheromone(const acsref_colony* c, float* tau_or_val,
                             int32_t* spm_idx, int32_t* spm_tail);
int     acsref_get_setup(const acsref_colony* c, int32_t* nn, float* w,
                         float* tau0, int64_t* L_nn, int32_t* cl_eff);
int64_t acsref_iteration(const acsref_colony* c);
void    acsref_stats(const acsref_colony* c, int64_t out[4]);
void    acsref_destroy(acsref_colony* c);

#ifdef __cplusplus
}
#endif
#endif
