/*
 * acs.h -- C ABI of libacs, a GB300 (sm_103a) implementation of the
 * synchronous-step Ant Colony System for the symmetric TSP, after
 * Skinderowicz, "The GPU-based Parallel Ant Colony System" (JPDC 2016).
 *
 * Problem (Sec. 3): a complete graph on n nodes with integer coordinates;
 * the cost d_ij is the EUC_2D distance nint(sqrt(dx^2+dy^2)); the output is a
 * short Hamiltonian cycle. One "colony" (instance) is solved by m ants per
 * iteration (Alg. 1): each ant starts at a random node and extends its tour
 * step by step with the pseudo-random-proportional rule (Eq. 1-2, Alg. 2)
 * over a candidate list of the cl nearest neighbours, falling back to the
 * best unvisited node when the list is exhausted; every step's edges get the
 * local pheromone update (Eq. 3); after the tours are closed and evaluated
 * the best-so-far tour gets the global update (eq. global_update). The
 * pheromone memory is either the n x n FP32 matrix or the selective
 * pheromone memory (Sec. 3.2, Alg. 3).
 *
 * Determinism contract (all modes but ACS_FLAG_RELAXED, which trades it for
 * speed): for a given (coordinates, parameters, seed, instance index) every
 * call sequence yields bit-identical tours, tour lengths and pheromone state,
 * equal to the CPU oracle shipped with the tests, whatever the launch shape
 * (threads per ant, cluster size, SPM record placement).
 * All ants of a step read the pheromone state left by the previous step; an
 * undirected edge taken by k ants in one step gets one local update with
 * factor (1-xi)^k (tau <- tau0 + P[k]*(tau - tau0), P[k] an FP32 table built
 * by repeated multiplication). Randomness is Philox4x32-10 keyed by the seed,
 * counter (iteration, ant, step, instance).
 *
 * Conventions for every entry point:
 *   - Pointers named coords, tour_out, ... are HOST pointers unless the name
 *     says dev_. Inputs are copied; the caller keeps ownership.
 *   - Output buffers are caller-allocated host memory. Calls that return data
 *     synchronise the context's stream first.
 *   - The context owns all device memory it allocates; acs_destroy frees it.
 *   - Every call returns an acs_status and never aborts. On ACS_EINVAL /
 *     ACS_ENOMEM the context is unchanged. After ACS_ECUDA or ACS_ETIMEOUT
 *     the context is poisoned: later calls on it return ACS_ESTATE.
 *   - Limits: 3 <= n <= 65536 per instance; 1 <= B <= 65535 instances per
 *     context; coordinates in [0, 2^20); 1 <= m <= 1024; 1 <= cl <= 32
 *     (clamped to n-1); 0 <= beta <= 8; 1 <= spm_slots <= 32.
 *   - A context is not thread-safe; use one host thread per context.
 */
#ifndef ACS_H
#define ACS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ACS_OK = 0,
    ACS_EINVAL = 1,   /* bad argument; nothing changed */
    ACS_ENOMEM = 2,   /* device or host allocation failed; nothing changed */
    ACS_ECUDA = 3,    /* a CUDA call or a kernel failed; context poisoned */
    ACS_ETIMEOUT = 4, /* a bounded device wait gave up; context poisoned */
    ACS_ESTATE = 5    /* context poisoned earlier, or no result yet */
} acs_status;

typedef enum { ACS_MEM_MATRIX = 0, ACS_MEM_SPM = 1 } acs_memory;

/* Parameters shared by all instances of a context. Names follow the ACS
 * literature; note the paper writes the local evaporation as rho (Eq. 3) and
 * the global one as alpha (eq. global_update). */
typedef struct {
    int32_t  m;            /* ants per instance, 1..1024 */
    int32_t  cl;           /* candidate-list width, 1..32, clamped to n-1 */
    int32_t  beta;         /* integer exponent of eta = 1/max(d,1), 0..8 */
    float    q0;           /* exploit iff q < q0, q uniform on [0,1); [0,1] */
    float    rho;          /* global evaporation, (0,1) (paper's alpha) */
    float    xi;           /* local evaporation, (0,1) (paper's rho, Eq. 3) */
    int32_t  memory;       /* acs_memory */
    int32_t  spm_slots;    /* s, trails per node in the SPM, 1..32 */
    int32_t  local_period; /* local update only at steps s with s % k == 0
                              (Sec. 4, "Limiting the number of local
                              pheromone updates"); 1 = every step */
    int32_t  flags;        /* 0, or ACS_FLAG_RELAXED */
    uint64_t seed;         /* Philox key */
} acs_params;

/* ACS_FLAG_RELAXED: the relaxed construction of ACS-GPU-Alt (Sec. 3.1.2):
 * every ant builds its whole tour in one pass with no step barrier and
 * applies the local update to each edge at once with plain loads and stores,
 * so concurrent updates may be lost and results depend on timing (tours stay
 * valid; not bit-reproducible, no oracle parity). The evaluation and the
 * global update follow in a second kernel. Pheromone matrix only (an SPM
 * context with this flag is ACS_EINVAL). The autotuner has nothing to choose
 * for it. */
#define ACS_FLAG_RELAXED 1

/* ACS_FLAG_SPM_SKIP_DEFAULT: SPM variant of Alg. 3's insert rule. A local
 * update (Eq. 3) of an edge absent from a record yields exactly tau0; with
 * this flag it is not inserted (no eviction), and it still counts as a miss.
 * Off by default (the paper inserts it). No effect on the matrix. */
#define ACS_FLAG_SPM_SKIP_DEFAULT 2

typedef struct acs_ctx acs_ctx;

/* One instance. coords: host int32 [n][2] (x, y). Instance index 0.
 * Builds the candidate lists (cl nearest neighbours sorted by distance, then
 * index), the heuristic table w = 1/max(d,1)^beta, the nearest-neighbour tour
 * from node 0 and tau0 = 1/(n*L_nn), and initialises the pheromone memory. */
acs_status acs_create(const int32_t* coords, int32_t n, const acs_params* p,
                      acs_ctx** out);

/* B independent instances solved together (one persistent launch per
 * iteration). coords: host int32 [sum n_b][2]; offsets: host int64 [B+1],
 * offsets[0]=0, instance b owns nodes offsets[b]..offsets[b+1]-1. Instance b
 * uses Philox counter word 3 = b. */
acs_status acs_create_batch(const int32_t* coords, const int64_t* offsets,
                            int32_t B, const acs_params* p, acs_ctx** out);

/* acs_create_batch with the Philox counter word 3 of each instance given by
 * the caller: instance_ids host int32 [B], each >= 0 (NULL = 0..B-1). An
 * instance's random stream, and so its tours and pheromone state, depend only
 * on its coordinates, the parameters, the seed and its id, not on which
 * batch, context or GPU runs it: a batch split across GPUs by instance (with
 * global ids) gives every instance the result it has in the whole batch.
 * ACS_EINVAL for a negative id; otherwise as acs_create_batch. */
acs_status acs_create_batch_ids(const int32_t* coords, const int64_t* offsets,
                                const int32_t* instance_ids, int32_t B,
                                const acs_params* p, acs_ctx** out);

/* Run later work on this CUDA stream (a cudaStream_t; NULL = legacy default).
 * The CUDA graph captured for one iteration is rebuilt on the next run. */
acs_status acs_set_stream(acs_ctx* ctx, void* cuda_stream);

/* Run `iters` full iterations of Alg. 1 on every instance (stream-ordered,
 * asynchronous; replays a captured CUDA graph of one iteration). */
acs_status acs_run_iterations(acs_ctx* ctx, int32_t iters);

/* Lanes per ant in the construct kernel: 4, 8, 16 or 32. Only
 * speed depends on it: results are bit-identical for every value. ACS_EINVAL
 * if the value cannot launch. */
acs_status acs_set_threads_per_ant(acs_ctx* ctx, int32_t tpa);
int32_t acs_threads_per_ant(const acs_ctx* ctx);

/* CTAs per thread-block cluster that share one instance: 1, 2, 4, 8 or 16.
 * Each CTA owns ceil(m/csize) ants; the CTAs exchange each step's edges
 * through distributed shared memory. The default is the largest size that
 * leaves at least 16 ants per CTA and keeps every instance resident (with a
 * full warp per ant when the size is above 1). Only speed depends on it:
 * results are bit-identical for every value. */
acs_status acs_set_cluster_size(acs_ctx* ctx, int32_t csize);
int32_t acs_cluster_size(const acs_ctx* ctx);

/* SPM contexts (Sec. 3.2): 1 keeps record r in the shared memory of CTA
 * r mod csize for each launch when the records fit (the default), 0 keeps
 * the records in global memory (smaller CTAs, more of them per SM). Only
 * speed depends on it: results are bit-identical. ACS_EINVAL if the value
 * cannot launch (the previous setting is kept). No effect on the matrix. */
acs_status acs_set_spm_resident(acs_ctx* ctx, int32_t resident);

/* Variant of the construct kernel the context launches (no counterpart in the
 * paper; for profiling): 0 = pheromone matrix, 1 = SPM records in global
 * memory, 2 = SPM records resident in the shared memory of the cluster for
 * the launch. -1 for NULL. */
int32_t acs_kernel_mode(const acs_ctx* ctx);

/* Autotuner: for every (threads per ant, cluster size) pair that can launch
 * (and, on the SPM, both record placements of acs_set_spm_resident),
 * times `trial_iters` iterations after one warm-up iteration, restoring the
 * full colony state after every trial, and keeps the fastest pair (written to
 * *chosen_tpa / *chosen_csize when not NULL). Results and the iteration count
 * of the context are unchanged. Synchronous; uses temporary device memory
 * for the snapshot. */
acs_status acs_autotune(acs_ctx* ctx, int32_t trial_iters, int32_t* chosen_tpa,
                        int32_t* chosen_csize);

/* Joint autotuner (no counterpart in the paper) for k contexts that run
 * concurrently, each on its own stream (acs_set_stream), for instance one
 * per pheromone memory. A shape that is fastest alone can be slower beside
 * the others, which compete for the same SMs. Each context is first tuned
 * alone (acs_autotune). Then, by coordinate descent over the contexts (two
 * passes at most), every launch shape of one context that ran within twice
 * its best time alone is timed with all k running together, the others'
 * shapes fixed; a switch needs a 1 % shorter group time. The descent runs
 * from two starts, the shapes best alone and each context's smallest shape
 * (fewest lanes x CTAs per instance), and the better end point is kept. The shape kept is the one that
 * gives the shortest group time: from a common start to the end of the
 * slowest context's `trial_iters` iterations, after one warm-up iteration
 * each. Every context's state is restored after every trial, so results and
 * iteration counts are unchanged. ctxs: host array of k distinct contexts.
 * ACS_EINVAL for a NULL or repeated context, k < 1 or trial_iters < 1;
 * ACS_ESTATE if one is poisoned; ACS_ENOMEM if a snapshot cannot be
 * allocated. Synchronous. */
acs_status acs_autotune_group(acs_ctx* const* ctxs, int32_t k, int32_t trial_iters);

/* Multi-colony exchange (the paper's related work, Sec. 2; no counterpart in
 * its algorithms): offer `tour` (host int32 [n], a permutation of the
 * instance's nodes) as the best-so-far of `instance`. Its length is computed
 * on the device; it replaces the best-so-far only if strictly shorter, the
 * replacement rule of Alg. 1, so the next global update deposits on it.
 * len_out (optional) receives the offered tour's length. ACS_EINVAL if the
 * tour is not a permutation. Works before the first iteration too. */
acs_status acs_offer_best_tour(acs_ctx* ctx, int32_t instance, const int32_t* tour,
                               int64_t* len_out);

/* Best-so-far tour (n node indices, 0-based, starting at the ant's first
 * node, closing implicitly) and its length. ACS_ESTATE before the first
 * iteration (unless acs_set_state restored a best-so-far tour). */
acs_status acs_best_tour(acs_ctx* ctx, int32_t instance, int32_t* tour_out,
                         int64_t* len_out);

/* Tours [m][n] and lengths [m] of the last iteration (either may be NULL). */
acs_status acs_get_tours(acs_ctx* ctx, int32_t instance, int32_t* tours,
                         int64_t* lens);

/* Pheromone state. Matrix: tau_or_val = float [n][n]; spm_idx/spm_tail
 * ignored. SPM: tau_or_val = float [n][s] trail values, spm_idx = int32
 * [n][s] neighbour per slot (-1 = empty), spm_tail = int32 [n] most recently
 * written slot. NULL outputs are skipped. */
acs_status acs_get_pheromone(acs_ctx* ctx, int32_t instance, float* tau_or_val,
                             int32_t* spm_idx, int32_t* spm_tail);

/* Set-up tables: nn int32 [n][cl_eff], w float [n][cl_eff], tau0, L_nn and
 * the effective candidate width (any output may be NULL). */
acs_status acs_get_setup(acs_ctx* ctx, int32_t instance, int32_t* nn, float* w,
                         float* tau0, int64_t* L_nn, int32_t* cl_eff);

/* Counters accumulated over all iterations of one instance:
 * out[0] full-scan fallback selections, out[1] all selections,
 * out[2] SPM hits, out[3] SPM misses (Sec. 3.2, Fig. spm-hit-ratio). */
acs_status acs_get_stats(acs_ctx* ctx, int32_t instance, int64_t out[4]);

/* Checkpoint and resume of one instance: the loop state that Alg. 1 carries
 * from one iteration to the next -- the pheromone memory (matrix, or the SPM
 * records of Sec. 3.2 / Alg. 3), the best-so-far tour and its length L_gb,
 * the iteration counter (Philox counter word 0 of the next iteration), the
 * candidate rows in use (a learned prior may have rewritten them) and the
 * counters of acs_get_stats. The tours of the last iteration are not part of
 * it. The buffer is caller-allocated HOST memory of acs_state_size bytes, an
 * opaque little-endian image (a 128-byte header, then the rows, the best
 * tour and the pheromone arrays).
 *   acs_state_size: bytes of instance's state (no device work).
 *   acs_get_state:  synchronises the context's stream, writes the image.
 *   acs_set_state:  replaces the instance's state with the image, after
 *                   checking on the host that it was written for the same
 *                   instance (n and tau0, i.e. the same coordinates) and the
 *                   same parameters except the seed, and that every index is
 *                   in range and the best tour is a permutation; ACS_EINVAL
 *                   (nothing changed) otherwise, or when bytes is too small.
 * With the same seed, running k iterations, saving, restoring into a fresh
 * context of the same instance and running the rest is bit-identical to the
 * unsplit run. acs_iteration reports instance 0's counter, so restoring
 * instance 0 sets it. */
acs_status acs_state_size(const acs_ctx* ctx, int32_t instance, int64_t* bytes);
acs_status acs_get_state(acs_ctx* ctx, int32_t instance, void* buf, int64_t bytes);
acs_status acs_set_state(acs_ctx* ctx, int32_t instance, const void* buf, int64_t bytes);

/* Iterations completed by instance 0 (every instance of a context runs the
 * same number of iterations; acs_set_state may restore another counter). */
int64_t acs_iteration(const acs_ctx* ctx);
int32_t acs_num_instances(const acs_ctx* ctx);
int32_t acs_instance_size(const acs_ctx* ctx, int32_t instance);

/* Kernel launches made by the last acs_run_iterations call (for accounting). */
int64_t acs_last_launch_count(const acs_ctx* ctx);

/* No-allocation variant of one iteration (the paper has no counterpart; it
 * exists for callers that cannot allocate device memory, such as code running
 * inside a memory arena or pool it does not own, or a hot path where
 * cudaMalloc is not allowed). It runs the same iteration as
 * acs_run_iterations(ctx, 1) on an acs_create context -- the same construct
 * kernel and the same results -- on one instance whose state lives entirely
 * in caller-owned DEVICE buffers, FP32 matrix memory only, Philox instance
 * index 0:
 *   dev_coords   int32 [n][2] node coordinates (input)
 *   dev_nn32     int32 [n][32] candidate lists padded with -1 (input)
 *   dev_w32      float [n][32] heuristic weights padded with 0 (input)
 *   cl           candidate width used by the rows (1..32, <= n-1)
 *   tau0         initial trail 1/(n*L_nn)
 *   dev_tau      float [n][n] pheromone matrix (in/out; start filled with tau0)
 *   dev_tours    int32 [m][n] tours of this iteration (output)
 *   dev_lens     int64 [m] their lengths (output)
 *   dev_best     int32 [n] best-so-far tour (in/out)
 *   dev_best_len int64 [1] its length (in/out; INT64_MAX before the first call)
 *   iteration    Philox counter word 0 (0 for the first call, then 1, 2, ...)
 *   stream       cudaStream_t (NULL = legacy default stream)
 * The call allocates nothing: its scratch (visited bitmasks, decay table,
 * descriptor, counters) is one static device array of 4 MiB that every GPU
 * loading the library keeps until the process exits. Sizes with
 * m*ceil(n/32) > 1046464 scratch words are rejected with ACS_EINVAL before any
 * device work. The first call on a device looks the array's address up (once
 * per device, with that device current); make that first call before any
 * stream capture. Every call shares the one array: calls that overlap on the
 * GPU (other streams, other host threads) race and corrupt each other. The
 * call blocks until the iteration has finished and returns ACS_ECUDA if a
 * launch or an internal device check failed. */
acs_status acs_iterate_noalloc(const int32_t* dev_coords, int32_t n, const int32_t* dev_nn32,
                               const float* dev_w32, int32_t cl, float tau0, float* dev_tau,
                               int32_t* dev_tours, int64_t* dev_lens, int32_t* dev_best,
                               int64_t* dev_best_len, int64_t iteration, const acs_params* p,
                               void* stream);

const char* acs_strerror(acs_status s);
void acs_destroy(acs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
