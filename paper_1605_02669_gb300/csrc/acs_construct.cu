// acs_construct.cu -- the construct kernel: one full iteration of the Ant
// Colony System (Alg. 1) per instance, one thread-block cluster per instance.
//
// Mapping. The C CTAs of a cluster share one instance; CTA r owns ants
// r*mc .. r*mc+mc-1 (their visited bitmasks live in its shared memory). A
// group of TPA consecutive lanes builds one ant's tour; lane l of the group
// owns candidate ranks l*V .. l*V+V-1 (V = 32/TPA), so the 128-byte
// candidate row (node index and heuristic weight, padded to 32) is read with
// vector loads. Per construction step:
//   A  every ant reads its candidate row, its visited bits, the pheromone of
//      the unvisited candidates (a gather from row c of the matrix, or a probe
//      of record c of the SPM), draws Philox(iteration, ant, step, instance)
//      and applies Eq. 1-2: a group argmax of tau*eta^beta (q < q0) or a
//      Hillis-Steele roulette (Sec. 3.1.1). An ant whose candidate set is
//      empty is queued.
//   B  after the step's selections every warp of the CTA scans all n nodes
//      for the CTA's queued ants (split among them) and takes the argmax of
//      tau*eta^beta over the unvisited ones (ties -> lowest node): the
//      block-level reduction of Sec. 3.1.1. On the SPM the scan reads only
//      the heuristic (every absent trail is tau0) and the record's own
//      entries are offered with their stored trails.
//   C  every CTA reads all m edges through distributed shared memory and
//      counts equal undirected edges (no atomics: each edge is compared with
//      all others by a few threads). An edge taken by k ants gets
//      one folded local update (Eq. 3 applied k times in closed form): on the
//      matrix the CTA of the lowest such ant writes both halves; on the SPM
//      record r is updated by CTA r mod C, which replays that record's events
//      in (ant, side) order (Alg. 3). A second cluster barrier publishes the
//      writes before the next step.
// After the closing edges the cluster sums the tour lengths, keeps the
// best-so-far tour and applies the global update to its n edges.
//
// Mutable global state (pheromone, SPM records, best tour) is written by one
// SM and read by others after a cluster barrier, so it is always read with
// L2-coherent loads (ld.global.cg).
#include <cstdint>
#include <mutex>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "acs_device.cuh"
#include "acs_internal.cuh"

namespace cg = cooperative_groups;

namespace acs {

namespace {

struct Misc {
    int qn[2];                    // queued ants of this CTA, by step parity
    int improved;
    int bestant;
    unsigned long long stat[4];   // fallback, selections, spm hits, spm misses
    long long best_len;
    long long iteration;
    int nrel;                     // edges this CTA writes in the current step
    int next;                     // the cluster's next instance (drawn by rank 0)
    int next_local;               // this CTA's copy of rank 0's draw
};

__device__ __forceinline__ bool visited(const uint32_t* vis, int j)
{
    return (vis[j >> 5] >> (j & 31)) & 1u;
}

// Loads of mutable state: records in shared memory (local or another CTA's,
// through a generic pointer) are read directly; global state is read at L2
// (ld.global.cg) because other SMs of the cluster may have written it.
template <bool GLOBAL>
__device__ __forceinline__ int ld_i(const int32_t* p)
{
    if constexpr (GLOBAL) return __ldcg(p);
    else return *p;
}

template <bool GLOBAL>
__device__ __forceinline__ float ld_f(const float* p)
{
    if constexpr (GLOBAL) return __ldcg(p);
    else return *p;
}

// One SPM record (Sec. 3.2): s neighbour indices, s trails, the tail.
struct Rec {
    int32_t* idx;
    float* val;
    int32_t* tail;
};

// Alg. 3 on one record: a hit updates in place, a miss evicts the slot after
// tail. mode 0 = local (coef = P[k]), 1 = global (coef = rho, target = Delta).
// skip: a local update of an absent edge keeps tau0 and inserts nothing (the
// variant of the insert rule; a miss all the same).
template <bool GLOBAL>
__device__ __forceinline__ bool spm_apply(const Rec& R, int s, int nb, float tau0, int mode,
                                          float coef, float target, bool skip = false)
{
    int hit = -1;
#pragma unroll 8
    for (int i = 0; i < s; ++i)
        if (ld_i<GLOBAL>(R.idx + i) == nb) hit = i;
    if (hit >= 0) {
        const float t = ld_f<GLOBAL>(R.val + hit);
        R.val[hit] = mode == 0 ? local_rule(t, tau0, coef) : global_rule(t, target, coef);
        return true;
    }
    if (skip && mode == 0) return false;
    int t = ld_i<GLOBAL>(R.tail) + 1;
    if (t == s) t = 0;
    *R.tail = t;
    R.idx[t] = nb;
    R.val[t] = mode == 0 ? local_rule(tau0, tau0, coef) : global_rule(tau0, target, coef);
    return false;
}

template <int TPA>
__device__ __forceinline__ unsigned group_mask(int lane)
{
    if constexpr (TPA == 32) return 0xffffffffu;
    else return ((1u << TPA) - 1u) << (lane & ~(TPA - 1));
}

// Warp maximum of the packed keys: the largest high word (product bits) by a
// hardware reduction, then the largest low word among the lanes that hold it.
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k)
{
    const uint32_t hi = (uint32_t)(k >> 32), lo = (uint32_t)k;
    const uint32_t mh = __reduce_max_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    return ((unsigned long long)mh << 32) | ml;
}

template <int V>
__device__ __forceinline__ void load_row(const int32_t* nrow, const float* wrow, int* nv, float* wv)
{
    if constexpr (V == 8) {
        const int4 t0 = reinterpret_cast<const int4*>(nrow)[0];
        const int4 t1 = reinterpret_cast<const int4*>(nrow)[1];
        const float4 u0 = reinterpret_cast<const float4*>(wrow)[0];
        const float4 u1 = reinterpret_cast<const float4*>(wrow)[1];
        nv[0] = t0.x; nv[1] = t0.y; nv[2] = t0.z; nv[3] = t0.w;
        nv[4] = t1.x; nv[5] = t1.y; nv[6] = t1.z; nv[7] = t1.w;
        wv[0] = u0.x; wv[1] = u0.y; wv[2] = u0.z; wv[3] = u0.w;
        wv[4] = u1.x; wv[5] = u1.y; wv[6] = u1.z; wv[7] = u1.w;
    } else if constexpr (V == 4) {
        const int4 t = *reinterpret_cast<const int4*>(nrow);
        const float4 u = *reinterpret_cast<const float4*>(wrow);
        nv[0] = t.x; nv[1] = t.y; nv[2] = t.z; nv[3] = t.w;
        wv[0] = u.x; wv[1] = u.y; wv[2] = u.z; wv[3] = u.w;
    } else if constexpr (V == 2) {
        const int2 t = *reinterpret_cast<const int2*>(nrow);
        const float2 u = *reinterpret_cast<const float2*>(wrow);
        nv[0] = t.x; nv[1] = t.y;
        wv[0] = u.x; wv[1] = u.y;
    } else {
        nv[0] = nrow[0];
        wv[0] = wrow[0];
    }
}

}  // namespace

// Total of `v` over the T consecutive lanes of this lane's segment (a
// hardware warp reduction when the segment is the whole warp).
__device__ __forceinline__ int seg_sum(int v, int T)
{
    if (T == 32) return (int)__reduce_add_sync(0xffffffffu, (unsigned)v);
    for (int off = T / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, T);
    return v;
}

__device__ __forceinline__ int seg_min(int v, int T)
{
    if (T == 32) return __reduce_min_sync(0xffffffffu, v);
    for (int off = T / 2; off >= 1; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off, T));
    return v;
}

// The two halves of a cluster barrier: arrive (release: this thread's prior
// writes become visible to the cluster) and wait (acquire). Work placed
// between them overlaps the barrier's latency.
__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// Bring the line holding p into L2 (no register result, no L1 fill: other SMs
// may write the line before it is read).
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Bring the line holding p into this SM's L1 (read-only data only).
__device__ __forceinline__ void prefetch_l1(const void* p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// MODE 0: pheromone matrix. MODE 1: SPM records in global memory. MODE 2: SPM
// record r resident, for the launch, in the shared memory of CTA r mod C
// (loaded at the start, written back after the global update); other CTAs
// read it through distributed shared memory.
// EXT (SPM only): empty candidate sets are settled from the extended
// neighbour lists where a full scan would be long (a separate variant, so that
// the launches that never use the lists keep the register allocation of the
// plain kernel).
template <int TPA, int MODE, bool EXT>
__global__ void __launch_bounds__(1024, 1) construct_kernel(const ConstructArgs A)
{
    constexpr bool SPM = MODE != 0;
    static_assert(!EXT || SPM, "the extended lists serve the SPM only");
    constexpr bool RG = MODE == 1;   // SPM record loads go through L2
    constexpr int V = 32 / TPA;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31;
    const int gl = lane & (TPA - 1);
    const int group = tid / TPA;
    const int ngroups = nthr / TPA;
    const unsigned gmask = group_mask<TPA>(lane);
    const int gbase = lane & ~(TPA - 1);
    const int m = A.m;
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int mc = A.mc;
    const int a0 = rank * mc;
    const int ml = max(0, min(m, a0 + mc) - a0);   // ants owned by this CTA
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    const int s_slots = A.s;

    for (int oi = cid; oi < A.num_inst;) {
        const int b = A.order[oi];
        const InstDesc D = A.desc[b];
        const int n = D.n, cl = D.cl, W = D.W;
        const float tau0 = D.tau0;
        const SmemLayout L = smem_layout(m, mc, A.nrec, s_slots, W, A.max_n, A.vis_in_smem,
                                         A.xy_in_smem);
        float* sP = (float*)(smem + L.P);
        int* s_cur = (int*)(smem + L.cur);
        int* s_start = (int*)(smem + L.start);
        int* s_nxt = (int*)(smem + L.nxt);
        long long* s_len = (long long*)(smem + L.len);
        uint32_t* pedge = (uint32_t*)(smem + L.pedge);   // (u << 16) | v, or queued | index
        int* qant = (int*)(smem + L.qant);
        int* qc = (int*)(smem + L.qc);
        unsigned long long* qpart = (unsigned long long*)(smem + L.qpart);  // by queue entry
        int* eqal = (int*)(smem + L.eqal);
        uint32_t* gkey = (uint32_t*)(smem + L.gkey);
        int* gu = (int*)(smem + L.gu);
        int* gv = (int*)(smem + L.gv);
        int* grep = (int*)(smem + L.grep);
        int* gcnt = (int*)(smem + L.gcnt);
        int* ev0 = (int*)(smem + L.ev0);
        int* ev1 = (int*)(smem + L.ev1);
        Misc* misc = (Misc*)(smem + L.misc);
        int* s_xj = (int*)(smem + L.xj);   // an ant's list node, when its candidates are visited
        int32_t* ridx_s = (int32_t*)(smem + L.ridx);
        float* rval_s = (float*)(smem + L.rval);
        int32_t* rtail_s = (int32_t*)(smem + L.rtail);
        uint32_t* vis_base = A.vis_in_smem ? (uint32_t*)(smem + L.vis)
                                           : A.vis_global + D.vis_off + (size_t)a0 * W;
        const int2* xy = A.xy_in_smem ? (const int2*)(smem + L.xy)
                                      : (const int2*)(A.xy) + D.xy_off;
        const int32_t* nn_rows = A.nn + 32 * D.row_off;
        const float* w_rows = A.w + 32 * D.row_off;
        const float* hw = A.hw ? A.hw + D.hw_off : nullptr;
        float* tau = A.tau + D.tau_off;           // matrix rows, or SPM values
        int32_t* sidx = A.spm_idx + D.tau_off;    // SPM only
        int32_t* stail = A.spm_tail + D.node_off; // SPM only
        int32_t* tours = A.tours + D.tour_off;
        // SPM: extended neighbour lists of this instance (null = full scans only)
        const int32_t* ext_rows = (EXT && A.ext) ? A.ext + (size_t)kExtList * D.row_off : nullptr;
        int32_t* best = A.best + D.node_off;

        // SPM record r: this CTA's shared copy, another CTA's through DSMEM, or global
        auto rec = [&](int r) -> Rec {
            if constexpr (MODE == 2) {
                const int o = r % C, li = r / C;
                if (o == rank) return Rec{ridx_s + li * s_slots, rval_s + li * s_slots, rtail_s + li};
                return Rec{cluster.map_shared_rank(ridx_s, o) + li * s_slots,
                           cluster.map_shared_rank(rval_s, o) + li * s_slots,
                           cluster.map_shared_rank(rtail_s, o) + li};
            } else {
                return Rec{sidx + (size_t)r * s_slots, tau + (size_t)r * s_slots, stail + r};
            }
        };
        // visited bitmask of ant al of CTA r (for the cluster-wide full scan)
        auto vis_of = [&](int r, int al) -> const uint32_t* {
            if (A.vis_in_smem) return cluster.map_shared_rank(vis_base, r) + (size_t)al * W;
            return A.vis_global + D.vis_off + (size_t)(r * mc + al) * W;
        };

        // ---- per-instance shared set-up
        for (int i = tid; i <= m; i += nthr) sP[i] = A.P[i];
        if (A.xy_in_smem) {
            const int2* gxy = (const int2*)(A.xy) + D.xy_off;
            int2* sxy = (int2*)(smem + L.xy);
            for (int i = tid; i < n; i += nthr) sxy[i] = gxy[i];
        }
        if constexpr (MODE == 2) {
            for (int li = tid; li < A.nrec; li += nthr) {
                const int r = rank + li * C;
                if (r >= n) continue;
                for (int q = 0; q < s_slots; ++q) {
                    ridx_s[li * s_slots + q] = __ldcg(sidx + (size_t)r * s_slots + q);
                    rval_s[li * s_slots + q] = __ldcg(tau + (size_t)r * s_slots + q);
                }
                rtail_s[li] = __ldcg(stail + r);
            }
        }
        if (tid == 0) {
            misc->qn[0] = 0;
            misc->qn[1] = 0;
            misc->best_len = __ldcg(A.best_len + b);
            misc->iteration = __ldcg(A.iteration + b);
            for (int i = 0; i < 4; ++i) misc->stat[i] = 0ull;
        }
        for (int i = tid; i < ml * W; i += nthr) vis_base[i] = 0u;
        __syncthreads();

        const uint32_t it = (uint32_t)misc->iteration;
        const uint32_t inst = (uint32_t)D.instance;

        // ---- step 0: first node of every ant (Alg. 1, uniform draw)
        for (int al = tid; al < ml; al += nthr) {
            const int a = a0 + al;
            const uint4 x = philox4x32_10(make_uint4(it, (uint32_t)a, 0u, inst), A.key0, A.key1);
            const int start = (int)__umulhi(x.z, (uint32_t)n);
            s_cur[al] = start;
            s_start[al] = start;
            tours[(size_t)a * n] = start;
            vis_base[(size_t)al * W + (start >> 5)] |= 1u << (start & 31);
        }
        cluster.sync();

        unsigned long long n_fb = 0, n_hit = 0, n_miss = 0;
        // node of ant al after step s: nodeb[s & 1][al]
        int* const nodeb[2] = {s_cur, s_nxt};
        // Phase A: pseudo-random-proportional rule on the candidate list.
        // stage(): candidate row, visited bits and the step's Philox draw;
        // an ant whose candidate set is empty is queued for phase B.
        auto stage = [&](int stp, int al, int& c, int (&nv)[V], float (&wv)[V],
                         bool (&unv)[V], uint4& x) -> bool {
            const int a = a0 + al;
            c = nodeb[(stp - 1) & 1][al];
            const uint32_t* vis = vis_base + (size_t)al * W;
            load_row<V>(nn_rows + (size_t)c * 32 + gl * V, w_rows + (size_t)c * 32 + gl * V,
                        nv, wv);
            // drawn here so that the rounds overlap the loads' latency
            x = philox4x32_10(make_uint4(it, (uint32_t)a, (uint32_t)stp, inst), A.key0,
                              A.key1);
            bool lane_any = false;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int k = gl * V + i;
                unv[i] = (k < cl) && !visited(vis, nv[i]);
                lane_any |= unv[i];
            }
            const unsigned anyb = __ballot_sync(gmask, lane_any) & gmask;
            if (anyb != 0u) return true;
            if constexpr (EXT) {
                // the list path only where a full scan would deal each of the
                // CTA's warps more than two 128-node items: shorter scans end
                // sooner than the list path's dependent loads
                if (ext_rows && ((n + 127) >> 7) > 2 * (nthr >> 5)) {
                    // the candidate set is empty: the first unvisited node of
                    // the extended list (static data and this ant's own visited
                    // bits, so it is found inside the barrier) stands for every
                    // absent trail of the full scan; choose() weighs it against
                    // the record's entries after the barrier
                    const int32_t* xrow = ext_rows + (size_t)c * kExtList;
                    constexpr int NE = 8;
                    int js = -1;
                    for (int b0 = 0; b0 < kExtList && js < 0; b0 += NE * TPA) {
                        int e[NE];
#pragma unroll
                        for (int i = 0; i < NE; ++i) e[i] = __ldg(xrow + b0 + i * TPA + gl);
#pragma unroll
                        for (int i = 0; i < NE; ++i) {
                            const bool u = e[i] >= 0 && !visited(vis, e[i]);
                            const unsigned bu = __ballot_sync(gmask, u) & gmask;
                            if (bu != 0u && js < 0) js = __shfl_sync(gmask, e[i], __ffs(bu) - 1 - gbase, TPA);
                        }
                    }
                    if (js >= 0) {
                        if (gl == 0) s_xj[al] = js;
                        return true;
                    }
                }
            }
            if (gl == 0) {
                const int qi = atomicAdd(&misc->qn[stp & 1], 1);
                qant[qi] = al;
                qc[qi] = c;
                qpart[qi] = 0ull;
            }
            // phase B scans row c: stage the pheromone row in L2 and the heuristic
            // row (read-only) in this SM's L1
            for (int j = gl * 32; j < n; j += TPA * 32) {
                if constexpr (!SPM) prefetch_l2(tau + (size_t)c * n + j);
                if (hw) prefetch_l1(hw + (size_t)c * n + j);
            }
            return false;
        };
        // choose(): Eq. 1 or Eq. 2 over the unvisited candidates
        auto choose = [&](int stp, int al, int c, const int (&nv)[V], const float (&wv)[V],
                          const bool (&unv)[V], const uint4& x) {
            const int a = a0 + al;
            if constexpr (EXT) {
                bool lane_any = false;
#pragma unroll
                for (int i = 0; i < V; ++i) lane_any |= unv[i];
                if (ext_rows && (__ballot_sync(gmask, lane_any) & gmask) == 0u) {
                    // Alg. 2's full scan, resolved by the extended list: the
                    // largest key among the list's first unvisited node (trail
                    // tau0) and the record's unvisited entries (stored trails)
                    const int js = s_xj[al];
                    const uint32_t* vis = vis_base + (size_t)al * W;
                    const float* hrow = hw ? hw + (size_t)c * n : nullptr;
                    const int2 pc = xy[c];
                    unsigned long long key = 0ull;
                    if (gl == 0) {
                        const float h = hrow ? __ldg(hrow + js) : heuristic(euc2d(pc, xy[js]), A.beta);
                        key = pack_pj(__fmul_rn(tau0, h), js);
                    }
                    const Rec R = rec(c);
                    for (int q = gl; q < s_slots; q += TPA) {
                        const int oj = ld_i<RG>(R.idx + q);
                        const float ot = ld_f<RG>(R.val + q);
                        if (oj >= 0 && !visited(vis, oj)) {
                            const float hj = hrow ? __ldg(hrow + oj) : heuristic(euc2d(pc, xy[oj]), A.beta);
                            const unsigned long long k2 = pack_pj(__fmul_rn(ot, hj), oj);
                            key = k2 > key ? k2 : key;
                        }
                    }
                    if constexpr (TPA == 32) {
                        key = warp_max_u64(key);
                    } else {
#pragma unroll
                        for (int off = TPA / 2; off >= 1; off >>= 1) {
                            const unsigned long long o = __shfl_xor_sync(gmask, key, off, TPA);
                            key = o > key ? o : key;
                        }
                    }
                    const int next = (int)(0xffffffffu - (uint32_t)(key & 0xffffffffull));
                    if (gl == 0) {
                        nodeb[stp & 1][al] = next;
                        pedge[al] = ((uint32_t)c << 16) | (uint32_t)next;
                        tours[(size_t)a * n + stp] = next;
                        vis_base[(size_t)al * W + (next >> 5)] |= 1u << (next & 31);
                        atomicAdd(&misc->stat[0], 1ull);   // a full-scan selection
                    }
                    return;
                }
            }
            float tv[V];
            if constexpr (!SPM) {
                const float* trow = tau + (size_t)c * n;
#pragma unroll
                for (int i = 0; i < V; ++i) tv[i] = unv[i] ? __ldcg(trow + nv[i]) : 0.0f;
            } else {
                const Rec R = rec(c);
#pragma unroll
                for (int i = 0; i < V; ++i) tv[i] = tau0;
                if (s_slots <= TPA) {
                    // lane q of the group loads slot q (one round trip);
                    // the group sees every slot through shuffles
                    int sj = -1;
                    float st = 0.0f;
                    if (gl < s_slots) {
                        sj = ld_i<RG>(R.idx + gl);
                        st = ld_f<RG>(R.val + gl);
                    }
                    for (int q = 0; q < s_slots; ++q) {
                        const int j = __shfl_sync(gmask, sj, q, TPA);
                        const float t = __shfl_sync(gmask, st, q, TPA);
#pragma unroll
                        for (int i = 0; i < V; ++i)
                            if (nv[i] == j) tv[i] = t;
                    }
                } else {
#pragma unroll 8
                    for (int q = 0; q < s_slots; ++q) {
                        const int j = ld_i<RG>(R.idx + q);
                        const float t = ld_f<RG>(R.val + q);
#pragma unroll
                        for (int i = 0; i < V; ++i)
                            if (nv[i] == j) tv[i] = t;
                    }
                }
            }
            float v[V];
#pragma unroll
            for (int i = 0; i < V; ++i) v[i] = unv[i] ? __fmul_rn(tv[i], wv[i]) : 0.0f;

            const float q = unit24(x.x);
            int kpick;
            if (q < A.q0) {
                // exploitation: argmax of tau*eta^beta, ties -> lowest rank.
                // Non-negative floats order like their bit patterns.
                uint32_t mb = 0u;
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (unv[i]) mb = max(mb, __float_as_uint(v[i]));
                if constexpr (TPA == 32) {
                    mb = __reduce_max_sync(0xffffffffu, mb);
                } else {
#pragma unroll
                    for (int off = TPA / 2; off >= 1; off >>= 1)
                        mb = max(mb, __shfl_xor_sync(gmask, mb, off, TPA));
                }
                int first = -1;
#pragma unroll
                for (int i = V - 1; i >= 0; --i)
                    if (unv[i] && __float_as_uint(v[i]) == mb) first = i;
                const unsigned bf = __ballot_sync(gmask, first >= 0) & gmask;
                const int src = __ffs(bf) - 1 - gbase;
                kpick = src * V + __shfl_sync(gmask, first, src, TPA);
            } else {
                // exploration: roulette of Eq. 2 over a 32-position
                // inclusive Hillis-Steele scan (offsets 1,2,4,8,16)
                const float r = unit24(x.y);
                float P[V];
#pragma unroll
                for (int i = 0; i < V; ++i) P[i] = v[i];
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    float y[V];
                    if (off >= V) {
                        const int dl = off / V;
#pragma unroll
                        for (int i = 0; i < V; ++i) {
                            const float o = __shfl_up_sync(gmask, P[i], dl, TPA);
                            y[i] = gl >= dl ? __fadd_rn(P[i], o) : P[i];
                        }
                    } else {
                        float prev[V];
#pragma unroll
                        for (int i = 0; i < V; ++i) {
                            // positions i < off read the previous lane's V-off+i
                            if (i < off) prev[i] = __shfl_up_sync(gmask, P[i - off + V], 1, TPA);
                        }
#pragma unroll
                        for (int i = 0; i < V; ++i) {
                            if (i >= off) y[i] = __fadd_rn(P[i], P[i - off]);
                            else y[i] = gl >= 1 ? __fadd_rn(P[i], prev[i]) : P[i];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < V; ++i) P[i] = y[i];
                }
                const float total = __shfl_sync(gmask, P[V - 1], TPA - 1, TPA);
                const float t = __fmul_rn(r, total);
                int first = -1, last = -1, firstu = -1;
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const bool pos = unv[i] && v[i] > 0.0f;
                    if (first < 0 && pos && P[i] > t) first = i;
                    if (pos) last = i;
                    if (firstu < 0 && unv[i]) firstu = i;
                }
                const unsigned bf = __ballot_sync(gmask, first >= 0) & gmask;
                const unsigned bl = __ballot_sync(gmask, last >= 0) & gmask;
                const unsigned bu = __ballot_sync(gmask, firstu >= 0) & gmask;
                if (bf) {
                    const int src = __ffs(bf) - 1 - gbase;
                    kpick = src * V + __shfl_sync(gmask, first, src, TPA);
                } else if (bl) {
                    const int src = 31 - __clz(bl) - gbase;
                    kpick = src * V + __shfl_sync(gmask, last, src, TPA);
                } else {
                    const int src = __ffs(bu) - 1 - gbase;
                    kpick = src * V + __shfl_sync(gmask, firstu, src, TPA);
                }
            }
            // broadcast the chosen node and its pheromone from the owning lane
            const int owner = kpick / V, ii = kpick - owner * V;
            int myn = nv[0];
#pragma unroll
            for (int i = 1; i < V; ++i)
                if (ii == i) myn = nv[i];
            const int next = __shfl_sync(gmask, myn, owner, TPA);
            if (gl == 0) {
                nodeb[stp & 1][al] = next;
                pedge[al] = ((uint32_t)c << 16) | (uint32_t)next;
                tours[(size_t)a * n + stp] = next;
                vis_base[(size_t)al * W + (next >> 5)] |= 1u << (next & 31);
            }
        };
        // at most one ant per group ("split" steps): the group stages the coming
        // step's candidate row during the barrier that ends a step
        const bool split = ml <= ngroups;
        int st_c = 0, st_nv[V];
        float st_wv[V];
        bool st_unv[V];
        uint4 st_x = make_uint4(0u, 0u, 0u, 0u);
        bool st_busy = false;
        if (split && n > 1 && group < ml) st_busy = stage(1, group, st_c, st_nv, st_wv, st_unv, st_x);
        __syncthreads();   // step 1's queue is complete

        // ---- steps 1 .. n (n = the closing edges)
        for (int step = 1; step <= n; ++step) {
            const bool closing = (step == n);
            const bool upd = (step % A.period) == 0;
            int* qn = &misc->qn[step & 1];
            // the next step's queue counter was last read before the barrier
            // that ended phase B of the previous step
            if (tid == 0) {
                misc->qn[(step + 1) & 1] = 0;
                misc->nrel = 0;   // last read before the barrier that ended the previous step
            }

            if (!closing) {
                // Phase A: pseudo-random-proportional rule on the candidate list
                if (split) {
                    // staged, and the queue published by a CTA barrier, during the
                    // cluster barrier that ended the previous step: warps without
                    // a selection to make start the full scans at once
                    if (st_busy) choose(step, group, st_c, st_nv, st_wv, st_unv, st_x);
                } else {
                    for (int al = group; al < ml; al += ngroups) {
                        int c = 0, nv[V];
                        float wv[V];
                        bool unv[V];
                        uint4 x;
                        if (stage(step, al, c, nv, wv, unv, x)) choose(step, al, c, nv, wv, unv, x);
                    }
                    __syncthreads();   // the step's queue is complete
                }
                __syncwarp();

                // Phase B: the CTA's queued ants take the argmax of tau*eta^beta
                // over all their unvisited nodes (Alg. 2, Sec. 3.1.1). The scan is
                // cut into items of 128 nodes of one queued ant, dealt round-robin
                // to the warps that hold no ant of a split step (they start at
                // once), or to every warp when there are none.
                const int E = *qn;
                const int nch = (n + 127) >> 7;
                const int items = E * nch;
                const int nwarps = nthr >> 5, warp = tid >> 5;
                const int antw = split ? (ml * TPA + 31) >> 5 : 0;   // warps holding ants
                const int fw0 = antw < nwarps ? antw : 0;
                const int nscan = nwarps - fw0;
                for (int item = warp - fw0; warp >= fw0 && item < items; item += nscan) {
                    const int e = item / nch, ch = item - e * nch;
                    const int c = qc[e];
                    const uint32_t* vis = vis_base + (size_t)qant[e] * W;
                    const float* trow = tau + (size_t)c * n;
                    const float* hrow = hw ? hw + (size_t)c * n : nullptr;
                    const int2 pc = xy[c];
                    unsigned long long key = 0ull;
                    uint32_t word[4];
                    float t[4], h[4];
                    // SPM: the record's own entries ride with the first item of
                    // the ant (slot `lane`), loaded first so that they overlap
                    int oj = -1;
                    float ot = 0.0f;
                    if constexpr (SPM) {
                        if (ch == 0 && lane < s_slots) {
                            const Rec R = rec(c);
                            oj = ld_i<RG>(R.idx + lane);
                            ot = ld_f<RG>(R.val + lane);
                        }
                    }
                    // all loads of the item are issued before any is used
                    const int jb = (ch << 7) + lane;
                    if (hrow) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            h[i] = jb + i * 32 < n ? __ldg(hrow + jb + i * 32) : 0.0f;
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j = jb + i * 32;
                        t[i] = tau0;
                        if constexpr (!SPM) if (j < n) t[i] = __ldcg(trow + j);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j = jb + i * 32;
                        word[i] = j < n ? vis[j >> 5] : 0xffffffffu;
                    }
                    if (!hrow) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int j = jb + i * 32;
                            h[i] = j < n ? heuristic(euc2d(pc, xy[j]), A.beta) : 0.0f;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j = (ch << 7) + i * 32 + lane;
                        if (j >= n || ((word[i] >> (j & 31)) & 1u)) continue;
                        const unsigned long long k2 = pack_pj(__fmul_rn(t[i], h[i]), j);
                        key = k2 > key ? k2 : key;
                    }
                    if constexpr (SPM) {
                        // Stored trails are never below tau0 (local and global
                        // updates move a trail towards tau0 or Delta > tau0 without
                        // crossing it), so the scan takes tau0 for every node and
                        // the record's own entries are offered with their stored
                        // trails: the largest product and its lowest node are the
                        // same as with every trail read from the record.
                        if (oj >= 0 && !visited(vis, oj)) {
                            const float hj = hrow ? __ldg(hrow + oj) : heuristic(euc2d(pc, xy[oj]), A.beta);
                            const unsigned long long k2 = pack_pj(__fmul_rn(ot, hj), oj);
                            key = k2 > key ? k2 : key;
                        }
                    }
                    key = warp_max_u64(key);
                    if (lane == 0 && key != 0ull) atomicMax(&qpart[e], key);
                }
                if (E > 0) {
                    __syncthreads();   // every item is merged
                    for (int qi = tid; qi < E; qi += nthr) {
                        const int al = qant[qi], c = qc[qi];
                        const unsigned long long key = qpart[qi];
                        int next = (int)(0xffffffffu - (uint32_t)(key & 0xffffffffull));
                        if (key == 0ull || next < 0 || next >= n) {
                            // no unvisited node: cannot happen before step n
                            atomicExch(A.status, 4);
                            next = c;
                        }
                        nodeb[step & 1][al] = next;
                        tours[(size_t)(a0 + al) * n + step] = next;
                        vis_base[(size_t)al * W + (next >> 5)] |= 1u << (next & 31);
                        pedge[al] = ((uint32_t)c << 16) | (uint32_t)next;
                    }
                    if (tid == 0) n_fb += (unsigned long long)E;
                }
            } else {
                // closing edges (step n): last node back to the first
                for (int al = tid; al < ml; al += nthr) {
                    const int c = nodeb[(step - 1) & 1][al], next = s_start[al];
                    nodeb[step & 1][al] = next;
                    pedge[al] = ((uint32_t)c << 16) | (uint32_t)next;
                }
            }
            cluster.sync();   // the step's edges are visible cluster-wide

            // Phase C: folded local update of the step's distinct edges
            if (upd) {
                // the current trail of this CTA's own edges (matrix): nobody
                // writes them before this CTA applies the update below
                float t_own = 0.0f;
                if constexpr (!SPM) {
                    if (tid < ml) {
                        const uint32_t e = pedge[tid];
                        t_own = __ldcg(tau + (size_t)(e >> 16) * n + (e & 0xffffu));
                    }
                }
                // every CTA gathers all m edges (one thread per ant: m <= nthr).
                // This CTA only needs the edges it writes: on the matrix its own
                // ants' edges, on the SPM the edges that touch one of its records
                // (their events are the only ones replayed here), compacted with
                // one shared-memory atomic per warp.
                if (tid < ((m + 31) & ~31)) {
                    const int a = tid;
                    bool rel = false;
                    if (a < m) {
                        const int r = a / mc;
                        const uint32_t e = cluster.map_shared_rank(pedge, r)[a - r * mc];
                        const int u = (int)(e >> 16), v = (int)(e & 0xffffu);
                        gkey[a] = (uint32_t)min(u, v) * (uint32_t)n + (uint32_t)max(u, v);
                        gu[a] = u;
                        gv[a] = v;
                        rel = (u % C) == rank || (v % C) == rank;
                    }
                    if constexpr (SPM) {
                        const unsigned bal = __ballot_sync(0xffffffffu, rel);
                        int base = 0;
                        if (lane == 0 && bal) base = atomicAdd(&misc->nrel, __popc(bal));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (rel) eqal[base + __popc(bal & ((1u << lane) - 1u))] = a;
                    }
                }
                __syncthreads();
                const int NR = SPM ? misc->nrel : ml;
                // k = ants on the same undirected edge, representative = lowest
                // ant; T threads per relevant edge compare it with every T-th edge
                // (whole warps take part so that the segmented shuffles are valid)
                int T = 1;
                while (T < 32 && 2 * T * NR <= nthr) T *= 2;
                const int tm = (T * NR + 31) & ~31;
                if (tid < tm) {
                    const int i = tid / T, part = tid - i * T;
                    const bool valid = i < NR;
                    const int a = !valid ? 0 : (SPM ? eqal[i] : a0 + i);
                    const uint32_t key = gkey[a];
                    int cnt = 0, rep = a;
                    if (valid) {
                        for (int bb = part; bb < m; bb += T) {
                            if (gkey[bb] == key) {
                                ++cnt;
                                rep = min(rep, bb);
                            }
                        }
                    }
                    cnt = seg_sum(cnt, T);
                    rep = seg_min(rep, T);
                    if (valid && part == 0) {
                        grep[a] = rep;
                        gcnt[a] = cnt;
                        ev0[a] = rep == a ? gu[a] : -1;
                        ev1[a] = rep == a ? gv[a] : -1;
                    }
                }
                __syncthreads();
                if constexpr (!SPM) {
                    // the CTA of the lowest ant on an edge writes both halves
                    if (tid < ml) {
                        const int a = a0 + tid;
                        if (grep[a] == a) {
                            const float t2 = local_rule(t_own, tau0, sP[gcnt[a]]);
                            const int u = gu[a], v = gv[a];
                            tau[(size_t)u * n + v] = t2;
                            tau[(size_t)v * n + u] = t2;
                        }
                    }
                } else {
                    // record r belongs to CTA r mod C. An event's rank among the
                    // events on its record, in (ant, side) order, is its round.
                    bool p0 = false, p1 = false;
                    int u = 0, v = 0, r0 = 0, r1 = 0;
                    float coef = 0.0f;
                    if (tid < tm) {
                        const int i = tid / T, part = tid - i * T;
                        const bool valid = i < NR;
                        const int a = valid ? eqal[i] : 0;
                        const bool isrep = valid && grep[a] == a;
                        u = gu[a];
                        v = gv[a];
                        const bool own0 = isrep && (u % C) == rank;
                        const bool own1 = isrep && (v % C) == rank;
                        if (own0 || own1) {
                            // earlier events (lower ant) on the same records; every
                            // such event belongs to a relevant edge
                            for (int jj = part; jj < NR; jj += T) {
                                const int bb = eqal[jj];
                                if (bb >= a) continue;
                                const int x0 = ev0[bb], x1 = ev1[bb];
                                r0 += (x0 == u) + (x1 == u);
                                r1 += (x0 == v) + (x1 == v);
                            }
                        }
                        r0 = seg_sum(r0, T);
                        r1 = seg_sum(r1, T);
                        if (part == 0 && isrep) {
                            p0 = own0;
                            p1 = own1;
                            coef = sP[gcnt[a]];
                        }
                    }
                    for (int t = 0;; ++t) {
                        if (p0 && r0 == t) {
                            const bool hit = spm_apply<RG>(rec(u), s_slots, v, tau0, 0, coef, 0.0f, A.skip_default);
                            if (hit) ++n_hit; else ++n_miss;
                            p0 = false;
                        }
                        if (p1 && r1 == t) {
                            const bool hit = spm_apply<RG>(rec(v), s_slots, u, tau0, 0, coef, 0.0f, A.skip_default);
                            if (hit) ++n_hit; else ++n_miss;
                            p1 = false;
                        }
                        if (!__syncthreads_or(p0 || p1)) break;
                        if (t > 2 * m + 2) {   // ranks are < 2m: only a bug gets here
                            if (tid == 0) atomicExch(A.status, 5);
                            break;
                        }
                    }
                }
            }
            cluster_arrive();
            // the next step's candidate row, visited bits and draw (static data and
            // this CTA's own state) are staged, and its queue published, while the
            // cluster barrier completes
            if (split) {
                st_busy = false;
                if (step + 1 < n && group < ml)
                    st_busy = stage(step + 1, group, st_c, st_nv, st_wv, st_unv, st_x);
                __syncthreads();
            }
            cluster_wait();
        }

        // ---- tour lengths (Alg. 1 select_best), one group per ant
        for (int al = group; al < ml; al += ngroups) {
            const int a = a0 + al;
            const int32_t* t = tours + (size_t)a * n;
            long long sum = 0;
            for (int i = gl; i < n; i += TPA) {
                const int x = t[i], y = t[i + 1 < n ? i + 1 : 0];
                sum += euc2d(xy[x], xy[y]);
            }
#pragma unroll
            for (int off = TPA / 2; off >= 1; off >>= 1) sum += __shfl_xor_sync(gmask, sum, off, TPA);
            if (gl == 0) {
                s_len[al] = sum;
                A.lens[D.ant_off + a] = sum;
            }
        }
        cluster.sync();
        if (tid < 32) {
            long long bl = 0x7fffffffffffffffll;
            int ba = 0x7fffffff;
            for (int a = tid; a < m; a += 32) {
                const int r = a / mc;
                const long long l = cluster.map_shared_rank(s_len, r)[a - r * mc];
                if (l < bl || (l == bl && a < ba)) { bl = l; ba = a; }
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const long long ol = __shfl_xor_sync(0xffffffffu, bl, off);
                const int oa = __shfl_xor_sync(0xffffffffu, ba, off);
                if (ol < bl || (ol == bl && oa < ba)) { bl = ol; ba = oa; }
            }
            if (tid == 0) {
                misc->improved = bl < misc->best_len ? 1 : 0;
                if (misc->improved) misc->best_len = bl;
                misc->bestant = ba;
            }
        }
        __syncthreads();
        if (misc->improved) {
            // the cluster copies the new best tour, one slice per CTA
            const int32_t* src = tours + (size_t)misc->bestant * n;
            for (int i = rank * nthr + tid; i < n; i += C * nthr) best[i] = __ldcg(src + i);
        }
        cluster.sync();

        // ---- global update on the best-so-far tour (eq. global_update)
        const long long Lgb = misc->best_len;
        const float delta = __double2float_rn(1.0 / (double)Lgb);
        if constexpr (!SPM) {
            for (int i = rank * nthr + tid; i < n; i += C * nthr) {
                const int u = __ldcg(best + i), v = __ldcg(best + (i + 1 < n ? i + 1 : 0));
                const float t2 = global_rule(__ldcg(tau + (size_t)u * n + v), delta, A.rho);
                tau[(size_t)u * n + v] = t2;
                tau[(size_t)v * n + u] = t2;
            }
        } else {
            // record best[i] (owned by CTA best[i] mod C) sees, in tour order, the
            // edge (best[i-1], best[i]) then (best[i], best[i+1]); record best[0]
            // sees edge 0 then edge n-1
            for (int i = tid; i < n; i += nthr) {
                const int r = __ldcg(best + i);
                if (r % C != rank) continue;
                const int prev = __ldcg(best + (i > 0 ? i - 1 : n - 1));
                const int nxt = __ldcg(best + (i + 1 < n ? i + 1 : 0));
                const int first = i > 0 ? prev : nxt;
                const int second = i > 0 ? nxt : prev;
                const Rec R = rec(r);
                bool h = spm_apply<RG>(R, s_slots, first, tau0, 1, A.rho, delta);
                if (h) ++n_hit; else ++n_miss;
                h = spm_apply<RG>(R, s_slots, second, tau0, 1, A.rho, delta);
                if (h) ++n_hit; else ++n_miss;
            }
            atomicAdd(&misc->stat[2], n_hit);
            atomicAdd(&misc->stat[3], n_miss);
        }
        __syncthreads();
        if constexpr (MODE == 2) {
            // write this CTA's records back to global memory
            for (int li = tid; li < A.nrec; li += nthr) {
                const int r = rank + li * C;
                if (r >= n) continue;
                for (int q = 0; q < s_slots; ++q) {
                    sidx[(size_t)r * s_slots + q] = ridx_s[li * s_slots + q];
                    tau[(size_t)r * s_slots + q] = rval_s[li * s_slots + q];
                }
                stail[r] = rtail_s[li];
            }
        }
        if (tid == 0) {
            unsigned long long* st = A.stats + 4 * (size_t)b;
            if constexpr (EXT) atomicAdd(st + 0, n_fb + misc->stat[0]);
            else atomicAdd(st + 0, n_fb);
            if (rank == 0) atomicAdd(st + 1, (unsigned long long)m * (unsigned long long)(n - 1));
            atomicAdd(st + 2, misc->stat[2]);
            atomicAdd(st + 3, misc->stat[3]);
            if (rank == 0) {
                A.best_len[b] = misc->best_len;
                A.iteration[b] = misc->iteration + 1;
            }
        }
        cluster.sync();
        // The first ncl instances (longest first) go to clusters 0..ncl-1; with
        // a counter, a cluster that finishes then takes the next untaken
        // instance. Rank 0 draws it; each CTA's thread 0 copies it from rank
        // 0's shared memory between two cluster barriers (the second keeps
        // rank 0 from rewriting it or exiting before every CTA has read it),
        // and the CTA reads its own copy, a load the compiler keeps
        // warp-uniform, so the instance's values stay in uniform registers.
        if (A.sched) {
            if (rank == 0 && tid == 0) misc->next = ncl + atomicAdd(A.sched, 1);
            cluster.sync();
            if (tid == 0) misc->next_local = cluster.map_shared_rank(misc, 0)->next;
            cluster.sync();
            oi = misc->next_local;
        } else {
            oi += ncl;
        }
    }
}

template <int TPA, int MODE, bool EXT>
static void* kernel_ptr()
{
    return reinterpret_cast<void*>(construct_kernel<TPA, MODE, EXT>);
}

template <int MODE, bool EXT>
static void* select_tpa(int tpa)
{
    switch (tpa) {
    case 4: return kernel_ptr<4, MODE, EXT>();
    case 8: return kernel_ptr<8, MODE, EXT>();
    case 16: return kernel_ptr<16, MODE, EXT>();
    case 32: return kernel_ptr<32, MODE, EXT>();
    default: return nullptr;
    }
}

// variant = kernel mode (0 matrix, 1 SPM in global memory, 2 SPM resident),
// plus kExtVariant for the SPM modes with the extended lists
static void* select_kernel(int tpa, int variant)
{
    switch (variant) {
    case 0: return select_tpa<0, false>(tpa);
    case 1: return select_tpa<1, false>(tpa);
    case 2: return select_tpa<2, false>(tpa);
    case 1 + kExtVariant: return select_tpa<1, true>(tpa);
    case 2 + kExtVariant: return select_tpa<2, true>(tpa);
    default: return nullptr;
    }
}

// Raises the kernel's dynamic shared-memory limit to at least `smem` and
// allows clusters above 8 CTAs (outside any stream capture). The limit is a
// per-function setting shared by every context in the process, so it is only
// ever raised: lowering it would make the launches of an existing context
// with a larger layout fail.
cudaError_t prepare_construct(int tpa, int mode, size_t smem)
{
    static std::mutex mu;
    void* k = select_kernel(tpa, mode);
    if (!k) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lock(mu);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Clusters of `csize` CTAs that can be resident at once (0 if none fits).
int construct_occupancy(int tpa, int mode, int block, size_t smem, int csize)
{
    void* k = select_kernel(tpa, mode);
    if (!k) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = csize;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nclusters;
}

// Stream-ordered launch of one iteration on clusters of `csize` CTAs; safe
// inside a stream capture (the counter reset becomes a memset node). grid
// must be a multiple of csize.
cudaError_t launch_construct(const ConstructArgs& A, int tpa, int mode, int grid, int block,
                             size_t smem, int csize, cudaStream_t stream)
{
    void* k = select_kernel(tpa, mode);
    if (!k) return cudaErrorInvalidValue;
    if (A.sched) {
        const cudaError_t e = cudaMemsetAsync(A.sched, 0, sizeof(int32_t), stream);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = csize;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<ConstructArgs*>(&A)};
    return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace acs
