// acs_construct.cu -- the construct kernel: one full iteration of the Ant
// Colony System (Alg. 1) per instance, one CTA per instance.
//
// Mapping. A group of TPA consecutive lanes builds one ant's tour; lane l of
// the group owns candidate ranks l*V .. l*V+V-1 (V = 32/TPA), so the
// 128-byte candidate row (node index and heuristic weight, padded to 32) is
// read with one vector load per lane. Groups loop over ants when m exceeds
// the groups of the CTA. Per step:
//   A  every ant reads its candidate row, the visited bitmask (shared memory
//      when it fits), the pheromone of the unvisited candidates (a gather
//      from row c of the matrix, or a probe of record c of the SPM), draws
//      Philox(iteration, ant, step, instance) and applies Eq. 1-2 with a
//      group argmax (q < q0) or a Hillis-Steele roulette (Sec. 3.1.1). An ant
//      whose candidate set is empty is queued.
//   B  the whole CTA scans all nodes for each queued ant and reduces the
//      argmax of tau*eta^beta with 64-bit shared atomics (the block-level
//      full scan of Sec. 3.1.1, here shared by all queued ants).
//   C  the step's edges, deduplicated in a shared hash table, receive one
//      folded local update each (Eq. 3 applied k times in closed form):
//      matrix entries are written in both halves; SPM records are updated in
//      rounds so that each record sees its events in (ant, side) order.
// After the closing edges the CTA sums the tour lengths, keeps the best-so-
// far tour and applies the global update to its n edges.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "acs_device.cuh"
#include "acs_internal.cuh"

namespace acs {

namespace {

struct Misc {
    int fbcount;
    int improved;
    int bestant;
    int pad;
    unsigned long long stat[4];   // fallback, selections, spm hits, spm misses
    unsigned long long red[32];
    long long best_len;
    long long iteration;
};

__device__ __forceinline__ bool visited(const uint32_t* vis, int j)
{
    return (vis[j >> 5] >> (j & 31)) & 1u;
}

__device__ __forceinline__ int2 load_xy(const int2* xy, int j)
{
    return xy[j];
}

// Probe record c of the SPM for neighbour j (absent -> tau0).
__device__ __forceinline__ float spm_read(const int32_t* idx, const float* val, int s, int j,
                                          float tau0)
{
    float t = tau0;
    for (int i = 0; i < s; ++i)
        if (idx[i] == j) t = val[i];
    return t;
}

// Alg. 3 on one record: a hit updates in place, a miss evicts the slot after
// tail. mode 0 = local (coef = P[k]), 1 = global (coef = rho, target = Delta).
__device__ __forceinline__ bool spm_apply(int32_t* idx, float* val, int32_t* tail, int s,
                                          int nb, float tau0, int mode, float coef, float target)
{
    for (int i = 0; i < s; ++i) {
        if (idx[i] == nb) {
            const float t = val[i];
            val[i] = mode == 0 ? local_rule(t, tau0, coef) : global_rule(t, target, coef);
            return true;
        }
    }
    int t = *tail + 1;
    if (t == s) t = 0;
    *tail = t;
    idx[t] = nb;
    val[t] = mode == 0 ? local_rule(tau0, tau0, coef) : global_rule(tau0, target, coef);
    return false;
}

// Edge hash insert: returns the slot; counts visits and keeps the lowest ant.
__device__ __forceinline__ int edge_insert(uint32_t* ekey, int* ecnt, int* erep, int H,
                                           uint32_t key, int ant, int32_t* status)
{
    const int shift = 32 - __ffs(H) + 1;
    int slot = (int)(hash32(key) >> shift);
    for (int probe = 0; probe < H; ++probe) {
        const uint32_t old = atomicCAS(&ekey[slot], kEmpty, key);
        if (old == kEmpty || old == key) {
            atomicAdd(&ecnt[slot], 1);
            atomicMin(&erep[slot], ant);
            return slot;
        }
        slot = (slot + 1) & (H - 1);
    }
    atomicExch(status, 2);
    return 0;
}

__device__ __forceinline__ int rec_insert(uint32_t* rkey, int H2, uint32_t rec, int32_t* status)
{
    const int shift = 32 - __ffs(H2) + 1;
    int slot = (int)(hash32(rec) >> shift);
    for (int probe = 0; probe < H2; ++probe) {
        const uint32_t old = atomicCAS(&rkey[slot], kEmpty, rec);
        if (old == kEmpty || old == rec) return slot;
        slot = (slot + 1) & (H2 - 1);
    }
    atomicExch(status, 3);
    return 0;
}

template <int TPA>
__device__ __forceinline__ unsigned group_mask(int lane)
{
    if constexpr (TPA == 32) return 0xffffffffu;
    else return ((1u << TPA) - 1u) << (lane & ~(TPA - 1));
}

}  // namespace

template <int TPA, bool SPM>
__global__ void __launch_bounds__(1024, 1) construct_kernel(const ConstructArgs A)
{
    constexpr int V = 32 / TPA;
    extern __shared__ __align__(16) unsigned char smem[];

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31;
    const int gl = lane & (TPA - 1);
    const int group = tid / TPA;
    const int ngroups = nthr / TPA;
    const unsigned gmask = group_mask<TPA>(lane);
    const int m = A.m;

    for (int oi = blockIdx.x; oi < A.num_inst; oi += gridDim.x) {
        const int b = A.order[oi];
        const InstDesc D = A.desc[b];
        const int n = D.n, cl = D.cl, W = D.W;
        const float tau0 = D.tau0;
        const SmemLayout L = smem_layout(m, A.H, A.H2, W, A.max_n, A.vis_in_smem, A.xy_in_smem);
        float* sP = (float*)(smem + L.P);
        int* s_cur = (int*)(smem + L.cur);
        int* s_start = (int*)(smem + L.start);
        int* s_nxt = (int*)(smem + L.nxt);
        int* s_slot = (int*)(smem + L.slot);
        float* s_tsel = (float*)(smem + L.tsel);
        long long* s_len = (long long*)(smem + L.len);
        uint32_t* ekey = (uint32_t*)(smem + L.ekey);
        int* ecnt = (int*)(smem + L.ecnt);
        int* erep = (int*)(smem + L.erep);
        uint32_t* rkey = (uint32_t*)(smem + L.rkey);
        uint32_t* rmin = (uint32_t*)(smem + L.rmin);  // two buffers of H2
        int* fbant = (int*)(smem + L.fbant);
        unsigned long long* fbkey = (unsigned long long*)(smem + L.fbkey);
        Misc* misc = (Misc*)(smem + L.misc);
        uint32_t* vis_base = A.vis_in_smem ? (uint32_t*)(smem + L.vis) : A.vis_global + D.vis_off;
        const int2* xy = A.xy_in_smem ? (const int2*)(smem + L.xy)
                                      : (const int2*)(A.xy) + D.xy_off;
        const int32_t* nn_rows = A.nn + 32 * D.row_off;
        const float* w_rows = A.w + 32 * D.row_off;
        float* tau = A.tau + D.tau_off;           // matrix rows, or SPM values
        int32_t* sidx = A.spm_idx + D.tau_off;    // SPM only
        int32_t* stail = A.spm_tail + D.node_off; // SPM only
        int32_t* tours = A.tours + D.tour_off;
        int32_t* best = A.best + D.node_off;
        const int s_slots = A.s;

        // ---- per-instance shared set-up
        for (int i = tid; i <= m; i += nthr) sP[i] = A.P[i];
        for (int i = tid; i < A.H; i += nthr) { ekey[i] = kEmpty; ecnt[i] = 0; erep[i] = 0x7fffffff; }
        for (int i = tid; i < A.H2; i += nthr) { rkey[i] = kEmpty; rmin[i] = kEmpty; rmin[A.H2 + i] = kEmpty; }
        if (A.xy_in_smem) {
            const int2* gxy = (const int2*)(A.xy) + D.xy_off;
            int2* sxy = (int2*)(smem + L.xy);
            for (int i = tid; i < n; i += nthr) sxy[i] = gxy[i];
        }
        if (tid == 0) {
            misc->fbcount = 0;
            misc->best_len = A.best_len[b];
            misc->iteration = A.iteration[b];
            for (int i = 0; i < 4; ++i) misc->stat[i] = 0ull;
        }
        for (int i = tid; i < m * W; i += nthr) vis_base[i] = 0u;
        __syncthreads();

        const uint32_t it = (uint32_t)misc->iteration;
        const uint32_t inst = (uint32_t)D.instance;

        // ---- step 0: first node of every ant (Alg. 1, uniform draw)
        for (int a = tid; a < m; a += nthr) {
            const uint4 x = philox4x32_10(make_uint4(it, (uint32_t)a, 0u, inst), A.key0, A.key1);
            const int start = (int)__umulhi(x.z, (uint32_t)n);
            s_cur[a] = start;
            s_start[a] = start;
            tours[(size_t)a * n] = start;
            vis_base[(size_t)a * W + (start >> 5)] |= 1u << (start & 31);
        }
        __syncthreads();

        unsigned long long n_fb = 0, n_sel = 0, n_hit = 0, n_miss = 0;

        // ---- steps 1 .. n (n = the closing edges)
        for (int step = 1; step <= n; ++step) {
            const bool closing = (step == n);
            const bool upd = (step % A.period) == 0;

            if (!closing) {
                // Phase A: pseudo-random-proportional rule on the candidate list
                for (int a = group; a < m; a += ngroups) {
                    const int c = s_cur[a];
                    const uint32_t* vis = vis_base + (size_t)a * W;
                    const int32_t* nrow = nn_rows + (size_t)c * 32 + gl * V;
                    const float* wrow = w_rows + (size_t)c * 32 + gl * V;
                    int nv[V];
                    float wv[V];
                    if (V == 4) {
                        const int4 t = *reinterpret_cast<const int4*>(nrow);
                        const float4 u = *reinterpret_cast<const float4*>(wrow);
                        nv[0] = t.x; nv[1] = t.y; nv[2 % V] = t.z; nv[3 % V] = t.w;
                        wv[0] = u.x; wv[1] = u.y; wv[2 % V] = u.z; wv[3 % V] = u.w;
                    } else if (V == 2) {
                        const int2 t = *reinterpret_cast<const int2*>(nrow);
                        const float2 u = *reinterpret_cast<const float2*>(wrow);
                        nv[0] = t.x; nv[1 % V] = t.y;
                        wv[0] = u.x; wv[1 % V] = u.y;
                    } else {
                        nv[0] = nrow[0];
                        wv[0] = wrow[0];
                    }
                    bool unv[V];
                    bool lane_any = false;
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        const int k = gl * V + i;
                        unv[i] = (k < cl) && !visited(vis, nv[i]);
                        lane_any |= unv[i];
                    }
                    const unsigned anyb = __ballot_sync(gmask, lane_any) & gmask;
                    if (anyb == 0u) {
                        if (gl == 0) {
                            const int e = atomicAdd(&misc->fbcount, 1);
                            fbant[e] = a;
                            fbkey[e] = 0ull;
                        }
                        continue;
                    }
                    float tv[V];
                    if (!SPM) {
                        const float* trow = tau + (size_t)c * n;
#pragma unroll
                        for (int i = 0; i < V; ++i) tv[i] = unv[i] ? trow[nv[i]] : 0.0f;
                    } else {
                        const int32_t* ri = sidx + (size_t)c * s_slots;
                        const float* rv = tau + (size_t)c * s_slots;
#pragma unroll
                        for (int i = 0; i < V; ++i) tv[i] = tau0;
                        for (int q = 0; q < s_slots; ++q) {
                            const int j = ri[q];
                            const float t = rv[q];
#pragma unroll
                            for (int i = 0; i < V; ++i)
                                if (nv[i] == j) tv[i] = t;
                        }
                    }
                    float v[V];
#pragma unroll
                    for (int i = 0; i < V; ++i) v[i] = unv[i] ? __fmul_rn(tv[i], wv[i]) : 0.0f;

                    const uint4 x = philox4x32_10(make_uint4(it, (uint32_t)a, (uint32_t)step, inst),
                                                  A.key0, A.key1);
                    const float q = unit24(x.x);
                    int kpick;
                    if (q < A.q0) {
                        // exploitation: argmax of tau*eta^beta, ties -> lowest rank
                        unsigned long long bk = 0ull;
#pragma unroll
                        for (int i = 0; i < V; ++i) {
                            if (unv[i]) {
                                const unsigned long long key =
                                    ((unsigned long long)__float_as_uint(v[i]) << 32) |
                                    (unsigned long long)(0xffffffffu - (uint32_t)(gl * V + i));
                                bk = key > bk ? key : bk;
                            }
                        }
#pragma unroll
                        for (int off = TPA / 2; off >= 1; off >>= 1) {
                            const unsigned long long o = __shfl_xor_sync(gmask, bk, off, TPA);
                            bk = o > bk ? o : bk;
                        }
                        kpick = (int)(0xffffffffu - (uint32_t)(bk & 0xffffffffull));
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
                                    if (i >= off) y[i] = __fadd_rn(P[i], P[(i - off + V) % V]);
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
                        const int base = lane & ~(TPA - 1);
                        if (bf) {
                            const int src = __ffs(bf) - 1;
                            kpick = (src - base) * V + __shfl_sync(gmask, first, src - base, TPA);
                        } else if (bl) {
                            const int src = 31 - __clz(bl);
                            kpick = (src - base) * V + __shfl_sync(gmask, last, src - base, TPA);
                        } else {
                            const int src = __ffs(bu) - 1;
                            kpick = (src - base) * V + __shfl_sync(gmask, firstu, src - base, TPA);
                        }
                    }
                    // broadcast the chosen node and its pheromone from the owning lane
                    const int owner = kpick / V, ii = kpick - owner * V;
                    int myn = nv[0];
                    float myt = tv[0];
#pragma unroll
                    for (int i = 1; i < V; ++i)
                        if (ii == i) { myn = nv[i]; myt = tv[i]; }
                    const int next = __shfl_sync(gmask, myn, owner, TPA);
                    const float tsel = __shfl_sync(gmask, myt, owner, TPA);
                    if (gl == 0) {
                        s_nxt[a] = next;
                        s_tsel[a] = tsel;
                        tours[(size_t)a * n + step] = next;
                        vis_base[(size_t)a * W + (next >> 5)] |= 1u << (next & 31);
                        if (upd) {
                            const uint32_t lo = (uint32_t)min(c, next), hi = (uint32_t)max(c, next);
                            s_slot[a] = edge_insert(ekey, ecnt, erep, A.H, lo * (uint32_t)n + hi, a,
                                                    A.status);
                        }
                    }
                }
                __syncthreads();

                // Phase B: full scan for ants whose candidate set is empty
                const int E = misc->fbcount;
                if (E > 0) {
                    for (int e = 0; e < E; ++e) {
                        const int a = fbant[e];
                        const int c = s_cur[a];
                        const uint32_t* vis = vis_base + (size_t)a * W;
                        const int2 pc = load_xy(xy, c);
                        unsigned long long bk = 0ull;
                        if (!SPM) {
                            const float* trow = tau + (size_t)c * n;
                            for (int j = tid; j < n; j += nthr) {
                                if (visited(vis, j)) continue;
                                const float p = __fmul_rn(trow[j], heuristic(euc2d(pc, load_xy(xy, j)), A.beta));
                                const unsigned long long key =
                                    ((unsigned long long)__float_as_uint(p) << 32) | (0xffffffffu - (uint32_t)j);
                                bk = key > bk ? key : bk;
                            }
                        } else {
                            const int32_t* ri = sidx + (size_t)c * s_slots;
                            const float* rv = tau + (size_t)c * s_slots;
                            for (int j = tid; j < n; j += nthr) {
                                if (visited(vis, j)) continue;
                                const float t = spm_read(ri, rv, s_slots, j, tau0);
                                const float p = __fmul_rn(t, heuristic(euc2d(pc, load_xy(xy, j)), A.beta));
                                const unsigned long long key =
                                    ((unsigned long long)__float_as_uint(p) << 32) | (0xffffffffu - (uint32_t)j);
                                bk = key > bk ? key : bk;
                            }
                        }
#pragma unroll
                        for (int off = 16; off >= 1; off >>= 1) {
                            const unsigned long long o = __shfl_xor_sync(0xffffffffu, bk, off);
                            bk = o > bk ? o : bk;
                        }
                        if (lane == 0 && bk != 0ull) atomicMax(&fbkey[e], bk);
                    }
                    __syncthreads();
                    for (int e = tid; e < E; e += nthr) {
                        const int a = fbant[e];
                        const int c = s_cur[a];
                        const unsigned long long bk = fbkey[e];
                        const int next = (int)(0xffffffffu - (uint32_t)(bk & 0xffffffffull));
                        if (bk == 0ull || next < 0 || next >= n) { atomicExch(A.status, 4); continue; }
                        s_nxt[a] = next;
                        if (!SPM) {
                            s_tsel[a] = tau[(size_t)c * n + next];
                        } else {
                            s_tsel[a] = 0.0f;
                        }
                        tours[(size_t)a * n + step] = next;
                        vis_base[(size_t)a * W + (next >> 5)] |= 1u << (next & 31);
                        if (upd) {
                            const uint32_t lo = (uint32_t)min(c, next), hi = (uint32_t)max(c, next);
                            s_slot[a] = edge_insert(ekey, ecnt, erep, A.H, lo * (uint32_t)n + hi, a,
                                                    A.status);
                        }
                    }
                    if (tid == 0) {
                        n_fb += (unsigned long long)E;
                        misc->fbcount = 0;
                    }
                    __syncthreads();
                }
                if (tid == 0) n_sel += (unsigned long long)m;
            } else {
                // closing edges (step n): last node back to the first
                for (int a = tid; a < m; a += nthr) {
                    const int c = s_cur[a], next = s_start[a];
                    s_nxt[a] = next;
                    if (upd) {
                        if (!SPM) s_tsel[a] = tau[(size_t)c * n + next];
                        const uint32_t lo = (uint32_t)min(c, next), hi = (uint32_t)max(c, next);
                        s_slot[a] = edge_insert(ekey, ecnt, erep, A.H, lo * (uint32_t)n + hi, a, A.status);
                    }
                }
                __syncthreads();
            }

            // Phase C: folded local update of the step's distinct edges (thread a = ant a)
            if (!SPM) {
                if (tid < m) {
                    const int a = tid;
                    const int u = s_cur[a], v = s_nxt[a];
                    if (upd) {
                        const int slot = s_slot[a];
                        if (erep[slot] == a) {
                            const int k = ecnt[slot];
                            const float t2 = local_rule(s_tsel[a], tau0, sP[k]);
                            tau[(size_t)u * n + v] = t2;
                            tau[(size_t)v * n + u] = t2;
                            ekey[slot] = kEmpty;
                            ecnt[slot] = 0;
                            erep[slot] = 0x7fffffff;
                        }
                    }
                    s_cur[a] = v;
                }
                __syncthreads();
            } else {
                bool p0 = false, p1 = false;
                int u = 0, v = 0, rs0 = 0, rs1 = 0;
                float coef = 0.0f;
                if (tid < m) {
                    const int a = tid;
                    u = s_cur[a];
                    v = s_nxt[a];
                    if (upd) {
                        const int slot = s_slot[a];
                        if (erep[slot] == a) {
                            coef = sP[ecnt[slot]];
                            rs0 = rec_insert(rkey, A.H2, (uint32_t)u, A.status);
                            rs1 = rec_insert(rkey, A.H2, (uint32_t)v, A.status);
                            p0 = p1 = true;
                            ekey[slot] = kEmpty;
                            ecnt[slot] = 0;
                            erep[slot] = 0x7fffffff;
                        }
                    }
                    s_cur[a] = v;
                }
                int round = 0;
                bool used0 = p0, used1 = p1;
                // each round retires the lowest pending event of every record, so
                // at most 2m rounds are needed; the bound only guards against a bug
                while (__syncthreads_or(p0 || p1)) {
                    if (round > 2 * m + 2) {
                        if (tid == 0) atomicExch(A.status, 5);
                        p0 = p1 = false;
                        continue;
                    }
                    uint32_t* rm = rmin + (round & 1) * A.H2;
                    const uint32_t o0 = 2u * (uint32_t)tid, o1 = o0 + 1u;
                    if (p0) atomicMin(&rm[rs0], o0);
                    if (p1) atomicMin(&rm[rs1], o1);
                    __syncthreads();
                    if (p0 && rm[rs0] == o0) {
                        const bool hit = spm_apply(sidx + (size_t)u * s_slots, tau + (size_t)u * s_slots,
                                                   stail + u, s_slots, v, tau0, 0, coef, 0.0f);
                        if (hit) ++n_hit; else ++n_miss;
                        rm[rs0] = kEmpty;
                        p0 = false;
                    }
                    if (p1 && rm[rs1] == o1) {
                        const bool hit = spm_apply(sidx + (size_t)v * s_slots, tau + (size_t)v * s_slots,
                                                   stail + v, s_slots, u, tau0, 0, coef, 0.0f);
                        if (hit) ++n_hit; else ++n_miss;
                        rm[rs1] = kEmpty;
                        p1 = false;
                    }
                    ++round;
                }
                if (used0) rkey[rs0] = kEmpty;
                if (used1) rkey[rs1] = kEmpty;
                // the next writer of rkey is the next step's phase C, two barriers away
            }
        }

        // ---- tour lengths (Alg. 1 select_best), one group per ant
        for (int a = group; a < m; a += ngroups) {
            const int32_t* t = tours + (size_t)a * n;
            long long sum = 0;
            for (int i = gl; i < n; i += TPA) {
                const int x = t[i], y = t[i + 1 < n ? i + 1 : 0];
                sum += euc2d(load_xy(xy, x), load_xy(xy, y));
            }
#pragma unroll
            for (int off = TPA / 2; off >= 1; off >>= 1) sum += __shfl_xor_sync(gmask, sum, off, TPA);
            if (gl == 0) {
                s_len[a] = sum;
                A.lens[D.ant_off + a] = sum;
            }
        }
        __syncthreads();
        if (tid < 32) {
            long long bl = 0x7fffffffffffffffll;
            int ba = 0x7fffffff;
            for (int a = tid; a < m; a += 32) {
                const long long l = s_len[a];
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
            const int32_t* src = tours + (size_t)misc->bestant * n;
            for (int i = tid; i < n; i += nthr) best[i] = src[i];
            __syncthreads();
        }

        // ---- global update on the best-so-far tour (eq. global_update)
        const long long Lgb = misc->best_len;
        const float delta = __double2float_rn(1.0 / (double)Lgb);
        if (!SPM) {
            for (int i = tid; i < n; i += nthr) {
                const int u = best[i], v = best[i + 1 < n ? i + 1 : 0];
                const float t2 = global_rule(tau[(size_t)u * n + v], delta, A.rho);
                tau[(size_t)u * n + v] = t2;
                tau[(size_t)v * n + u] = t2;
            }
        } else {
            // record best[i] sees, in tour order, the edge (best[i-1], best[i])
            // then (best[i], best[i+1]); record best[0] sees edge 0 then edge n-1
            for (int i = tid; i < n; i += nthr) {
                const int r = best[i];
                const int prev = best[i > 0 ? i - 1 : n - 1];
                const int nxt = best[i + 1 < n ? i + 1 : 0];
                const int first = i > 0 ? prev : nxt;
                const int second = i > 0 ? nxt : prev;
                int32_t* ri = sidx + (size_t)r * s_slots;
                float* rv = tau + (size_t)r * s_slots;
                bool h = spm_apply(ri, rv, stail + r, s_slots, first, tau0, 1, A.rho, delta);
                if (h) ++n_hit; else ++n_miss;
                h = spm_apply(ri, rv, stail + r, s_slots, second, tau0, 1, A.rho, delta);
                if (h) ++n_hit; else ++n_miss;
            }
        }
        if (SPM) {
            atomicAdd(&misc->stat[2], n_hit);
            atomicAdd(&misc->stat[3], n_miss);
        }
        __syncthreads();
        if (tid == 0) {
            A.best_len[b] = misc->best_len;
            A.iteration[b] = misc->iteration + 1;
            unsigned long long* st = A.stats + 4 * (size_t)b;
            st[0] += n_fb;
            st[1] += n_sel;
            st[2] += misc->stat[2];
            st[3] += misc->stat[3];
        }
        __syncthreads();
    }
}

template <int TPA, bool SPM>
static void* kernel_ptr()
{
    return reinterpret_cast<void*>(construct_kernel<TPA, SPM>);
}

static void* select_kernel(int tpa, bool spm)
{
    switch (tpa) {
    case 8: return spm ? kernel_ptr<8, true>() : kernel_ptr<8, false>();
    case 16: return spm ? kernel_ptr<16, true>() : kernel_ptr<16, false>();
    case 32: return spm ? kernel_ptr<32, true>() : kernel_ptr<32, false>();
    default: return nullptr;
    }
}

// Raises the kernel's dynamic shared-memory limit to at least `smem` (outside
// any stream capture). The limit is a per-function setting shared by every
// context in the process, so it is only ever raised: lowering it would make
// the launches of an existing context with a larger layout fail.
cudaError_t prepare_construct(int tpa, bool spm, size_t smem)
{
    static std::mutex mu;
    void* k = select_kernel(tpa, spm);
    if (!k) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int construct_occupancy(int tpa, bool spm, int block, size_t smem)
{
    void* k = select_kernel(tpa, spm);
    int occ = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return occ;
}

// Stream-ordered launch of one iteration; safe inside a stream capture.
cudaError_t launch_construct(const ConstructArgs& A, int tpa, bool spm, int grid, int block,
                             size_t smem, cudaStream_t stream)
{
    void* k = select_kernel(tpa, spm);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {const_cast<ConstructArgs*>(&A)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, stream);
}

}  // namespace acs
