// acs_relaxed.cu -- the relaxed construction of ACS-GPU-Alt (Sec. 3.1.2):
// every ant builds its whole tour in one kernel pass with no step barrier,
// and applies the local update (Eq. 3) to each edge as soon as it takes it,
// with plain loads and stores. Concurrent updates of one edge may be lost and
// an ant may see another ant's update of the same step or not: the results
// depend on timing (the paper accepts this for speed; the tours stay valid).
// The iteration's evaluation, best-so-far and global update (eq.
// global_update) run in a second kernel, one CTA per instance.
//
// Mapping: one warp per ant (the candidate list is 32 wide: lane k holds
// candidate k), four ants per CTA, the CTAs of all instances in one launch.
// The rules are those of the synchronous kernel: Eq. 1 argmax (ties -> lowest
// rank), Eq. 2 roulette over the inclusive Hillis-Steele scan of the 32
// candidates, the full scan of Alg. 2 (ties -> lowest node) when every
// candidate is visited, Philox4x32-10 keyed by (iteration, ant, step,
// instance). Matrix memory only.
#include <cstdint>

#include <cuda_runtime.h>

#include "acs_device.cuh"
#include "acs_internal.cuh"

namespace acs {

namespace {

constexpr int kAntsPerCta = 4;

__device__ __forceinline__ unsigned long long pack_key(float p, int j)
{
    return ((unsigned long long)__float_as_uint(p) << 32) |
           (unsigned long long)(0xffffffffu - (uint32_t)j);
}

__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k)
{
    const uint32_t hi = (uint32_t)(k >> 32), lo = (uint32_t)k;
    const uint32_t mh = __reduce_max_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    return ((unsigned long long)mh << 32) | ml;
}

__global__ void __launch_bounds__(32 * kAntsPerCta)
relaxed_construct_kernel(const ConstructArgs A)
{
    extern __shared__ uint32_t rsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.y;
    const InstDesc D = A.desc[b];
    const int n = D.n, cl = D.cl, W = D.W;
    const int m = A.m;
    const int a = blockIdx.x * kAntsPerCta + warp;
    if (a >= m) return;   // whole warps leave; no block barrier follows
    uint32_t* vis = rsm + (size_t)warp * W;
    for (int i = lane; i < W; i += 32) vis[i] = 0u;
    __syncwarp();

    const int2* xy = reinterpret_cast<const int2*>(A.xy) + D.xy_off;
    const int32_t* nn_rows = A.nn + 32 * D.row_off;
    const float* w_rows = A.w + 32 * D.row_off;
    const float* hw = A.hw ? A.hw + D.hw_off : nullptr;
    float* tau = A.tau + D.tau_off;
    int32_t* tour = A.tours + D.tour_off + (size_t)a * n;
    const float tau0 = D.tau0;
    const float P1 = A.P[1];
    const uint32_t it = (uint32_t)A.iteration[b];
    const uint32_t inst = (uint32_t)D.instance;

    // step 0: first node (Alg. 1)
    const uint4 x0 = philox4x32_10(make_uint4(it, (uint32_t)a, 0u, inst), A.key0, A.key1);
    const int start = (int)__umulhi(x0.z, (uint32_t)n);
    if (lane == 0) tour[0] = start;
    if (lane == 0) vis[start >> 5] |= 1u << (start & 31);
    __syncwarp();

    int c = start;
    unsigned long long n_fb = 0;
    // the candidate row of the current city, loaded one step ahead
    int nb = nn_rows[(size_t)c * 32 + lane];
    float wv = w_rows[(size_t)c * 32 + lane];
    for (int step = 1; step <= n; ++step) {
        int next;
        float tnext;   // the trail of the edge taken, as read for the choice
        if (step < n) {
            const uint4 x = philox4x32_10(make_uint4(it, (uint32_t)a, (uint32_t)step, inst), A.key0,
                                          A.key1);
            const bool unv = lane < cl && !((vis[nb >> 5] >> (nb & 31)) & 1u);
            const unsigned anyb = __ballot_sync(0xffffffffu, unv);
            if (anyb) {
                const float t = unv ? __ldcg(tau + (size_t)c * n + nb) : 0.0f;
                const float v = unv ? __fmul_rn(t, wv) : 0.0f;
                int k;
                if (unit24(x.x) < A.q0) {
                    // Eq. 1: argmax, ties -> lowest rank (non-negative floats
                    // order like their bit patterns)
                    const uint32_t mb = __reduce_max_sync(0xffffffffu, unv ? __float_as_uint(v) : 0u);
                    const unsigned bf = __ballot_sync(0xffffffffu, unv && __float_as_uint(v) == mb);
                    k = __ffs(bf) - 1;
                } else {
                    // Eq. 2: roulette over the inclusive scan of the 32 positions
                    float P = v;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const float o = __shfl_up_sync(0xffffffffu, P, off);
                        if (lane >= off) P = __fadd_rn(P, o);
                    }
                    const float total = __shfl_sync(0xffffffffu, P, 31);
                    const float thr = __fmul_rn(unit24(x.y), total);
                    const bool pos = unv && v > 0.0f;
                    const unsigned bf = __ballot_sync(0xffffffffu, pos && P > thr);
                    const unsigned bl = __ballot_sync(0xffffffffu, pos);
                    k = bf ? __ffs(bf) - 1 : (bl ? 31 - __clz(bl) : __ffs(anyb) - 1);
                }
                next = __shfl_sync(0xffffffffu, nb, k);
                tnext = __shfl_sync(0xffffffffu, t, k);
            } else {
                // Alg. 2's full scan by the ant's warp: argmax of tau*eta^beta
                // over the unvisited nodes, ties -> lowest node
                unsigned long long key = 0ull;
                const float* trow = tau + (size_t)c * n;
                const float* hrow = hw ? hw + (size_t)c * n : nullptr;
                const int2 pc = xy[c];
                for (int j0 = lane; j0 < n; j0 += 128) {
                    float t4[4], h4[4];
                    uint32_t w4[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j = j0 + i * 32;
                        t4[i] = j < n ? __ldcg(trow + j) : 0.0f;
                        h4[i] = (j < n && hrow) ? __ldg(hrow + j) : 0.0f;
                        w4[i] = j < n ? vis[j >> 5] : 0xffffffffu;
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j = j0 + i * 32;
                        if (j >= n || ((w4[i] >> (j & 31)) & 1u)) continue;
                        const float h = hrow ? h4[i] : heuristic(euc2d(pc, xy[j]), A.beta);
                        const unsigned long long k2 = pack_key(__fmul_rn(t4[i], h), j);
                        key = k2 > key ? k2 : key;
                    }
                }
                key = warp_max_key(key);
                next = (int)(0xffffffffu - (uint32_t)(key & 0xffffffffull));
                if (key == 0ull || next < 0 || next >= n) {
                    if (lane == 0) atomicExch(A.status, 4);
                    next = c;
                }
                tnext = __ldcg(trow + next);
                ++n_fb;
            }
            if (lane == 0) {
                tour[step] = next;
                vis[next >> 5] |= 1u << (next & 31);
            }
        } else {
            next = start;   // the closing edge
            tnext = __ldcg(tau + (size_t)c * n + next);
        }
        // the next city's candidate row (static data) is requested before the
        // update, so that its latency overlaps
        if (step + 1 < n) {
            nb = nn_rows[(size_t)next * 32 + lane];
            wv = w_rows[(size_t)next * 32 + lane];
        }
        // local update of the edge just taken (Eq. 3), immediately, from the
        // trail read for the choice, with plain stores: a concurrent update of
        // the same edge may be lost
        if ((step % A.period) == 0 && lane == 0) {
            const float t2 = local_rule(tnext, tau0, P1);
            __stcg(tau + (size_t)c * n + next, t2);
            __stcg(tau + (size_t)next * n + c, t2);
        }
        __syncwarp();
        c = next;
    }
    // tour length (Alg. 1 evaluation)
    long long sum = 0;
    for (int i = lane; i < n; i += 32) sum += euc2d(xy[tour[i]], xy[tour[i + 1 < n ? i + 1 : 0]]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) {
        A.lens[D.ant_off + a] = sum;
        if (n_fb) atomicAdd(A.stats + 4 * (size_t)b, n_fb);
    }
}

// Iteration best (ties -> lowest ant), best-so-far (strict improvement) and
// the global update on the best-so-far tour; one CTA per instance.
__global__ void __launch_bounds__(1024) relaxed_epilogue_kernel(const ConstructArgs A)
{
    __shared__ long long s_len[32];
    __shared__ int s_ant[32];
    __shared__ int s_improved;
    const int b = blockIdx.x;
    const InstDesc D = A.desc[b];
    const int n = D.n, m = A.m;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long bl = 0x7fffffffffffffffll;
    int ba = 0x7fffffff;
    for (int a = tid; a < m; a += blockDim.x) {
        const long long l = A.lens[D.ant_off + a];
        if (l < bl || (l == bl && a < ba)) { bl = l; ba = a; }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const long long ol = __shfl_xor_sync(0xffffffffu, bl, off);
        const int oa = __shfl_xor_sync(0xffffffffu, ba, off);
        if (ol < bl || (ol == bl && oa < ba)) { bl = ol; ba = oa; }
    }
    if (lane == 0) { s_len[warp] = bl; s_ant[warp] = ba; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (s_len[w] < bl || (s_len[w] == bl && s_ant[w] < ba)) { bl = s_len[w]; ba = s_ant[w]; }
        s_improved = bl < A.best_len[b];
        if (s_improved) A.best_len[b] = bl;
        s_ant[0] = ba;
    }
    __syncthreads();
    int32_t* best = A.best + D.node_off;
    if (s_improved) {
        const int32_t* src = A.tours + D.tour_off + (size_t)s_ant[0] * n;
        for (int i = tid; i < n; i += blockDim.x) best[i] = src[i];
    }
    __syncthreads();
    const float delta = __double2float_rn(1.0 / (double)A.best_len[b]);
    float* tau = A.tau + D.tau_off;
    for (int i = tid; i < n; i += blockDim.x) {
        const int u = best[i], v = best[i + 1 < n ? i + 1 : 0];
        const float t2 = global_rule(__ldcg(tau + (size_t)u * n + v), delta, A.rho);
        tau[(size_t)u * n + v] = t2;
        tau[(size_t)v * n + u] = t2;
    }
    if (tid == 0) {
        atomicAdd(A.stats + 4 * (size_t)b + 1, (unsigned long long)m * (unsigned long long)(n - 1));
        A.iteration[b] = A.iteration[b] + 1;
    }
}

}  // namespace

// One relaxed iteration of every instance: construction, then evaluation and
// global update. Stream-ordered; safe inside a stream capture.
cudaError_t launch_relaxed(const ConstructArgs& A, int num_inst, int max_w, cudaStream_t stream)
{
    const dim3 grid((A.m + kAntsPerCta - 1) / kAntsPerCta, num_inst);
    const size_t smem = sizeof(uint32_t) * (size_t)kAntsPerCta * max_w;
    relaxed_construct_kernel<<<grid, 32 * kAntsPerCta, smem, stream>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    relaxed_epilogue_kernel<<<num_inst, 1024, 0, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace acs
