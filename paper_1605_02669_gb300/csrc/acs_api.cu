// acs_api.cu -- host side of libacs: the C ABI of include/acs.h, the set-up
// kernels (candidate lists, nearest-neighbour tour, pheromone initialisation)
// and the per-iteration CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <utility>
#include <vector>

#include "acs.h"
#include "acs_device.cuh"
#include "acs_internal.cuh"

namespace acs {
cudaError_t prepare_construct(int tpa, int mode, size_t smem);
cudaError_t launch_construct(const ConstructArgs& A, int tpa, int mode, int grid, int block,
                             size_t smem, int csize, cudaStream_t stream);
int construct_occupancy(int tpa, int mode, int block, size_t smem, int csize);
cudaError_t launch_relaxed(const ConstructArgs& A, int num_inst, int max_w, cudaStream_t stream);
}  // namespace acs

using namespace acs;

// ------------------------------------------------------------------ kernels

// Candidate lists (Sec. 3, Alg. 2): one warp per node c selects the cl
// smallest keys (d_cj, j) in cl rounds of a warp-wide minimum above the
// previous key; rows are padded to 32 with -1 / 0.
__global__ void knn_kernel(const InstDesc* desc, const int32_t* xy, int32_t* nn, float* w, int beta)
{
    const InstDesc D = desc[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= D.n) return;
    const int2* p = reinterpret_cast<const int2*>(xy) + D.xy_off;
    const int2 pc = p[c];
    int32_t* nrow = nn + 32 * (D.row_off + c);
    float* wrow = w + 32 * (D.row_off + c);
    unsigned long long prev = 0ull;
    for (int r = 0; r < 32; ++r) {
        if (r >= D.cl) {
            if (lane == 0) { nrow[r] = -1; wrow[r] = 0.0f; }
            continue;
        }
        unsigned long long bk = ~0ull;
        for (int j = lane; j < D.n; j += 32) {
            if (j == c) continue;
            const unsigned long long key = ((unsigned long long)euc2d(pc, p[j]) << 32) | (uint32_t)j;
            if ((r == 0 || key > prev) && key < bk) bk = key;
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, bk, off);
            bk = o < bk ? o : bk;
        }
        prev = bk;
        if (lane == 0) {
            nrow[r] = (int32_t)(bk & 0xffffffffull);
            wrow[r] = heuristic((int32_t)(bk >> 32), beta);
        }
    }
}

// Nearest-neighbour tour from node 0 (ties -> lowest index), one CTA per
// instance; sets tau0 = (float)(1/((double)n * L_nn)).
// Offer a tour (already checked to be a permutation) as the best-so-far of
// instance b: its EUC_2D length is summed by one CTA and the tour replaces
// the best-so-far only when strictly shorter (Alg. 1's rule).
__global__ void offer_best_kernel(const InstDesc* desc, int b, const int32_t* xy,
                                  const int32_t* tour, int32_t* best, int64_t* best_len,
                                  int64_t* len_out)
{
    __shared__ long long part[32];
    __shared__ int take;
    const InstDesc D = desc[b];
    const int n = D.n, tid = threadIdx.x;
    const int2* p = reinterpret_cast<const int2*>(xy) + D.xy_off;
    long long sum = 0;
    for (int i = tid; i < n; i += blockDim.x) sum += euc2d(p[tour[i]], p[tour[i + 1 < n ? i + 1 : 0]]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if ((tid & 31) == 0) part[tid >> 5] = sum;
    __syncthreads();
    if (tid == 0) {
        long long L = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) L += part[w];
        take = L < best_len[b];
        if (take) best_len[b] = L;
        *len_out = L;
    }
    __syncthreads();
    if (take)
        for (int i = tid; i < n; i += blockDim.x) best[D.node_off + i] = tour[i];
}

// Nearest-neighbour tour from node 0 (ties -> lowest index) and tau0 =
// 1/(n*L_nn), one warp per instance. The candidate list of the current node
// holds its cl nearest nodes in (distance, index) order, so while one of them
// is unvisited the first such one is the nearest unvisited node; only when
// all are visited does the warp scan every node.
__global__ void nn_tour_kernel(InstDesc* desc, const int32_t* xy, const int32_t* nn,
                               int64_t* L_out)
{
    extern __shared__ uint32_t vis[];
    InstDesc* D = desc + blockIdx.x;
    const int n = D->n, cl = D->cl, lane = threadIdx.x;
    const int W = (n + 31) >> 5;
    const int2* p = reinterpret_cast<const int2*>(xy) + D->xy_off;
    const int32_t* rows = nn + 32 * D->row_off;
    for (int i = lane; i < W; i += 32) vis[i] = 0u;
    __syncwarp();
    if (lane == 0) vis[0] = 1u;
    __syncwarp();
    long long L = 0;
    int cur = 0;
    for (int step = 1; step < n; ++step) {
        const int2 pc = p[cur];
        const int j = lane < cl ? rows[(size_t)cur * 32 + lane] : -1;
        const bool unv = j >= 0 && !((vis[j >> 5] >> (j & 31)) & 1u);
        const unsigned bal = __ballot_sync(0xffffffffu, unv);
        int nx;
        if (bal) {
            nx = __shfl_sync(0xffffffffu, j, __ffs(bal) - 1);
        } else {
            unsigned long long bk = ~0ull;
            for (int q = lane; q < n; q += 32) {
                if ((vis[q >> 5] >> (q & 31)) & 1u) continue;
                const unsigned long long key = ((unsigned long long)euc2d(pc, p[q]) << 32) | (uint32_t)q;
                bk = key < bk ? key : bk;
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, bk, off);
                bk = o < bk ? o : bk;
            }
            nx = (int)(bk & 0xffffffffull);
        }
        if (lane == 0) {
            L += euc2d(pc, p[nx]);
            vis[nx >> 5] |= 1u << (nx & 31);
        }
        __syncwarp();
        cur = nx;
    }
    if (lane == 0) {
        L += euc2d(p[cur], p[0]);
        L_out[blockIdx.x] = L;
        D->tau0 = __double2float_rn(1.0 / ((double)n * (double)L));
    }
}

__global__ void init_matrix_kernel(const InstDesc* desc, float* tau)
{
    const InstDesc D = desc[blockIdx.y];
    const size_t total = (size_t)D.n * D.n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        tau[D.tau_off + i] = D.tau0;
}

__global__ void init_spm_kernel(const InstDesc* desc, int32_t* idx, float* val, int32_t* tail, int s)
{
    const InstDesc D = desc[blockIdx.y];
    const size_t total = (size_t)D.n * s;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        idx[D.tau_off + i] = -1;
        val[D.tau_off + i] = 0.0f;
    }
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)D.n;
         i += (size_t)gridDim.x * blockDim.x)
        tail[D.node_off + i] = s - 1;
}

// Heuristic matrix hw[c][j] = eta_cj^beta of every pair (the full scan of the
// fallback reads it instead of recomputing EUC_2D and the division).
__global__ void hw_kernel(const InstDesc* desc, const int32_t* xy, float* hw, int beta)
{
    const InstDesc D = desc[blockIdx.y];
    const int2* p = reinterpret_cast<const int2*>(xy) + D.xy_off;
    const size_t total = (size_t)D.n * D.n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / D.n), j = (int)(i - (size_t)c * D.n);
        hw[D.hw_off + i] = heuristic(euc2d(p[c], p[j]), beta);
    }
}

// Bitonic network on keys[0..N) in shared memory, largest first, by the
// CTA's 256 threads (N = 256 or 512).
template <int N>
__device__ void sort_desc(unsigned long long* keys)
{
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += 256) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = keys[i], b = keys[ixj];
                    if (((i & k) == 0) ? (a < b) : (a > b)) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// SPM extended neighbour lists. For node c: the kExtList nodes j != c with
// the largest full-scan keys pack_pj(tau0 * eta(c, j)^beta, j) of an absent
// trail, largest first (-1 padded when n - 1 < kExtList). Every trail absent
// from a record is tau0 (Sec. 3.2), so the first unvisited node of this list
// is the full scan's choice among absent trails (Alg. 2); the construct
// kernel compares it with the record's entries and scans all n nodes only
// when every listed node is visited. One CTA of 256 threads per node: a
// sorted top list, refreshed from a buffer of the keys that beat its last
// entry (bitonic sort and merge).
__global__ void __launch_bounds__(256) ext_list_kernel(const InstDesc* desc, const int32_t* xy,
                                                       int32_t* ext, int beta)
{
    __shared__ unsigned long long top[kExtList];
    __shared__ unsigned long long buf[2 * kExtList];
    __shared__ int cnt;
    const InstDesc D = desc[blockIdx.y];
    const int n = D.n, t = threadIdx.x;
    const int2* p = reinterpret_cast<const int2*>(xy) + D.xy_off;
    auto key_of = [&](int c, int j) -> unsigned long long {
        if (j == c || j >= n) return 0ull;
        return pack_pj(__fmul_rn(D.tau0, heuristic(euc2d(p[c], p[j]), beta)), j);
    };
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        top[t] = key_of(c, t);
        if (t == 0) cnt = 0;
        __syncthreads();
        sort_desc<kExtList>(top);
        for (int j0 = kExtList; j0 < n; j0 += 256) {
            const unsigned long long thr = top[kExtList - 1];
            const unsigned long long k = key_of(c, j0 + t);
            if (k > thr) buf[atomicAdd(&cnt, 1)] = k;
            __syncthreads();
            const int nb = cnt;
            __syncthreads();   // every thread has read cnt before it changes again
            if (nb >= kExtList || (j0 + 256 >= n && nb > 0)) {
                for (int i = nb + t; i < 2 * kExtList; i += 256) buf[i] = 0ull;
                __syncthreads();
                sort_desc<2 * kExtList>(buf);
                // the kExtList largest of both sorted lists form a bitonic
                // sequence: the larger of top[i] and buf[kExtList - 1 - i]
                const unsigned long long a = top[t], b = buf[kExtList - 1 - t];
                __syncthreads();
                top[t] = a > b ? a : b;
                if (t == 0) cnt = 0;
                __syncthreads();
                for (int j = kExtList >> 1; j > 0; j >>= 1) {
                    const int ixj = t ^ j;
                    if (ixj > t) {
                        const unsigned long long x = top[t], y = top[ixj];
                        if (x < y) {
                            top[t] = y;
                            top[ixj] = x;
                        }
                    }
                    __syncthreads();
                }
            }
        }
        const unsigned long long k = top[t];
        ext[((size_t)D.row_off + c) * kExtList + t] = k ? (int32_t)(0xffffffffu - (uint32_t)k) : -1;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ context

struct acs_ctx {
    int B = 0;
    acs_params p{};
    int m = 0, s = 0;
    std::vector<int32_t> n, cl;
    std::vector<InstDesc> desc_h;
    int max_n = 0;
    // device memory
    InstDesc* d_desc = nullptr;
    int32_t* d_order = nullptr;
    int32_t* d_xy = nullptr;
    int32_t* d_nn = nullptr;
    float* d_w = nullptr;
    float* d_hw = nullptr;
    int32_t* d_ext = nullptr;    // SPM extended neighbour lists [rows][kExtList]
    float* d_tau = nullptr;
    int32_t* d_spm_idx = nullptr;
    int32_t* d_spm_tail = nullptr;
    int32_t* d_tours = nullptr;
    int64_t* d_lens = nullptr;
    int32_t* d_best = nullptr;
    int64_t* d_best_len = nullptr;
    int64_t* d_iter = nullptr;
    unsigned long long* d_stats = nullptr;
    uint32_t* d_vis = nullptr;
    float* d_P = nullptr;
    int32_t* d_status = nullptr;
    int32_t* d_sched = nullptr;   // next-instance counter of the dynamic schedule
    int64_t* d_Lnn = nullptr;
    std::vector<void*> allocs;
    // execution
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ConstructArgs args{};
    int tpa = 8, grid = 1, block = 256, sms = 1, csize = 1, max_smem = 0, mode = 0;
    int variant = 0;   // mode, plus kExtVariant when the SPM kernel uses the extended lists
    bool vis_smem = true, xy_smem = false;
    bool spm_resident = true;   // SPM records in shared memory when they fit
    size_t smem = 0;
    int64_t iteration = 0;             // iterations completed by instance 0
    std::vector<uint8_t> has_best;     // per instance: a best-so-far tour exists
    std::vector<int32_t> ids;          // per instance: Philox counter word 3
    bool poisoned = false;
    int64_t last_launches = 0;
};

namespace {

template <typename T>
cudaError_t dalloc(acs_ctx* c, T** p, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
}

void free_all(acs_ctx* c)
{
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    for (void* q : c->allocs) cudaFree(q);
    c->allocs.clear();
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    c->own_stream = nullptr;
}

acs_status validate_params(const acs_params* p)
{
    if (!p) return ACS_EINVAL;
    if (p->m < 1 || p->m > kMaxM) return ACS_EINVAL;
    if (p->cl < 1 || p->cl > kMaxCl) return ACS_EINVAL;
    if (p->beta < 0 || p->beta > 8) return ACS_EINVAL;
    if (!(p->q0 >= 0.0f && p->q0 <= 1.0f)) return ACS_EINVAL;
    if (!(p->rho > 0.0f && p->rho < 1.0f)) return ACS_EINVAL;
    if (!(p->xi > 0.0f && p->xi < 1.0f)) return ACS_EINVAL;
    if (p->memory != ACS_MEM_MATRIX && p->memory != ACS_MEM_SPM) return ACS_EINVAL;
    if (p->memory == ACS_MEM_SPM && (p->spm_slots < 1 || p->spm_slots > 32)) return ACS_EINVAL;
    if (p->local_period < 1 ||
        (p->flags & ~(ACS_FLAG_RELAXED | ACS_FLAG_SPM_SKIP_DEFAULT)) != 0)
        return ACS_EINVAL;
    if ((p->flags & ACS_FLAG_RELAXED) && p->memory != ACS_MEM_MATRIX) return ACS_EINVAL;
    return ACS_OK;
}

acs_status fail_cuda(acs_ctx* c, cudaError_t e)
{
    if (e != cudaSuccess) {
        if (c) c->poisoned = true;
        return ACS_ECUDA;
    }
    return ACS_OK;
}

#define ACS_TRY(expr)                                   \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) {                        \
            cudaGetLastError();                         \
            return _e;                                  \
        }                                               \
    } while (0)

// Shared-memory plan and block/grid of the construct launch for a
// (threads-per-ant, cluster size) pair: each CTA of a cluster owns
// mc = ceil(m/csize) ants, one group of tpa lanes per ant, at least one thread
// per ant of the instance (the update phase), at most 1024 threads (all 1024
// when the clusters of all instances fit on the GPU at once); as many
// clusters as fit on the GPU, at most one per instance.
cudaError_t configure(acs_ctx* c, int tpa, int csize)
{
    const int m = c->m;
    const int mc = (m + csize - 1) / csize;
    const int W = (c->max_n + 31) / 32;
    const bool spm = c->p.memory == ACS_MEM_SPM;
    const uint32_t lim = (uint32_t)c->max_smem;
    // SPM records resident in shared memory when this CTA's share fits
    int nrec = 0;
    if (spm) {
        const int want = (c->max_n + csize - 1) / csize;
        if (c->spm_resident && smem_layout(m, mc, want, c->s, W, c->max_n, false, false).total <= lim)
            nrec = want;
    }
    const int s = c->s;
    const SmemLayout base = smem_layout(m, mc, nrec, s, W, c->max_n, false, false);
    const bool vis_smem = base.total + 4ull * mc * W <= (unsigned long long)lim;
    const bool xy_smem =
        vis_smem && smem_layout(m, mc, nrec, s, W, c->max_n, true, true).total <= lim;
    const SmemLayout L = smem_layout(m, mc, nrec, s, W, c->max_n, vis_smem, xy_smem);
    if (L.total > lim) return cudaErrorInvalidConfiguration;
    if (!vis_smem && !c->d_vis) {
        size_t words = 0;
        for (int b = 0; b < c->B; ++b) {
            c->desc_h[b].vis_off = (int64_t)words;
            words += (size_t)m * c->desc_h[b].W;
        }
        ACS_TRY(dalloc(c, &c->d_vis, words));
        ACS_TRY(cudaMemcpyAsync(c->d_desc, c->desc_h.data(), sizeof(InstDesc) * c->B,
                                cudaMemcpyHostToDevice, c->stream));
        ACS_TRY(cudaStreamSynchronize(c->stream));
    }
    int block = std::max(mc * tpa, m);
    // Spare warps speed up the full scan of the fallback: when every instance's
    // cluster has SMs of its own, each CTA gets the full 1024 threads.
    if ((long long)c->B * csize <= (long long)c->sms) block = 1024;
    block = std::min(1024, std::max(64, block));
    block = (block + 31) / 32 * 32;
    if (block < m) return cudaErrorInvalidConfiguration;
    const int mode = !spm ? 0 : (nrec > 0 ? 2 : 1);
    // the SPM variant with the extended lists when some instance's full scan
    // would deal each warp of a CTA more than two 128-node items (the kernel
    // applies the same test per instance)
    const bool ext = spm && ((c->max_n + 127) >> 7) > 2 * (block >> 5);
    const int variant = mode + (ext ? kExtVariant : 0);
    if (ext && !c->d_ext) {
        // built once, the first time a launch shape uses them (tau0 is in the
        // descriptors by now); stream-ordered before any launch that reads them
        size_t rows = 0;
        for (int b = 0; b < c->B; ++b) rows += (size_t)c->n[b];
        ACS_TRY(dalloc(c, &c->d_ext, (size_t)kExtList * rows));
        ext_list_kernel<<<dim3(std::min(c->max_n, 4096), c->B), 256, 0, c->stream>>>(c->d_desc, c->d_xy,
                                                                                  c->d_ext, c->p.beta);
        ACS_TRY(cudaGetLastError());
        c->args.ext = c->d_ext;
    }
    ACS_TRY(prepare_construct(tpa, variant, L.total));
    const int ncl = construct_occupancy(tpa, variant, block, L.total, csize);
    if (ncl < 1) return cudaErrorInvalidConfiguration;
    c->tpa = tpa;
    c->csize = csize;
    c->mode = mode;
    c->variant = variant;
    c->block = block;
    c->smem = L.total;
    c->vis_smem = vis_smem;
    c->xy_smem = xy_smem;
    c->grid = std::min(c->B, ncl) * csize;
    // more instances than resident clusters: a cluster that finishes takes the
    // next instance in longest-first order (list scheduling) instead of a
    // fixed share; results do not depend on which cluster runs an instance
    c->args.sched = c->B > ncl ? c->d_sched : nullptr;
    c->args.vis_in_smem = vis_smem ? 1 : 0;
    c->args.xy_in_smem = xy_smem ? 1 : 0;
    c->args.vis_global = c->d_vis;
    c->args.mc = mc;
    c->args.nrec = nrec;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    return cudaSuccess;
}

// Default cluster size: the largest power of two up to 16 that leaves at
// least 16 ants per CTA and lets every instance's cluster be resident at once.
int default_cluster_size(const acs_ctx* c)
{
    int cs = 16;
    while (cs > 1 && (c->m / cs < 16 || c->B * cs > c->sms)) cs >>= 1;
    return cs;
}

// Default lanes per ant: a full warp per ant when an instance spans a cluster
// (few instances, latency-bound steps); 8 lanes otherwise, so that several
// CTAs share an SM when many instances run at once.
int default_tpa(const acs_ctx* c, int cs)
{
    if (cs == 1) return 8;
    const int mc = (c->m + cs - 1) / cs;
    int tpa = 32;
    while (tpa > 4 && mc * tpa > 1024) tpa >>= 1;
    return tpa;
}

cudaError_t plan_launch(acs_ctx* c)
{
    int dev = 0;
    ACS_TRY(cudaGetDevice(&dev));
    ACS_TRY(cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    ACS_TRY(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
    ConstructArgs& A = c->args;
    A.desc = c->d_desc;
    A.order = c->d_order;
    A.num_inst = c->B;
    A.m = c->m;
    A.xy = c->d_xy;
    A.nn = c->d_nn;
    A.w = c->d_w;
    A.hw = c->d_hw;
    A.ext = c->d_ext;
    A.tau = c->d_tau;
    A.spm_idx = c->d_spm_idx;
    A.spm_tail = c->d_spm_tail;
    A.tours = c->d_tours;
    A.lens = c->d_lens;
    A.best = c->d_best;
    A.best_len = c->d_best_len;
    A.iteration = c->d_iter;
    A.stats = c->d_stats;
    A.P = c->d_P;
    A.status = c->d_status;
    A.q0 = c->p.q0;
    A.rho = c->p.rho;
    A.beta = c->p.beta;
    A.s = c->s;
    A.period = c->p.local_period;
    A.skip_default = (c->p.flags & ACS_FLAG_SPM_SKIP_DEFAULT) ? 1 : 0;
    A.key0 = (uint32_t)(c->p.seed & 0xffffffffull);
    A.key1 = (uint32_t)(c->p.seed >> 32);
    A.max_n = c->max_n;
    // largest cluster that fits, falling back to smaller ones
    for (int cs = default_cluster_size(c); cs >= 1; cs >>= 1) {
        cudaError_t e = configure(c, default_tpa(c, cs), cs);
        if (e == cudaSuccess) return e;
        if (e != cudaErrorInvalidConfiguration) return e;
        cudaGetLastError();
    }
    return cudaErrorInvalidConfiguration;
}

cudaError_t build(acs_ctx* c, const int32_t* coords, const int64_t* offsets)
{
    const int B = c->B, m = c->m;
    int64_t total_n = offsets[B];
    size_t tau_total = 0, tour_total = 0;
    c->desc_h.resize(B);
    for (int b = 0; b < B; ++b) {
        InstDesc& D = c->desc_h[b];
        const int n = c->n[b];
        D.n = n;
        D.cl = c->cl[b];
        D.W = (n + 31) / 32;
        D.instance = c->ids[b];
        D.xy_off = offsets[b];
        D.row_off = offsets[b];
        D.tau_off = (int64_t)tau_total;
        D.node_off = offsets[b];
        D.tour_off = (int64_t)tour_total;
        D.ant_off = (int64_t)b * m;
        D.vis_off = 0;
        D.hw_off = D.tau_off;
        D.tau0 = 0.0f;
        D.pad = 0;
        tau_total += c->p.memory == ACS_MEM_MATRIX ? (size_t)n * n : (size_t)n * c->s;
        tour_total += (size_t)m * n;
    }
    std::vector<int32_t> order(B);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return c->n[a] > c->n[b]; });

    ACS_TRY(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    c->stream = c->own_stream;
    ACS_TRY(dalloc(c, &c->d_desc, B));
    ACS_TRY(dalloc(c, &c->d_order, B));
    ACS_TRY(dalloc(c, &c->d_xy, 2 * (size_t)total_n));
    ACS_TRY(dalloc(c, &c->d_nn, 32 * (size_t)total_n));
    ACS_TRY(dalloc(c, &c->d_w, 32 * (size_t)total_n));
    // heuristic matrix for the full scan, when all instances' n^2 floats fit
    // the budget (always for the matrix memory, whose offsets it shares)
    size_t hw_total = 0;
    for (int b = 0; b < B; ++b) hw_total += (size_t)c->n[b] * c->n[b];
    const size_t kHwBudget = (size_t)64 << 30;
    if (hw_total * sizeof(float) <= kHwBudget) {
        if (c->p.memory == ACS_MEM_SPM) {
            size_t off = 0;
            for (int b = 0; b < B; ++b) {
                c->desc_h[b].hw_off = (int64_t)off;
                off += (size_t)c->n[b] * c->n[b];
            }
        }
        ACS_TRY(dalloc(c, &c->d_hw, hw_total));
    }
    ACS_TRY(dalloc(c, &c->d_tau, tau_total));
    if (c->p.memory == ACS_MEM_SPM) {
        ACS_TRY(dalloc(c, &c->d_spm_idx, tau_total));
        ACS_TRY(dalloc(c, &c->d_spm_tail, (size_t)total_n));
    }
    ACS_TRY(dalloc(c, &c->d_tours, tour_total));
    ACS_TRY(dalloc(c, &c->d_lens, (size_t)B * m));
    ACS_TRY(dalloc(c, &c->d_best, (size_t)total_n));
    ACS_TRY(dalloc(c, &c->d_best_len, B));
    ACS_TRY(dalloc(c, &c->d_iter, B));
    ACS_TRY(dalloc(c, &c->d_stats, 4 * (size_t)B));
    ACS_TRY(dalloc(c, &c->d_P, (size_t)m + 1));
    ACS_TRY(dalloc(c, &c->d_status, 1));
    ACS_TRY(dalloc(c, &c->d_sched, 1));
    ACS_TRY(dalloc(c, &c->d_Lnn, B));

    // decay table P[0] = 1, P[k] = P[k-1]*(1-xi), FP32
    std::vector<float> P(m + 1);
    const float f = 1.0f - c->p.xi;
    P[0] = 1.0f;
    for (int k = 1; k <= m; ++k) P[k] = P[k - 1] * f;

    cudaStream_t st = c->stream;
    ACS_TRY(cudaMemcpyAsync(c->d_xy, coords, sizeof(int32_t) * 2 * total_n, cudaMemcpyHostToDevice, st));
    ACS_TRY(cudaMemcpyAsync(c->d_desc, c->desc_h.data(), sizeof(InstDesc) * B, cudaMemcpyHostToDevice, st));
    ACS_TRY(cudaMemcpyAsync(c->d_order, order.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, st));
    ACS_TRY(cudaMemcpyAsync(c->d_P, P.data(), sizeof(float) * (m + 1), cudaMemcpyHostToDevice, st));
    std::vector<int64_t> big(B, INT64_MAX);
    ACS_TRY(cudaMemcpyAsync(c->d_best_len, big.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice, st));
    ACS_TRY(cudaMemsetAsync(c->d_iter, 0, sizeof(int64_t) * B, st));
    ACS_TRY(cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * 4 * B, st));
    ACS_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), st));

    dim3 kg((c->max_n + 7) / 8, B);
    knn_kernel<<<kg, 256, 0, st>>>(c->d_desc, c->d_xy, c->d_nn, c->d_w, c->p.beta);
    ACS_TRY(cudaGetLastError());
    const size_t vis_bytes = sizeof(uint32_t) * ((c->max_n + 31) / 32);
    nn_tour_kernel<<<B, 32, vis_bytes, st>>>(c->d_desc, c->d_xy, c->d_nn, c->d_Lnn);
    ACS_TRY(cudaGetLastError());
    dim3 ig(256, B);
    if (c->d_hw) {
        hw_kernel<<<dim3(1024, B), 256, 0, st>>>(c->d_desc, c->d_xy, c->d_hw, c->p.beta);
        ACS_TRY(cudaGetLastError());
    }
    if (c->p.memory == ACS_MEM_MATRIX) {
        init_matrix_kernel<<<ig, 256, 0, st>>>(c->d_desc, c->d_tau);
    } else {
        init_spm_kernel<<<ig, 256, 0, st>>>(c->d_desc, c->d_spm_idx, c->d_tau, c->d_spm_tail, c->s);
    }
    ACS_TRY(cudaGetLastError());
    ACS_TRY(cudaMemcpyAsync(c->desc_h.data(), c->d_desc, sizeof(InstDesc) * B, cudaMemcpyDeviceToHost, st));
    ACS_TRY(cudaStreamSynchronize(st));
    ACS_TRY(plan_launch(c));
    // plan_launch may have assigned global visited offsets
    ACS_TRY(cudaMemcpyAsync(c->d_desc, c->desc_h.data(), sizeof(InstDesc) * B, cudaMemcpyHostToDevice, st));
    ACS_TRY(cudaStreamSynchronize(st));
    return cudaSuccess;
}

acs_status check_device_status(acs_ctx* c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->poisoned = true;
        return ACS_ECUDA;
    }
    int32_t st = 0;
    e = cudaMemcpy(&st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || st != 0) {
        c->poisoned = true;
        return ACS_ECUDA;
    }
    return ACS_OK;
}

}  // namespace

// ------------------------------------------------------------------ for acs_prior.cu

namespace acs {

acs_status ctx_view(acs_ctx* c, int b, CtxView* v)
{
    if (!c || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    const InstDesc& D = c->desc_h[b];
    v->n = D.n;
    v->cl = D.cl;
    v->xy = c->d_xy + 2 * D.xy_off;
    v->nn = c->d_nn + 32 * D.row_off;
    v->w = c->d_w + 32 * D.row_off;
    v->best = c->d_best + D.node_off;
    v->stream = c->stream;
    v->has_best = c->has_best[b] != 0;
    return check_device_status(c);
}

// New effective candidate width of instance b (rows already rewritten on the
// context's stream). The descriptor copy is ordered on the same stream.
cudaError_t ctx_set_cl(acs_ctx* c, int b, int cl)
{
    c->desc_h[b].cl = cl;
    c->cl[b] = cl;
    cudaError_t e = cudaMemcpyAsync(c->d_desc + b, &c->desc_h[b], sizeof(InstDesc),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e;
}

void ctx_poison(acs_ctx* c) { c->poisoned = true; }

}  // namespace acs

// ------------------------------------------------------------------ C ABI

extern "C" {

acs_status acs_create_batch_ids(const int32_t* coords, const int64_t* offsets,
                                const int32_t* instance_ids, int32_t B, const acs_params* p,
                                acs_ctx** out)
{
    if (!out) return ACS_EINVAL;
    *out = nullptr;
    // B is a grid dimension of the set-up kernels (one grid row per instance)
    if (!coords || !offsets || B < 1 || B > 65535) return ACS_EINVAL;
    acs_status vs = validate_params(p);
    if (vs != ACS_OK) return vs;
    if (offsets[0] != 0) return ACS_EINVAL;
    int max_n = 0;
    for (int b = 0; b < B; ++b) {
        const int64_t n = offsets[b + 1] - offsets[b];
        if (n < 3 || n > kMaxN) return ACS_EINVAL;
        max_n = std::max<int>(max_n, (int)n);
    }
    const int64_t total = offsets[B];
    for (int64_t i = 0; i < 2 * total; ++i)
        if (coords[i] < 0 || coords[i] >= kCoordLimit) return ACS_EINVAL;
    if (instance_ids)
        for (int b = 0; b < B; ++b)
            if (instance_ids[b] < 0) return ACS_EINVAL;

    acs_ctx* c = new (std::nothrow) acs_ctx();
    if (!c) return ACS_ENOMEM;
    c->B = B;
    c->p = *p;
    c->m = p->m;
    c->s = p->memory == ACS_MEM_SPM ? p->spm_slots : 0;
    c->max_n = max_n;
    c->n.resize(B);
    c->cl.resize(B);
    c->has_best.assign(B, 0);
    c->ids.resize(B);
    for (int b = 0; b < B; ++b) c->ids[b] = instance_ids ? instance_ids[b] : b;
    for (int b = 0; b < B; ++b) {
        c->n[b] = (int32_t)(offsets[b + 1] - offsets[b]);
        c->cl[b] = std::min(p->cl, c->n[b] - 1);
    }
    cudaError_t e = build(c, coords, offsets);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        free_all(c);
        delete c;
        return oom ? ACS_ENOMEM : (e == cudaErrorInvalidConfiguration ? ACS_EINVAL : ACS_ECUDA);
    }
    *out = c;
    return ACS_OK;
}

acs_status acs_create_batch(const int32_t* coords, const int64_t* offsets, int32_t B,
                            const acs_params* p, acs_ctx** out)
{
    return acs_create_batch_ids(coords, offsets, nullptr, B, p, out);
}

acs_status acs_create(const int32_t* coords, int32_t n, const acs_params* p, acs_ctx** out)
{
    const int64_t off[2] = {0, (int64_t)n};
    return acs_create_batch(coords, off, 1, p, out);
}

acs_status acs_set_stream(acs_ctx* c, void* cuda_stream)
{
    if (!c) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
    if (s != c->stream) {
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
        c->stream = s;
        if (c->exec) cudaGraphExecDestroy(c->exec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->exec = nullptr;
        c->graph = nullptr;
    }
    return ACS_OK;
}

acs_status acs_run_iterations(acs_ctx* c, int32_t iters)
{
    if (!c || iters < 0) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    c->last_launches = 0;
    if (iters == 0) return ACS_OK;
    if (!c->exec) {
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail_cuda(c, e);
        cudaError_t le = (c->p.flags & ACS_FLAG_RELAXED)
                             ? launch_relaxed(c->args, c->B, (c->max_n + 31) / 32, c->stream)
                             : launch_construct(c->args, c->tpa, c->variant, c->grid, c->block,
                                                c->smem, c->csize, c->stream);
        e = cudaStreamEndCapture(c->stream, &c->graph);
        if (le != cudaSuccess) return fail_cuda(c, le);
        if (e != cudaSuccess) return fail_cuda(c, e);
        e = cudaGraphInstantiate(&c->exec, c->graph, 0);
        if (e != cudaSuccess) return fail_cuda(c, e);
    }
    for (int32_t i = 0; i < iters; ++i) {
        cudaError_t e = cudaGraphLaunch(c->exec, c->stream);
        if (e != cudaSuccess) return fail_cuda(c, e);
    }
    c->iteration += iters;
    std::fill(c->has_best.begin(), c->has_best.end(), (uint8_t)1);
    c->last_launches = (c->p.flags & ACS_FLAG_RELAXED) ? 2ll * iters : iters;
    return ACS_OK;
}

acs_status acs_set_threads_per_ant(acs_ctx* c, int32_t tpa)
{
    if (!c || (tpa != 4 && tpa != 8 && tpa != 16 && tpa != 32)) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
    cudaError_t e = configure(c, tpa, c->csize);
    if (e == cudaErrorInvalidConfiguration) {
        cudaGetLastError();
        return ACS_EINVAL;
    }
    return fail_cuda(c, e);
}

int32_t acs_threads_per_ant(const acs_ctx* c) { return c ? c->tpa : -1; }

acs_status acs_set_spm_resident(acs_ctx* c, int32_t resident)
{
    if (!c || (resident != 0 && resident != 1)) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
    const bool old = c->spm_resident;
    c->spm_resident = resident != 0;
    cudaError_t e = configure(c, c->tpa, c->csize);
    if (e == cudaErrorInvalidConfiguration) {
        cudaGetLastError();
        c->spm_resident = old;
        configure(c, c->tpa, c->csize);
        return ACS_EINVAL;
    }
    return fail_cuda(c, e);
}

acs_status acs_set_cluster_size(acs_ctx* c, int32_t csize)
{
    if (!c || (csize != 1 && csize != 2 && csize != 4 && csize != 8 && csize != 16)) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
    cudaError_t e = configure(c, c->tpa, csize);
    if (e == cudaErrorInvalidConfiguration) {
        cudaGetLastError();
        return ACS_EINVAL;
    }
    return fail_cuda(c, e);
}

int32_t acs_cluster_size(const acs_ctx* c) { return c ? c->csize : -1; }
int32_t acs_kernel_mode(const acs_ctx* c) { return c ? c->mode : -1; }

namespace {

// Every mutable array of a context, copied aside (on the context's stream)
// and put back after each autotuning trial, with the host-side loop state.
struct Snapshot {
    struct Buf { void* p; size_t bytes; void* save; };
    std::vector<Buf> bufs;
    int64_t iter0 = 0;
    std::vector<uint8_t> has_best0;
    bool taken = false;

    Snapshot() = default;
    Snapshot(const Snapshot&) = delete;
    Snapshot& operator=(const Snapshot&) = delete;
    ~Snapshot()
    {
        for (Buf& x : bufs) if (x.save) cudaFree(x.save);
    }

    acs_status take(acs_ctx* c)
    {
        size_t tau_n = 0, tour_n = 0, node_n = 0;
        for (int b = 0; b < c->B; ++b) {
            const size_t n = (size_t)c->n[b];
            tau_n += c->p.memory == ACS_MEM_MATRIX ? n * n : n * c->s;
            tour_n += (size_t)c->m * n;
            node_n += n;
        }
        bufs = {
            {c->d_tau, sizeof(float) * tau_n, nullptr},
            {c->d_tours, sizeof(int32_t) * tour_n, nullptr},
            {c->d_lens, sizeof(int64_t) * (size_t)c->B * c->m, nullptr},
            {c->d_best, sizeof(int32_t) * node_n, nullptr},
            {c->d_best_len, sizeof(int64_t) * c->B, nullptr},
            {c->d_iter, sizeof(int64_t) * c->B, nullptr},
            {c->d_stats, sizeof(unsigned long long) * 4 * c->B, nullptr},
        };
        if (c->p.memory == ACS_MEM_SPM) {
            bufs.push_back({c->d_spm_idx, sizeof(int32_t) * tau_n, nullptr});
            bufs.push_back({c->d_spm_tail, sizeof(int32_t) * node_n, nullptr});
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
        // All copies go on the context's stream, in order with the trials: a
        // device-to-device cudaMemcpy returns before the copy is done and runs
        // on the legacy stream, which does not order against this one.
        for (Buf& x : bufs) {
            if (cudaMalloc(&x.save, x.bytes) != cudaSuccess) {
                cudaGetLastError();
                x.save = nullptr;
                return ACS_ENOMEM;
            }
            if (cudaMemcpyAsync(x.save, x.p, x.bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                return fail_cuda(c, cudaErrorUnknown);
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
        iter0 = c->iteration;
        has_best0 = c->has_best;
        taken = true;
        return ACS_OK;
    }

    // puts the state back; nothing to do when take() did not complete (no
    // trial ran then)
    acs_status restore(acs_ctx* c)
    {
        if (!taken) return ACS_OK;
        for (Buf& x : bufs)
            if (cudaMemcpyAsync(x.p, x.save, x.bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                return fail_cuda(c, cudaErrorUnknown);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
        c->iteration = iter0;
        c->has_best = has_best0;
        c->last_launches = 0;
        return ACS_OK;
    }
};

struct Shape {
    int tpa, cs;
    bool res;
};

// Every launch shape the context can take: (threads per ant, cluster size)
// and, on the SPM, the global-memory record placement where it differs from
// the resident one. Leaves the context configured with the last one tried.
std::vector<Shape> launch_shapes(acs_ctx* c)
{
    static const int tpas[4] = {4, 8, 16, 32};
    static const int css[5] = {1, 2, 4, 8, 16};
    std::vector<Shape> out;
    const int nres = c->p.memory == ACS_MEM_SPM ? 2 : 1;
    for (int ri = 0; ri < nres; ++ri)
        for (int ci = 0; ci < 5; ++ci)
            for (int ti = 0; ti < 4; ++ti) {
                if (css[ci] > c->m) continue;
                c->spm_resident = ri == 0;
                if (configure(c, tpas[ti], css[ci]) != cudaSuccess) { cudaGetLastError(); continue; }
                if (ri == 1 && c->mode != 1) continue;   // nothing new to try
                out.push_back({tpas[ti], css[ci], ri == 0});
            }
    return out;
}

cudaError_t apply_shape(acs_ctx* c, const Shape& sh)
{
    c->spm_resident = sh.res;
    return configure(c, sh.tpa, sh.cs);
}

// One trial: every context starts together (the others' streams wait on the
// first's), runs one warm-up and then `iters` iterations; the group's time is
// the slowest context's, from the common start.
acs_status time_group(acs_ctx* const* cs, int k, int iters, float* ms_out)
{
    cudaEvent_t e0 = nullptr;
    std::vector<cudaEvent_t> ends((size_t)k, nullptr);
    acs_status st = ACS_OK;
    for (int i = 0; i < k && st == ACS_OK; ++i) st = acs_run_iterations(cs[i], 1);   // captures graphs
    for (int i = 0; i < k && st == ACS_OK; ++i)
        if (cudaStreamSynchronize(cs[i]->stream) != cudaSuccess) st = fail_cuda(cs[i], cudaErrorUnknown);
    if (st == ACS_OK && cudaEventCreate(&e0) != cudaSuccess) st = fail_cuda(cs[0], cudaErrorUnknown);
    for (int i = 0; i < k && st == ACS_OK; ++i)
        if (cudaEventCreate(&ends[i]) != cudaSuccess) st = fail_cuda(cs[i], cudaErrorUnknown);
    if (st == ACS_OK) {
        cudaEventRecord(e0, cs[0]->stream);
        for (int i = 1; i < k; ++i) cudaStreamWaitEvent(cs[i]->stream, e0, 0);
        for (int it = 0; it < iters && st == ACS_OK; ++it)
            for (int i = 0; i < k && st == ACS_OK; ++i) st = acs_run_iterations(cs[i], 1);
        float worst = 0.0f;
        for (int i = 0; i < k && st == ACS_OK; ++i) {
            cudaEventRecord(ends[i], cs[i]->stream);
            if (cudaEventSynchronize(ends[i]) != cudaSuccess) { st = fail_cuda(cs[i], cudaErrorUnknown); break; }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, ends[i]);
            worst = std::max(worst, ms);
        }
        *ms_out = worst;
    }
    if (e0) cudaEventDestroy(e0);
    for (cudaEvent_t e : ends) if (e) cudaEventDestroy(e);
    return st;
}

}  // namespace

namespace {

// Times every launch shape of the context alone (state restored after each
// trial), applies the fastest and returns each shape's time in `timed`.
acs_status tune_alone(acs_ctx* c, int32_t trial_iters, std::vector<std::pair<Shape, float>>* timed)
{
    Snapshot snap;
    acs_status st = snap.take(c);
    Shape best{c->tpa, c->csize, c->spm_resident};
    float best_ms = 0.0f;
    if (st == ACS_OK) {
        const std::vector<Shape> shapes = launch_shapes(c);
        for (const Shape& sh : shapes) {
            if (apply_shape(c, sh) != cudaSuccess) { cudaGetLastError(); continue; }
            float ms = 0.0f;
            st = time_group(&c, 1, trial_iters, &ms);
            if (st != ACS_OK) break;
            if (timed) timed->push_back({sh, ms});
            if (best_ms == 0.0f || ms < best_ms) {
                best_ms = ms;
                best = sh;
            }
            st = snap.restore(c);
            if (st != ACS_OK) break;
        }
    }
    if (st != ACS_OK) {
        snap.restore(c);
        return st;
    }
    if (apply_shape(c, best) != cudaSuccess) return fail_cuda(c, cudaErrorUnknown);
    return ACS_OK;
}

}  // namespace

acs_status acs_autotune(acs_ctx* c, int32_t trial_iters, int32_t* chosen_tpa,
                        int32_t* chosen_csize)
{
    if (!c || trial_iters < 1) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    if (c->p.flags & ACS_FLAG_RELAXED) {   // one launch shape only
        if (chosen_tpa) *chosen_tpa = 32;
        if (chosen_csize) *chosen_csize = 1;
        return ACS_OK;
    }
    const acs_status st = tune_alone(c, trial_iters, nullptr);
    if (st != ACS_OK) return st;
    if (chosen_tpa) *chosen_tpa = c->tpa;
    if (chosen_csize) *chosen_csize = c->csize;
    return ACS_OK;
}

acs_status acs_autotune_group(acs_ctx* const* ctxs, int32_t k, int32_t trial_iters)
{
    if (!ctxs || k < 1 || trial_iters < 1) return ACS_EINVAL;
    for (int i = 0; i < k; ++i) {
        if (!ctxs[i]) return ACS_EINVAL;
        for (int j = 0; j < i; ++j) if (ctxs[j] == ctxs[i]) return ACS_EINVAL;
    }
    for (int i = 0; i < k; ++i) if (ctxs[i]->poisoned) return ACS_ESTATE;
    // each context's own choice first; the joint passes then try only the
    // shapes that ran within twice the context's best time alone
    std::vector<std::vector<Shape>> shapes((size_t)k);
    for (int i = 0; i < k; ++i) {
        if (ctxs[i]->p.flags & ACS_FLAG_RELAXED) continue;   // one launch shape only
        std::vector<std::pair<Shape, float>> timed;
        const acs_status st = tune_alone(ctxs[i], trial_iters, &timed);
        if (st != ACS_OK) return st;
        float best = 0.0f;
        for (const auto& t : timed) best = best == 0.0f ? t.second : std::min(best, t.second);
        for (const auto& t : timed)
            if (t.second <= 2.0f * best) shapes[i].push_back(t.first);
    }
    if (k == 1) return ACS_OK;
    std::vector<Snapshot> snaps((size_t)k);
    std::vector<Shape> cur((size_t)k);
    acs_status st = ACS_OK;
    for (int i = 0; i < k && st == ACS_OK; ++i) {
        acs_ctx* c = ctxs[i];
        cur[i] = {c->tpa, c->csize, c->spm_resident};
        st = snaps[i].take(c);
    }
    auto restore_all = [&]() -> acs_status {
        for (int i = 0; i < k; ++i) {
            const acs_status r = snaps[i].restore(ctxs[i]);
            if (r != ACS_OK) return r;
        }
        return ACS_OK;
    };
    // Coordinate descent (one context's shape at a time, the others fixed,
    // every trial timed with the whole group running; two passes at most)
    // from two starts: the shapes best alone, and each context's smallest
    // shape (fewest lanes x CTAs per instance, records in global memory
    // first), which leaves room on the SMs for the others. The better end
    // point is kept.
    auto apply_all = [&](const std::vector<Shape>& sh) -> acs_status {
        for (int i = 0; i < k; ++i) {
            if (ctxs[i]->p.flags & ACS_FLAG_RELAXED) continue;
            if (apply_shape(ctxs[i], sh[i]) != cudaSuccess) return fail_cuda(ctxs[i], cudaErrorUnknown);
        }
        return ACS_OK;
    };
    auto descend = [&](std::vector<Shape>& at, float* ms_out) -> acs_status {
        acs_status r = apply_all(at);
        float best_ms = 0.0f;
        if (r == ACS_OK) r = time_group(ctxs, k, trial_iters, &best_ms);
        if (r == ACS_OK) r = restore_all();
        for (int pass = 0; pass < 2 && r == ACS_OK; ++pass) {
            bool improved = false;
            for (int i = 0; i < k && r == ACS_OK; ++i) {
                for (const Shape& sh : shapes[i]) {
                    if (sh.tpa == at[i].tpa && sh.cs == at[i].cs && sh.res == at[i].res) continue;
                    if (apply_shape(ctxs[i], sh) != cudaSuccess) { cudaGetLastError(); continue; }
                    float ms = 0.0f;
                    r = time_group(ctxs, k, trial_iters, &ms);
                    if (r == ACS_OK) r = restore_all();
                    if (r != ACS_OK) break;
                    if (ms < 0.99f * best_ms) {   // 1 %: beyond the trial-to-trial noise
                        best_ms = ms;
                        at[i] = sh;
                        improved = true;
                    }
                }
                if (r == ACS_OK && !(ctxs[i]->p.flags & ACS_FLAG_RELAXED) &&
                    apply_shape(ctxs[i], at[i]) != cudaSuccess)
                    r = fail_cuda(ctxs[i], cudaErrorUnknown);
            }
            if (!improved) break;
        }
        *ms_out = best_ms;
        return r;
    };
    std::vector<Shape> small = cur;
    for (int i = 0; i < k; ++i) {
        for (const Shape& sh : shapes[i]) {
            const Shape& b = small[i];
            const int fs = sh.tpa * sh.cs, fb = b.tpa * b.cs;
            if (fs < fb || (fs == fb && !sh.res && b.res)) small[i] = sh;
        }
    }
    float ms_a = 0.0f, ms_b = 0.0f;
    std::vector<Shape> end_a = cur, end_b = small;
    if (st == ACS_OK) st = descend(end_a, &ms_a);
    bool same_start = true;
    for (int i = 0; i < k; ++i)
        same_start &= small[i].tpa == cur[i].tpa && small[i].cs == cur[i].cs && small[i].res == cur[i].res;
    if (st == ACS_OK && !same_start) st = descend(end_b, &ms_b);
    if (st == ACS_OK) st = apply_all(!same_start && ms_b < ms_a ? end_b : end_a);
    if (st != ACS_OK) {
        restore_all();
        return st;
    }
    return ACS_OK;
}

acs_status acs_offer_best_tour(acs_ctx* c, int32_t b, const int32_t* tour, int64_t* len_out)
{
    if (!c || !tour || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    const InstDesc& D = c->desc_h[b];
    const int n = D.n;
    std::vector<uint8_t> seen((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        if (tour[i] < 0 || tour[i] >= n || seen[tour[i]]) return ACS_EINVAL;
        seen[tour[i]] = 1;
    }
    acs_status s = check_device_status(c);
    if (s != ACS_OK) return s;
    // scratch: the tour and the offered length, stream-ordered
    void* scratch = nullptr;
    const size_t bytes = sizeof(int64_t) + sizeof(int32_t) * (size_t)n;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, c->stream);
    if (e != cudaSuccess) { cudaGetLastError(); return ACS_ENOMEM; }
    int64_t* d_len = static_cast<int64_t*>(scratch);
    int32_t* d_tour = reinterpret_cast<int32_t*>(d_len + 1);
    e = cudaMemcpyAsync(d_tour, tour, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        offer_best_kernel<<<1, 1024, 0, c->stream>>>(c->d_desc, b, c->d_xy, d_tour, c->d_best,
                                                     c->d_best_len, d_len);
        e = cudaGetLastError();
    }
    int64_t L = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&L, d_len, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(scratch, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e);
    if (len_out) *len_out = L;
    return ACS_OK;
}

acs_status acs_best_tour(acs_ctx* c, int32_t b, int32_t* tour_out, int64_t* len_out)
{
    if (!c || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    acs_status s = check_device_status(c);
    if (s != ACS_OK) return s;
    if (!c->has_best[b]) return ACS_ESTATE;
    const InstDesc& D = c->desc_h[b];
    cudaError_t e = cudaSuccess;
    if (tour_out) e = cudaMemcpy(tour_out, c->d_best + D.node_off, sizeof(int32_t) * D.n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && len_out) e = cudaMemcpy(len_out, c->d_best_len + b, sizeof(int64_t), cudaMemcpyDeviceToHost);
    return fail_cuda(c, e);
}

acs_status acs_get_tours(acs_ctx* c, int32_t b, int32_t* tours, int64_t* lens)
{
    if (!c || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    acs_status s = check_device_status(c);
    if (s != ACS_OK) return s;
    const InstDesc& D = c->desc_h[b];
    cudaError_t e = cudaSuccess;
    if (tours) e = cudaMemcpy(tours, c->d_tours + D.tour_off, sizeof(int32_t) * (size_t)c->m * D.n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && lens) e = cudaMemcpy(lens, c->d_lens + D.ant_off, sizeof(int64_t) * c->m, cudaMemcpyDeviceToHost);
    return fail_cuda(c, e);
}

acs_status acs_get_pheromone(acs_ctx* c, int32_t b, float* tau_or_val, int32_t* spm_idx, int32_t* spm_tail)
{
    if (!c || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    acs_status s = check_device_status(c);
    if (s != ACS_OK) return s;
    const InstDesc& D = c->desc_h[b];
    cudaError_t e = cudaSuccess;
    if (c->p.memory == ACS_MEM_MATRIX) {
        if (tau_or_val) e = cudaMemcpy(tau_or_val, c->d_tau + D.tau_off, sizeof(float) * (size_t)D.n * D.n, cudaMemcpyDeviceToHost);
    } else {
        const size_t ns = (size_t)D.n * c->s;
        if (tau_or_val) e = cudaMemcpy(tau_or_val, c->d_tau + D.tau_off, sizeof(float) * ns, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && spm_idx) e = cudaMemcpy(spm_idx, c->d_spm_idx + D.tau_off, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && spm_tail) e = cudaMemcpy(spm_tail, c->d_spm_tail + D.node_off, sizeof(int32_t) * D.n, cudaMemcpyDeviceToHost);
    }
    return fail_cuda(c, e);
}

acs_status acs_get_setup(acs_ctx* c, int32_t b, int32_t* nn, float* w, float* tau0, int64_t* L_nn, int32_t* cl_eff)
{
    if (!c || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    acs_status s = check_device_status(c);
    if (s != ACS_OK) return s;
    const InstDesc& D = c->desc_h[b];
    cudaError_t e = cudaSuccess;
    if (nn || w) {
        std::vector<int32_t> nb(32 * (size_t)D.n);
        std::vector<float> wb(32 * (size_t)D.n);
        e = cudaMemcpy(nb.data(), c->d_nn + 32 * D.row_off, sizeof(int32_t) * nb.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(wb.data(), c->d_w + 32 * D.row_off, sizeof(float) * wb.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(c, e);
        for (int i = 0; i < D.n; ++i)
            for (int k = 0; k < D.cl; ++k) {
                if (nn) nn[(size_t)i * D.cl + k] = nb[(size_t)i * 32 + k];
                if (w) w[(size_t)i * D.cl + k] = wb[(size_t)i * 32 + k];
            }
    }
    if (tau0) *tau0 = D.tau0;
    if (L_nn) e = cudaMemcpy(L_nn, c->d_Lnn + b, sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (cl_eff) *cl_eff = D.cl;
    return fail_cuda(c, e);
}

acs_status acs_get_stats(acs_ctx* c, int32_t b, int64_t out[4])
{
    if (!c || !out || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    acs_status s = check_device_status(c);
    if (s != ACS_OK) return s;
    unsigned long long v[4];
    cudaError_t e = cudaMemcpy(v, c->d_stats + 4 * (size_t)b, sizeof(v), cudaMemcpyDeviceToHost);
    for (int i = 0; i < 4; ++i) out[i] = (int64_t)v[i];
    return fail_cuda(c, e);
}

// ---- checkpoint / resume of one instance's loop state (Alg. 1)

namespace {

struct StateHeader {
    uint32_t magic;       // kStateMagic
    uint32_t version;     // kStateVersion
    acs_params p;         // the parameters of the context that wrote it
    int32_t n, cl;        // nodes, effective candidate width
    int32_t has_best, pad;
    int64_t iteration;    // Philox counter word 0 of the next iteration
    int64_t best_len;     // INT64_MAX when there is no best-so-far tour
    uint32_t tau0_bits;   // tau0 of the instance (identifies its coordinates)
    uint32_t pad2;
    int64_t stats[4];     // fallbacks, selections, SPM hits, SPM misses
};
static_assert(sizeof(StateHeader) == 128, "state header layout");
constexpr uint32_t kStateMagic = 0x53534341u;   // "ACSS"
constexpr uint32_t kStateVersion = 1;

size_t state_bytes(const acs_ctx* c, int b)
{
    const size_t n = (size_t)c->n[b];
    size_t bytes = sizeof(StateHeader) + 2 * 32 * 4 * n + 4 * n;   // rows, best tour
    if (c->p.memory == ACS_MEM_MATRIX) bytes += 4 * n * n;
    else bytes += 8 * n * c->s + 4 * n;
    return bytes;
}

bool same_params_but_seed(const acs_params& a, const acs_params& b)
{
    return a.m == b.m && a.cl == b.cl && a.beta == b.beta && a.q0 == b.q0 && a.rho == b.rho &&
           a.xi == b.xi && a.memory == b.memory && a.spm_slots == b.spm_slots &&
           a.local_period == b.local_period && a.flags == b.flags;
}

}  // namespace

acs_status acs_state_size(const acs_ctx* c, int32_t b, int64_t* bytes)
{
    if (!c || !bytes || b < 0 || b >= c->B) return ACS_EINVAL;
    *bytes = (int64_t)state_bytes(c, b);
    return ACS_OK;
}

acs_status acs_get_state(acs_ctx* c, int32_t b, void* buf, int64_t bytes)
{
    if (!c || !buf || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    if (bytes < (int64_t)state_bytes(c, b)) return ACS_EINVAL;
    acs_status st = check_device_status(c);
    if (st != ACS_OK) return st;
    const InstDesc& D = c->desc_h[b];
    const size_t n = (size_t)D.n;
    unsigned char* out = static_cast<unsigned char*>(buf);
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kStateMagic;
    h.version = kStateVersion;
    h.p = c->p;
    h.n = D.n;
    h.cl = D.cl;
    h.has_best = c->has_best[b];
    std::memcpy(&h.tau0_bits, &D.tau0, 4);
    unsigned long long stats[4];
    cudaError_t e = cudaMemcpy(&h.iteration, c->d_iter + b, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h.best_len, c->d_best_len + b, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(stats, c->d_stats + 4 * (size_t)b, sizeof(stats), cudaMemcpyDeviceToHost);
    for (int i = 0; i < 4; ++i) h.stats[i] = (int64_t)stats[i];
    size_t o = sizeof(StateHeader);
    if (e == cudaSuccess) e = cudaMemcpy(out + o, c->d_nn + 32 * D.row_off, 128 * n, cudaMemcpyDeviceToHost);
    o += 128 * n;
    if (e == cudaSuccess) e = cudaMemcpy(out + o, c->d_w + 32 * D.row_off, 128 * n, cudaMemcpyDeviceToHost);
    o += 128 * n;
    if (e == cudaSuccess) e = cudaMemcpy(out + o, c->d_best + D.node_off, 4 * n, cudaMemcpyDeviceToHost);
    o += 4 * n;
    if (c->p.memory == ACS_MEM_MATRIX) {
        if (e == cudaSuccess) e = cudaMemcpy(out + o, c->d_tau + D.tau_off, 4 * n * n, cudaMemcpyDeviceToHost);
    } else {
        const size_t ns = n * c->s;
        if (e == cudaSuccess) e = cudaMemcpy(out + o, c->d_spm_idx + D.tau_off, 4 * ns, cudaMemcpyDeviceToHost);
        o += 4 * ns;
        if (e == cudaSuccess) e = cudaMemcpy(out + o, c->d_tau + D.tau_off, 4 * ns, cudaMemcpyDeviceToHost);
        o += 4 * ns;
        if (e == cudaSuccess) e = cudaMemcpy(out + o, c->d_spm_tail + D.node_off, 4 * n, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return fail_cuda(c, e);
    std::memcpy(out, &h, sizeof(h));
    return ACS_OK;
}

acs_status acs_set_state(acs_ctx* c, int32_t b, const void* buf, int64_t bytes)
{
    if (!c || !buf || b < 0 || b >= c->B) return ACS_EINVAL;
    if (c->poisoned) return ACS_ESTATE;
    if (bytes < (int64_t)sizeof(StateHeader)) return ACS_EINVAL;
    const unsigned char* in = static_cast<const unsigned char*>(buf);
    StateHeader h;
    std::memcpy(&h, in, sizeof(h));
    const InstDesc& D = c->desc_h[b];
    const int n = D.n;
    if (h.magic != kStateMagic || h.version != kStateVersion) return ACS_EINVAL;
    if (h.n != n || !same_params_but_seed(h.p, c->p)) return ACS_EINVAL;
    if (bytes < (int64_t)state_bytes(c, b)) return ACS_EINVAL;
    uint32_t tb;
    std::memcpy(&tb, &D.tau0, 4);
    if (h.tau0_bits != tb) return ACS_EINVAL;   // other coordinates
    if (h.cl < 1 || h.cl > std::min(kMaxCl, n - 1) || h.iteration < 0 || h.iteration > INT32_MAX)
        return ACS_EINVAL;
    if (h.has_best != 0 && h.has_best != 1) return ACS_EINVAL;
    // host-side validation of every array before any device write
    size_t o = sizeof(StateHeader);
    const int32_t* nn = reinterpret_cast<const int32_t*>(in + o);
    o += 128 * (size_t)n;
    const float* w = reinterpret_cast<const float*>(in + o);
    o += 128 * (size_t)n;
    const int32_t* best = reinterpret_cast<const int32_t*>(in + o);
    o += 4 * (size_t)n;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 32; ++k) {
            int32_t j;
            float x;
            std::memcpy(&j, nn + 32 * (size_t)i + k, 4);
            std::memcpy(&x, w + 32 * (size_t)i + k, 4);
            if (k < h.cl ? (j < 0 || j >= n || j == i || !(x >= 0.0f)) : j != -1) return ACS_EINVAL;
        }
    if (h.has_best) {
        std::vector<uint8_t> seen((size_t)n, 0);
        for (int i = 0; i < n; ++i) {
            int32_t t;
            std::memcpy(&t, best + i, 4);
            if (t < 0 || t >= n || seen[t]) return ACS_EINVAL;
            seen[t] = 1;
        }
        if (h.best_len <= 0 || h.best_len == INT64_MAX) return ACS_EINVAL;
    } else if (h.best_len != INT64_MAX) {
        return ACS_EINVAL;
    }
    if (c->p.memory == ACS_MEM_SPM) {
        const size_t ns = (size_t)n * c->s;
        const unsigned char* p = in + o;
        for (size_t i = 0; i < ns; ++i) {
            int32_t j;
            std::memcpy(&j, p + 4 * i, 4);
            if (j < -1 || j >= n) return ACS_EINVAL;
        }
        for (int i = 0; i < n; ++i) {
            int32_t t;
            std::memcpy(&t, p + 8 * ns + 4 * (size_t)i, 4);
            if (t < 0 || t >= c->s) return ACS_EINVAL;
        }
    }
    acs_status st = check_device_status(c);
    if (st != ACS_OK) return st;
    cudaStream_t s = c->stream;
    unsigned long long stats[4];
    for (int i = 0; i < 4; ++i) stats[i] = (unsigned long long)h.stats[i];
    o = sizeof(StateHeader);
    cudaError_t e = cudaMemcpyAsync(c->d_nn + 32 * D.row_off, in + o, 128 * (size_t)n, cudaMemcpyHostToDevice, s);
    o += 128 * (size_t)n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_w + 32 * D.row_off, in + o, 128 * (size_t)n, cudaMemcpyHostToDevice, s);
    o += 128 * (size_t)n;
    if (e == cudaSuccess && h.has_best)
        e = cudaMemcpyAsync(c->d_best + D.node_off, in + o, 4 * (size_t)n, cudaMemcpyHostToDevice, s);
    o += 4 * (size_t)n;
    if (c->p.memory == ACS_MEM_MATRIX) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_tau + D.tau_off, in + o, 4 * (size_t)n * n, cudaMemcpyHostToDevice, s);
    } else {
        const size_t ns = (size_t)n * c->s;
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_spm_idx + D.tau_off, in + o, 4 * ns, cudaMemcpyHostToDevice, s);
        o += 4 * ns;
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_tau + D.tau_off, in + o, 4 * ns, cudaMemcpyHostToDevice, s);
        o += 4 * ns;
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_spm_tail + D.node_off, in + o, 4 * (size_t)n, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_iter + b, &h.iteration, 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_best_len + b, &h.best_len, 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_stats + 4 * (size_t)b, stats, sizeof(stats), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(c, e);
    if (h.cl != D.cl) {
        e = ctx_set_cl(c, b, h.cl);
        if (e != cudaSuccess) return fail_cuda(c, e);
    }
    c->has_best[b] = (uint8_t)h.has_best;
    if (b == 0) c->iteration = h.iteration;
    return ACS_OK;
}

int64_t acs_iteration(const acs_ctx* c) { return c ? c->iteration : -1; }
int32_t acs_num_instances(const acs_ctx* c) { return c ? c->B : -1; }
int32_t acs_instance_size(const acs_ctx* c, int32_t b)
{
    return (c && b >= 0 && b < c->B) ? c->n[b] : -1;
}
int64_t acs_last_launch_count(const acs_ctx* c) { return c ? c->last_launches : -1; }

const char* acs_strerror(acs_status s)
{
    switch (s) {
    case ACS_OK: return "ok";
    case ACS_EINVAL: return "invalid argument";
    case ACS_ENOMEM: return "out of memory";
    case ACS_ECUDA: return "CUDA error or failed device check";
    case ACS_ETIMEOUT: return "bounded device wait timed out";
    case ACS_ESTATE: return "context poisoned or no result yet";
    }
    return "unknown status";
}

void acs_destroy(acs_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
