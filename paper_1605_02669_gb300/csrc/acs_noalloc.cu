// acs_noalloc.cu -- acs_iterate_noalloc: one colony iteration on caller-owned
// device buffers that never allocates device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool
// or arena it does not own (an inference server that pre-reserves all device
// memory at start-up, a framework whose caching allocator must see every
// allocation), or code that must not allocate on its hot path. For them the
// per-iteration scratch of the construct kernel -- the visited bitmasks of
// all ants, the decay table P[k], the instance descriptor and the internal
// counters -- lives in one static device array of fixed size, kScratchBytes,
// that every GPU which loads this library keeps until the process exits.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "acs.h"
#include "acs_internal.cuh"

namespace acs {
cudaError_t prepare_construct(int tpa, int mode, size_t smem);
cudaError_t launch_construct(const ConstructArgs& A, int tpa, int mode, int grid, int block,
                             size_t smem, int csize, cudaStream_t stream);
}  // namespace acs

using namespace acs;

namespace {

constexpr size_t kScratchBytes = 4u << 20;   // 4 MiB per device
constexpr size_t kHeaderBytes = 256;         // descriptor, order, status, iteration, counters
constexpr size_t kTableBytes = 8192;         // decay table P[0..m], m <= 1024
constexpr size_t kVisOffset = kHeaderBytes + kTableBytes;
constexpr size_t kMaxVisWords = (kScratchBytes - kVisOffset) / 4;
constexpr int kMaxDevices = 64;

// The shared scratch. In host code this name is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Header {
    InstDesc desc;
    int32_t order;
    int32_t status;
    int64_t iteration;
    unsigned long long stats[4];
};
static_assert(sizeof(Header) <= kHeaderBytes, "scratch header too large");

std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Once per device, with that device current: look up the array's device address.
cudaError_t scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" acs_status acs_iterate_noalloc(const int32_t* dev_coords, int32_t n,
                                          const int32_t* dev_nn32, const float* dev_w32,
                                          int32_t cl, float tau0, float* dev_tau,
                                          int32_t* dev_tours, int64_t* dev_lens,
                                          int32_t* dev_best, int64_t* dev_best_len,
                                          int64_t iteration, const acs_params* p, void* stream)
{
    if (!p || !dev_coords || !dev_nn32 || !dev_w32 || !dev_tau || !dev_tours || !dev_lens ||
        !dev_best || !dev_best_len)
        return ACS_EINVAL;
    if (n < 3 || n > kMaxN || cl < 1 || cl > kMaxCl || cl > n - 1 || iteration < 0)
        return ACS_EINVAL;
    if (p->m < 1 || p->m > kMaxM || p->beta < 0 || p->beta > 8) return ACS_EINVAL;
    if (!(p->q0 >= 0.0f && p->q0 <= 1.0f) || !(p->rho > 0.0f && p->rho < 1.0f) ||
        !(p->xi > 0.0f && p->xi < 1.0f))
        return ACS_EINVAL;
    if (p->memory != ACS_MEM_MATRIX || p->local_period < 1 || p->flags != 0) return ACS_EINVAL;
    if (!(tau0 > 0.0f)) return ACS_EINVAL;
    const int m = p->m;
    const int W = (n + 31) / 32;
    if ((size_t)m * (size_t)W > kMaxVisWords) return ACS_EINVAL;  // scratch too small
    if (4u * ((size_t)m + 1) > kTableBytes) return ACS_EINVAL;

    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return ACS_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;

    Header h;
    std::memset(&h, 0, sizeof(h));
    h.desc.n = n;
    h.desc.cl = cl;
    h.desc.W = W;
    h.desc.instance = 0;
    h.desc.tau0 = tau0;
    h.order = 0;
    h.status = 0;
    h.iteration = iteration;
    std::vector<float> P(m + 1);
    const float f = 1.0f - p->xi;
    P[0] = 1.0f;
    for (int k = 1; k <= m; ++k) P[k] = P[k - 1] * f;

    // the kernel zeroes the visited words itself; the header (status and
    // counters included) and the table are rewritten on every call
    e = cudaMemcpyAsync(base, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kHeaderBytes, P.data(), sizeof(float) * (m + 1),
                            cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return ACS_ECUDA;

    Header* dh = reinterpret_cast<Header*>(base);
    ConstructArgs A{};
    A.desc = &dh->desc;
    A.order = &dh->order;
    A.num_inst = 1;
    A.m = m;
    A.xy = dev_coords;
    A.nn = dev_nn32;
    A.w = dev_w32;
    A.tau = dev_tau;
    A.spm_idx = nullptr;
    A.spm_tail = nullptr;
    A.tours = dev_tours;
    A.lens = dev_lens;
    A.best = dev_best;
    A.best_len = dev_best_len;
    A.iteration = &dh->iteration;
    A.stats = dh->stats;
    A.vis_global = reinterpret_cast<uint32_t*>(base + kVisOffset);
    A.P = reinterpret_cast<const float*>(base + kHeaderBytes);
    A.status = &dh->status;
    A.q0 = p->q0;
    A.rho = p->rho;
    A.beta = p->beta;
    A.s = 0;
    A.period = p->local_period;
    A.skip_default = 0;
    A.key0 = (uint32_t)(p->seed & 0xffffffffull);
    A.key1 = (uint32_t)(p->seed >> 32);
    A.vis_in_smem = 0;
    A.xy_in_smem = 0;
    A.max_n = n;
    A.mc = m;
    A.nrec = 0;
    const SmemLayout L = smem_layout(m, m, 0, 0, W, n, false, false);
    const int tpa = 8;
    int block = m * tpa < 64 ? 64 : (m * tpa > 1024 ? 1024 : m * tpa);
    block = (block + 31) / 32 * 32;
    if (block < m) block = (m + 31) / 32 * 32;
    e = prepare_construct(tpa, 0, L.total);
    if (e != cudaSuccess) return ACS_ECUDA;
    e = launch_construct(A, tpa, 0, 1, block, L.total, 1, st);
    if (e != cudaSuccess) return ACS_ECUDA;

    int32_t status = 0;
    e = cudaMemcpyAsync(&status, &dh->status, sizeof(status), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ACS_ECUDA;
    return status == 0 ? ACS_OK : ACS_ECUDA;
}
