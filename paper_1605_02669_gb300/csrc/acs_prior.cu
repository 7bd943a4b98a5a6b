// acs_prior.cu -- the learned edge prior: features, labels, the BF16
// tensor-core MLP (forward, fused forward+backward, Adam) and the pruning /
// reweighting of the candidate rows. See include/acs_prior.h.
//
// Both the scoring forward pass (acs_mlp_forward) and the fused forward +
// backward of training (acs_mlp_train_batch) run on the 5th-generation tensor
// cores (tcgen05): BF16 operands in shared memory, FP32 accumulators in
// tensor memory; their layouts are described above mlp_forward_tc_kernel and
// mlp_train_kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <new>

#include "acs.h"
#include "acs_device.cuh"
#include "acs_internal.cuh"
#include "acs_prior.h"

namespace acs {
acs_status ctx_view(acs_ctx* c, int b, CtxView* v);
cudaError_t ctx_set_cl(acs_ctx* c, int b, int cl);
void ctx_poison(acs_ctx* c);
}  // namespace acs

using namespace acs;

namespace {

constexpr int kW1 = 0, kB1 = 512, kW2 = 576, kB2 = 4672, kW3 = 4736, kB3 = 4800;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

// mean-BCE term of one row: max(z,0) - z y + log(1 + exp(-|z|))
__device__ __forceinline__ float bce_term(float z, float y)
{
    return fmaxf(z, 0.0f) - z * y + log1pf(expf(-fabsf(z)));
}

// ---------------------------------------------------------------------------
// Scoring forward pass on the 5th-generation tensor cores (tcgen05).
//
// A CTA holds G groups of four warps (G <= 8) that share the weights in
// shared memory; each group scores 128 feature rows per tile (row t of the
// tile is the group's thread t and TMEM lane t) and walks its own sequence
// of tiles, so G tile chains are in flight per CTA. The operands sit in
// shared memory in the canonical K-major layout without swizzle: 8 x 8 BF16
// core matrices of 128 contiguous bytes (8 rows of 16 B), K-adjacent core
// matrices 128 B apart (leading byte offset) and 8-row groups (K/8) x 128 B
// apart (stride byte offset). One thread of the group issues
//   layer 1: D[128 x 64] = [X | 1 1 1 0..][128 x 16] [W1 ; b1 split][16 x 64]
//   layer 2: D[128 x 64] = [H1 | 1 1 1 0..][128 x 80] [W2 ; b2 split][80 x 64]
// (one MMA, then five of K = 16) into the group's 64 FP32 TMEM columns, and
// commits each layer to the group's mbarrier. The biases ride in the K
// padding: each FP32 bias is split exactly into three BF16 parts that meet
// three constant-one columns, so the accumulator adds the bias in FP32. The
// epilogues read the accumulator back with tcgen05.ld (each warp its 32
// lanes): layer 1 rounds to BF16, applies ReLU and writes H1 into shared
// memory as the A operand of layer 2; layer 2 applies ReLU and takes the dot
// product with w3 in FP32 (N = 1 stays on the CUDA cores). Rounding points
// as in the training kernel: BF16 operands, FP32 accumulation, h2 in FP32.

constexpr int kTcRows = 128;
constexpr int kTcMaxGroups = 8;
constexpr int kK1 = 16, kK2 = 80;   // K of layer 1 (8 features, 3 bias columns) and layer 2 (64 + 3)
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;   // bound of one MMA-completion wait
// After a wait gave up, the bound of the wait for the MMA that was already
// issued: tensor memory is freed only once it has signalled completion.
constexpr unsigned long long kDrainNs = 2000ull * 1000 * 1000;

// Wait bounds handed to the tensor-core kernels. ns: bound of one wait.
// phantom != 0 (set only through the test hook acs_mlp_test_wait_hook) makes
// the first wait of every tile poll a second mbarrier that nothing arrives
// on, so the bound is reached while the real MMA still commits to its own
// barrier, which the failure path then drains.
struct TcWait {
    unsigned long long ns;
    int phantom;
};

// Status word of the tensor-core kernels on this device: 0, or ACS_ETIMEOUT
// once a bounded wait has given up (never cleared: the scores or gradients of
// that launch are incomplete, and the host refuses later tensor-core work).
__device__ int32_t g_tc_status;
// Set by apply_prior_kernel when a score is not a probability.
__device__ int32_t g_bad_score;
// instruction descriptor (kind::f16): D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28
constexpr uint32_t kIdescM128N64 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

struct TcWeights {
    uint16_t w1[64 * kK1];   // layer-1 B = [W1 ; b1]^T: 8 row groups (outputs) x 2 K groups
    uint16_t w2[64 * kK2];   // layer-2 B = [W2 ; b2]^T: 8 x 10
    float w3[64];
    float b3;
    uint32_t tmem;           // TMEM base address written by tcgen05.alloc
};
struct TcGroup {
    uint16_t x[kTcRows * kK1];    // layer-1 A: 16 row groups x 2 K groups
    uint16_t h1[kTcRows * kK2];   // layer-2 A: 16 row groups x 10 K groups
    unsigned long long bar;       // MMA completion barrier
    unsigned long long phantom;   // never arrived on (test hook of the bounded wait)
};
constexpr size_t kTcWeightBytes = (sizeof(TcWeights) + 127) & ~size_t(127);
constexpr size_t kTcGroupBytes = (sizeof(TcGroup) + 127) & ~size_t(127);
constexpr size_t tc_smem(int groups) { return kTcWeightBytes + groups * kTcGroupBytes; }
static_assert(tc_smem(kTcMaxGroups) <= 227 * 1024, "scoring CTA does not fit");
static_assert(offsetof(TcWeights, w2) % 128 == 0 && offsetof(TcGroup, h1) % 128 == 0,
              "operand tiles must start on core-matrix boundaries");

// TMEM columns of a CTA of G groups (64 each, a power of two >= 32). With
// the shared memory of tc_smem(G) at most 512 columns are held per SM:
// G = 1: 6 CTAs x 64; G = 2: 3 x 128; G = 3, 4: 2 x 256; G >= 5: 1 x 512.
constexpr uint32_t tc_tmem_cols(int groups)
{
    return groups <= 1 ? 64u : groups <= 2 ? 128u : groups <= 4 ? 256u : 512u;
}

// element index of (row r, column k) in a K-major no-swizzle tile with kg K groups
__device__ __forceinline__ int core_idx(int r, int k, int kg)
{
    return (((r >> 3) * kg + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (bits 16-29; the distance between K-adjacent core
// matrices, 128 B when they are packed), stride byte offset >> 4 (bits 32-45;
// between 8-row groups), descriptor version 1 (bits 46-48), base offset 0,
// no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t sbo, uint32_t lbo = 128u)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 :
                 : "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// generic-proxy writes to shared memory -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// the 128 threads of one group meet at named barrier `id` (1..8)
__device__ __forceinline__ void group_sync(int id)
{
    asm volatile("bar.sync %0, 128;\n" ::"r"(id) : "memory");
}
__device__ __forceinline__ bool group_sync_or(int id, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id)
        : "memory");
    return r != 0u;
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Waits for the completion of phase `parity` of the barrier; gives up after
// `ns` of wall time (%globaltimer) and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long ns)
{
    unsigned long long t0 = 0ull;
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        if (t0 == 0ull) t0 = now;
        else if (now - t0 > ns) return false;
    }
}

__device__ __forceinline__ uint4 load_feat(const uint16_t* feat, int64_t row, int64_t rows)
{
    return row < rows ? __ldg(reinterpret_cast<const uint4*>(feat) + row) : make_uint4(0u, 0u, 0u, 0u);
}

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bf16_value(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// One 16-byte core-matrix row holding the three BF16 parts of an FP32 bias
// (hi + mid + lo == b exactly: each part takes the next 8 significant bits)
// followed by zeros; with `ones` the row of constant-one columns instead.
__device__ __forceinline__ uint4 bias_row(float b, bool ones)
{
    if (ones) return make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u);
    const uint16_t hi = bf16_bits(b);
    const float r1 = b - bf16_value(hi);
    const uint16_t mid = bf16_bits(r1);
    const uint16_t lo = bf16_bits(r1 - bf16_value(mid));
    return make_uint4((uint32_t)hi | ((uint32_t)mid << 16), (uint32_t)lo, 0u, 0u);
}

__global__ void __launch_bounds__(kTcRows * kTcMaxGroups, 1)
mlp_forward_tc_kernel(const float* P, const uint16_t* feat, int64_t rows, float* pout, uint32_t tmem_cols,
                      TcWait wt)
{
    extern __shared__ __align__(128) unsigned char tsm[];
    TcWeights& W = *reinterpret_cast<TcWeights*>(tsm);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid >> 7, t = tid & (kTcRows - 1);   // group, row of the group's tile
    const int groups = blockDim.x >> 7;
    TcGroup& G = *reinterpret_cast<TcGroup*>(tsm + kTcWeightBytes + g * kTcGroupBytes);
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;
    const int64_t gstride = (int64_t)gridDim.x * groups;
    int64_t tile = (int64_t)blockIdx.x * groups + g;
    uint4 xv = load_feat(feat, tile * kTcRows + t, rows);   // first tile's row, in flight during the set-up
    // Weights, all loads issued before any is used (coalesced over the
    // outputs); 8 consecutive K values of one output form one 16-byte row of
    // a core matrix. Item i < 512: K group i / 64 of output i % 64 of W2;
    // 512-575: W1 and b1 of output i - 512; 576-639: b2; 640-703: w3, b3.
    for (int i = tid; i < 704; i += blockDim.x) {
        const int out = i & 63;
        if (i < 512) {
            const int c = i >> 6;
            float w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = __ldg(P + kW2 + (c * 8 + j) * 64 + out);
            *reinterpret_cast<uint4*>(&W.w2[core_idx(out, c * 8, kK2 / 8)]) =
                make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]),
                           pack_bf16(w[6], w[7]));
        } else if (i < 576) {
            float w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = __ldg(P + kW1 + j * 64 + out);
            const float b = __ldg(P + kB1 + out);
            *reinterpret_cast<uint4*>(&W.w1[core_idx(out, 0, kK1 / 8)]) =
                make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]),
                           pack_bf16(w[6], w[7]));
            *reinterpret_cast<uint4*>(&W.w1[core_idx(out, 8, kK1 / 8)]) = bias_row(b, false);
        } else if (i < 640) {
            *reinterpret_cast<uint4*>(&W.w2[core_idx(out, 64, kK2 / 8)]) = bias_row(__ldg(P + kB2 + out), false);
            *reinterpret_cast<uint4*>(&W.w2[core_idx(out, 72, kK2 / 8)]) = make_uint4(0u, 0u, 0u, 0u);
        } else {
            W.w3[out] = __ldg(P + kW3 + out);
            if (out == 0) W.b3 = __ldg(P + kB3);
        }
    }
    // constant-one columns of the group's A tiles (never overwritten)
    *reinterpret_cast<uint4*>(&G.x[core_idx(t, 8, kK1 / 8)]) = bias_row(0.0f, true);
    *reinterpret_cast<uint4*>(&G.h1[core_idx(t, 64, kK2 / 8)]) = bias_row(0.0f, true);
    *reinterpret_cast<uint4*>(&G.h1[core_idx(t, 72, kK2 / 8)]) = make_uint4(0u, 0u, 0u, 0u);
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&G.bar);
    const uint32_t ph = (uint32_t)__cvta_generic_to_shared(&G.phantom);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ph) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&W.tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = W.tmem;
    const uint32_t dcol = tmem + 64u * g;                                  // the group's accumulator
    const uint32_t lanes = dcol + ((uint32_t)((warp & 3) * 32) << 16);     // this warp's 32 lanes of it
    const uint64_t da1 = smem_desc(G.x, (kK1 / 8) * 128), db1 = smem_desc(W.w1, (kK1 / 8) * 128);
    const uint64_t da2 = smem_desc(G.h1, (kK2 / 8) * 128), db2 = smem_desc(W.w2, (kK2 / 8) * 128);
    const int bid = 1 + g;   // the group's named barrier
    uint32_t parity = 0;
    bool ok = true;
    for (; tile < tiles; tile += gstride) {
        const int64_t row = tile * kTcRows + t;
        *reinterpret_cast<uint4*>(&G.x[core_idx(t, 0, kK1 / 8)]) = xv;
        xv = load_feat(feat, row + gstride * kTcRows, rows);   // next tile's row, in flight during this one
        fence_async_smem();
        tc_fence_before();
        group_sync(bid);
        if (t == 0) {
            tc_fence_after();
            tc_mma(dcol, da1, db1, kIdescM128N64, 0u);
            tc_commit(bar);
        }
        ok = wt.phantom ? mbar_wait(ph, 0u, wt.ns) : mbar_wait(bar, parity, wt.ns);
        if (group_sync_or(bid, !ok)) {
            ok = false;   // every thread of the group takes the failure path
            break;
        }
        parity ^= 1u;
        tc_fence_after();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tc_ld32(lanes + 32 * half, v);
            tc_wait_ld();
            const __nv_bfloat162 zero2 = __float2bfloat162_rn(0.0f);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t q[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const __nv_bfloat162 h = __hmax2(__floats2bfloat162_rn(v[c * 8 + 2 * j], v[c * 8 + 2 * j + 1]), zero2);
                    q[j] = *reinterpret_cast<const uint32_t*>(&h);
                }
                *reinterpret_cast<uint4*>(&G.h1[core_idx(t, (half * 4 + c) * 8, kK2 / 8)]) =
                    make_uint4(q[0], q[1], q[2], q[3]);
            }
        }
        fence_async_smem();
        tc_fence_before();
        group_sync(bid);
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kK2 / 16; ++kk)   // K step of 16 = 256 B = 16 in the address field
                tc_mma(dcol, da2 + 16u * kk, db2 + 16u * kk, kIdescM128N64, kk > 0 ? 1u : 0u);
            tc_commit(bar);
        }
        ok = mbar_wait(bar, parity, wt.ns);
        if (group_sync_or(bid, !ok)) {
            ok = false;   // every thread of the group takes the failure path
            break;
        }
        parity ^= 1u;
        tc_fence_after();
        float z = W.b3;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tc_ld32(lanes + 32 * half, v);
            tc_wait_ld();
#pragma unroll
            for (int c = 0; c < 32; ++c) z = __fmaf_rn(fmaxf(v[c], 0.0f), W.w3[half * 32 + c], z);
        }
        if (row < rows) pout[row] = sigmoidf(z);
        tc_fence_before();
    }
    bool drained = true;
    if (!ok) {
        // a wait gave up: raise the status, wait (bounded) for the MMA already
        // issued, and leave NaN in every row of this group that was not scored
        if (t == 0) atomicExch(&g_tc_status, (int32_t)ACS_ETIMEOUT);
        drained = mbar_wait(bar, parity, kDrainNs);
        for (; tile < tiles; tile += gstride) {
            const int64_t row = tile * kTcRows + t;
            if (row < rows) pout[row] = __int_as_float(0x7fc00000);
        }
    }
    tc_fence_before();
    // tensor memory is freed only when no MMA of the CTA can still be in flight
    const bool can_free = __syncthreads_and(drained);
    if (warp == 0 && can_free) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Training: fused forward + backward over one mini-batch on tcgen05.
//
// A CTA of four warps takes 128 mini-batch rows per tile (row t = thread t =
// TMEM lane t), with the scoring kernel's operand layouts and rounding
// points, and accumulates the weight gradients of all its tiles in TMEM:
//   layer 1, layer 2      as in scoring (biases in the K padding)
//   dz = (sigmoid(z) - y) / batch,  dh2 = dz w3 relu'(a2)          (FP32)
//   dh1 = (dh2 W2^T) relu'(a1):  D[128 x 64] = DH2[128 x 64] W2n  (BF16 dh2)
//   [dW2  .  ]   [h1^T]
//   [ .  dW1 ] = [x^T ] [dh2 | dh1]: Dw[128 x 128] += A[128 x K] B[K x 128]
// with K = the tile's 128 rows (eight MMAs of K = 16): rows 0-63 of A are
// h1^T, rows 64-71 x^T, the rest zero; columns 0-63 of B are dh2, 64-127
// dh1 (both BF16), so the two diagonal blocks of Dw are dW2 and dW1 and the
// off-diagonal ones are not used. Transposed operands are written by the
// epilogues element by element, into tiles whose core matrices are padded
// along K to 144 B (leading byte offset 144 instead of 128): a warp then
// writes 32 K-consecutive values of one row into four 16-byte pieces on
// distinct banks instead of four pieces on the same four banks. The bias and w3 gradients are FP32 column
// sums over the tile, staged through shared memory. Dw sits in TMEM columns
// 128-255 and is added into the gradient once per CTA.

constexpr int kKr = kTcRows;   // K of the weight-gradient GEMM: the tile's rows
constexpr int kPadCore = 72;   // elements between K-adjacent core matrices of at / bt (144 B)
constexpr int kPadRows = kPadCore * (kKr / 8);   // elements between 8-row groups of at / bt
// descriptor start advance of one K = 16 step (two padded core matrices), in 16-byte units
constexpr uint32_t kPadStep = 2u * (2u * kPadCore) / 16u;

// element index of (row r, column k) in the padded at / bt tiles
__device__ __forceinline__ int pad_idx(int r, int k)
{
    return (r >> 3) * kPadRows + (k >> 3) * kPadCore + ((r & 7) << 3) + (k & 7);
}
constexpr int kStage = 68;     // FP32 staging row (64 + 4: conflict-free 16-byte stores)
constexpr uint32_t kIdescM128N128 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

struct TrainSmem {
    uint16_t w1[64 * kK1];        // layer-1 B = [W1 ; b1]^T
    uint16_t w2[64 * kK2];        // layer-2 B = [W2 ; b2]^T
    uint16_t w2n[64 * 64];        // dh1 B = W2 as [in][out] (K = out)
    uint16_t x[kTcRows * kK1];    // layer-1 A (16 row groups x 2 K groups; K 8-10 constant ones)
    uint16_t h1[kTcRows * kK2];   // layer-2 A (16 x 10; K 64-66 constant ones)
    uint16_t dh2[kTcRows * 64];   // dh1 A: dh2 [row][out]
    uint16_t at[16 * kPadRows];   // weight-gradient A: [h1^T ; x^T ; 0] (16 x 16 K groups, padded)
    uint16_t bt[16 * kPadRows];   // weight-gradient B: [dh2 | dh1]^T (padded)
    float stage[kTcRows * kStage];   // FP32 rows for the column sums
    float w3[64];
    float red[3 * 64 + 2];        // b1, b2, w3 gradient sums, b3 sum, loss sum
    float b3;
    uint32_t tmem;
    unsigned long long bar;
    unsigned long long phantom;   // never arrived on (test hook of the bounded wait)
};
static_assert(offsetof(TrainSmem, w2) % 128 == 0 && offsetof(TrainSmem, w2n) % 128 == 0 &&
                  offsetof(TrainSmem, x) % 128 == 0 && offsetof(TrainSmem, h1) % 128 == 0 &&
                  offsetof(TrainSmem, dh2) % 128 == 0 && offsetof(TrainSmem, at) % 128 == 0 &&
                  offsetof(TrainSmem, bt) % 128 == 0 && offsetof(TrainSmem, stage) % 16 == 0,
              "operand tiles must start on core-matrix boundaries");
static_assert(sizeof(TrainSmem) <= 227 * 1024, "training CTA does not fit");

// Column sums of the staged FP32 tile into red[0..63] (two threads per column).
__device__ __forceinline__ void stage_column_sums(const float* stage, float* red, int t)
{
    const int c = t & 63, r0 = (t >> 6) * 64;
    float s = 0.0f;
    for (int r = r0; r < r0 + 64; ++r) s += stage[r * kStage + c];
    atomicAdd(&red[c], s);
}

__global__ void __launch_bounds__(kTcRows, 1)
mlp_train_kernel(const float* P, const uint16_t* feat, const float* label, int64_t total, int64_t first,
                 int64_t batch, int64_t pa, int64_t pc, float* grad, float* loss, TcWait wt)
{
    extern __shared__ __align__(128) unsigned char tsm[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(tsm);
    const int t = threadIdx.x, warp = t >> 5;
    for (int i = t; i < 704; i += kTcRows) {
        const int out = i & 63;
        if (i < 512) {   // W2^T (forward) and W2 (dh1) K group c of output / input `out`
            const int c = i >> 6;
            float w[8], u[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                w[j] = __ldg(P + kW2 + (c * 8 + j) * 64 + out);   // W2[in = 8c+j][out]
                u[j] = __ldg(P + kW2 + out * 64 + c * 8 + j);     // W2[in = out][out' = 8c+j]
            }
            *reinterpret_cast<uint4*>(&S.w2[core_idx(out, c * 8, kK2 / 8)]) =
                make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]),
                           pack_bf16(w[6], w[7]));
            *reinterpret_cast<uint4*>(&S.w2n[core_idx(out, c * 8, 8)]) =
                make_uint4(pack_bf16(u[0], u[1]), pack_bf16(u[2], u[3]), pack_bf16(u[4], u[5]),
                           pack_bf16(u[6], u[7]));
        } else if (i < 576) {
            float w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = __ldg(P + kW1 + j * 64 + out);
            *reinterpret_cast<uint4*>(&S.w1[core_idx(out, 0, kK1 / 8)]) =
                make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]),
                           pack_bf16(w[6], w[7]));
            *reinterpret_cast<uint4*>(&S.w1[core_idx(out, 8, kK1 / 8)]) = bias_row(__ldg(P + kB1 + out), false);
        } else if (i < 640) {
            *reinterpret_cast<uint4*>(&S.w2[core_idx(out, 64, kK2 / 8)]) = bias_row(__ldg(P + kB2 + out), false);
            *reinterpret_cast<uint4*>(&S.w2[core_idx(out, 72, kK2 / 8)]) = make_uint4(0u, 0u, 0u, 0u);
        } else if (i < 704) {
            S.w3[out] = __ldg(P + kW3 + out);
            if (out == 0) S.b3 = __ldg(P + kB3);
        }
    }
    for (int i = t; i < 3 * 64 + 2; i += kTcRows) S.red[i] = 0.0f;
    // constant parts of the A tiles: the ones columns, and rows 72-127 of the
    // weight-gradient A (x^T fills rows 64-71 each tile)
    *reinterpret_cast<uint4*>(&S.x[core_idx(t, 8, kK1 / 8)]) = bias_row(0.0f, true);
    *reinterpret_cast<uint4*>(&S.h1[core_idx(t, 64, kK2 / 8)]) = bias_row(0.0f, true);
    *reinterpret_cast<uint4*>(&S.h1[core_idx(t, 72, kK2 / 8)]) = make_uint4(0u, 0u, 0u, 0u);
    for (int i = t; i < 56 * kKr / 8; i += kTcRows) {   // rows 72..127, 16 B at a time
        const int m = 72 + i / (kKr / 8), k = (i % (kKr / 8)) * 8;
        *reinterpret_cast<uint4*>(&S.at[pad_idx(m, k)]) = make_uint4(0u, 0u, 0u, 0u);
    }
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&S.bar);
    const uint32_t ph = (uint32_t)__cvta_generic_to_shared(&S.phantom);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ph) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&S.tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t lanes = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's lanes, columns 0-63
    const uint32_t dw = tmem + 128u;                                // weight-gradient accumulator
    const uint64_t dx = smem_desc(S.x, (kK1 / 8) * 128), dw1 = smem_desc(S.w1, (kK1 / 8) * 128);
    const uint64_t dh1a = smem_desc(S.h1, (kK2 / 8) * 128), dw2 = smem_desc(S.w2, (kK2 / 8) * 128);
    const uint64_t ddh2 = smem_desc(S.dh2, 8 * 128), dw2n = smem_desc(S.w2n, 8 * 128);
    const uint64_t dat = smem_desc(S.at, 2 * kPadRows, 2 * kPadCore);
    const uint64_t dbt = smem_desc(S.bt, 2 * kPadRows, 2 * kPadCore);
    const float inv_b = 1.0f / (float)batch;
    uint32_t parity = 0;
    bool ok = true, any = false;
    float dzsum = 0.0f, lsum = 0.0f;
    const int64_t blocks = (batch + kTcRows - 1) / kTcRows;
    for (int64_t blk = blockIdx.x; blk < blocks; blk += gridDim.x) {
        const int64_t b = blk * kTcRows + t;
        const bool valid = b < batch;
        const int64_t row =
            valid ? (int64_t)(((unsigned __int128)pa * (unsigned __int128)(first + b) + pc) % (unsigned __int128)total) : 0;
        const uint4 xv = valid ? __ldg(reinterpret_cast<const uint4*>(feat) + row) : make_uint4(0u, 0u, 0u, 0u);
        const float y = valid ? label[row] : 0.0f;
        *reinterpret_cast<uint4*>(&S.x[core_idx(t, 0, kK1 / 8)]) = xv;
        {   // x^T into rows 64-71 of the weight-gradient A
            const uint16_t* xs = reinterpret_cast<const uint16_t*>(&xv);
#pragma unroll
            for (int f = 0; f < 8; ++f) S.at[pad_idx(64 + f, t)] = xs[f];
        }
        // ---- layer 1
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            tc_mma(tmem, dx, dw1, kIdescM128N64, 0u);
            tc_commit(bar);
        }
        ok = wt.phantom ? mbar_wait(ph, 0u, wt.ns) : mbar_wait(bar, parity, wt.ns);
        if (__syncthreads_or(!ok)) {
            ok = false;   // every thread takes the failure path
            break;
        }
        parity ^= 1u;
        tc_fence_after();
        uint32_t m1[2] = {0u, 0u};   // relu'(a1)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tc_ld32(lanes + 32 * half, v);
            tc_wait_ld();
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t q[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = c * 8 + 2 * j;
                    q[j] = pack_bf16(fmaxf(v[k], 0.0f), fmaxf(v[k + 1], 0.0f));
                }
                *reinterpret_cast<uint4*>(&S.h1[core_idx(t, (half * 4 + c) * 8, kK2 / 8)]) =
                    make_uint4(q[0], q[1], q[2], q[3]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {   // h1^T into rows 0-63 of the weight-gradient A
                    const int in = half * 32 + c * 8 + 2 * j;
                    S.at[pad_idx(in, t)] = (uint16_t)(q[j] & 0xFFFFu);
                    S.at[pad_idx(in + 1, t)] = (uint16_t)(q[j] >> 16);
                }
            }
#pragma unroll
            for (int k = 0; k < 32; ++k)
                if (v[k] > 0.0f) m1[half] |= 1u << k;
        }
        // ---- layer 2
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kK2 / 16; ++kk)
                tc_mma(tmem, dh1a + 16u * kk, dw2 + 16u * kk, kIdescM128N64, kk > 0 ? 1u : 0u);
            tc_commit(bar);
        }
        ok = mbar_wait(bar, parity, wt.ns);
        if (__syncthreads_or(!ok)) {
            ok = false;   // every thread takes the failure path
            break;
        }
        parity ^= 1u;
        tc_fence_after();
        float a2[64];
        tc_ld32(lanes, a2);
        tc_ld32(lanes + 32, a2 + 32);
        tc_wait_ld();
        float z = S.b3;   // as in scoring
#pragma unroll
        for (int c = 0; c < 64; ++c) z = __fmaf_rn(fmaxf(a2[c], 0.0f), S.w3[c], z);
        const float dz = valid ? (sigmoidf(z) - y) * inv_b : 0.0f;
        if (valid) lsum += bce_term(z, y);
        dzsum += dz;
        // dw3 partials: h2 dz, staged for the column sums
#pragma unroll
        for (int c = 0; c < 64; c += 4)
            *reinterpret_cast<float4*>(&S.stage[t * kStage + c]) =
                make_float4(fmaxf(a2[c], 0.0f) * dz, fmaxf(a2[c + 1], 0.0f) * dz, fmaxf(a2[c + 2], 0.0f) * dz,
                            fmaxf(a2[c + 3], 0.0f) * dz);
        __syncthreads();
        stage_column_sums(S.stage, S.red + 128, t);
        __syncthreads();
        // dh2 = dz w3 relu'(a2): FP32 staged for db2; BF16 as the dh1 A and
        // as columns 0-63 of the weight-gradient B
#pragma unroll
        for (int c = 0; c < 64; ++c) a2[c] = a2[c] > 0.0f ? dz * S.w3[c] : 0.0f;
#pragma unroll
        for (int c = 0; c < 64; c += 4)
            *reinterpret_cast<float4*>(&S.stage[t * kStage + c]) = make_float4(a2[c], a2[c + 1], a2[c + 2], a2[c + 3]);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = pack_bf16(a2[c * 8 + 2 * j], a2[c * 8 + 2 * j + 1]);
            *reinterpret_cast<uint4*>(&S.dh2[core_idx(t, c * 8, 8)]) = make_uint4(q[0], q[1], q[2], q[3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int out = c * 8 + 2 * j;
                S.bt[pad_idx(out, t)] = (uint16_t)(q[j] & 0xFFFFu);
                S.bt[pad_idx(out + 1, t)] = (uint16_t)(q[j] >> 16);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        // ---- dh1 = dh2 W2^T (the tensor core) while the db2 sums run
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc_mma(tmem, ddh2 + 16u * kk, dw2n + 16u * kk, kIdescM128N64, kk > 0 ? 1u : 0u);
            tc_commit(bar);
        }
        stage_column_sums(S.stage, S.red + 64, t);
        ok = mbar_wait(bar, parity, wt.ns);
        if (__syncthreads_or(!ok)) {
            ok = false;   // every thread takes the failure path
            break;
        }
        parity ^= 1u;
        tc_fence_after();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tc_ld32(lanes + 32 * half, v);
            tc_wait_ld();
#pragma unroll
            for (int k = 0; k < 32; ++k)
                if (!((m1[half] >> k) & 1u)) v[k] = 0.0f;
#pragma unroll
            for (int c = 0; c < 32; c += 4)
                *reinterpret_cast<float4*>(&S.stage[t * kStage + half * 32 + c]) =
                    make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
#pragma unroll
            for (int j = 0; j < 16; ++j) {   // dh1 as columns 64-127 of the weight-gradient B
                const uint32_t q = pack_bf16(v[2 * j], v[2 * j + 1]);
                const int in = half * 32 + 2 * j;
                S.bt[pad_idx(64 + in, t)] = (uint16_t)(q & 0xFFFFu);
                S.bt[pad_idx(64 + in + 1, t)] = (uint16_t)(q >> 16);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        // ---- weight gradients, accumulated over the CTA's tiles
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kKr / 16; ++kk)
                tc_mma(dw, dat + kPadStep * kk, dbt + kPadStep * kk, kIdescM128N128, (any || kk > 0) ? 1u : 0u);
            tc_commit(bar);
        }
        any = true;
        stage_column_sums(S.stage, S.red, t);   // db1
        ok = mbar_wait(bar, parity, wt.ns);
        if (__syncthreads_or(!ok)) {
            ok = false;   // every thread takes the failure path
            break;
        }
        parity ^= 1u;
        tc_fence_after();
    }
    bool drained = true;
    if (!ok) {
        // a wait gave up: raise the status, wait (bounded) for the MMA already
        // issued; the loss becomes NaN and no gradient is added
        if (t == 0) {
            atomicExch(&g_tc_status, (int32_t)ACS_ETIMEOUT);
            atomicAdd(loss, __int_as_float(0x7fc00000));
        }
        drained = mbar_wait(bar, parity, kDrainNs);
    } else {
        if (any) {   // Dw rows: 0-63 dW2[in][out] (columns 0-63), 64-71 dW1[f][h] (columns 64-127)
            const int m = warp * 32 + (t & 31);
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                float v[32];
                tc_ld32(dw + ((uint32_t)(warp * 32) << 16) + 32 * q, v);
                tc_wait_ld();
                if (m < 64 && q < 2) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) atomicAdd(&grad[kW2 + m * 64 + q * 32 + c], v[c]);
                } else if (m >= 64 && m < 72 && q >= 2) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) atomicAdd(&grad[kW1 + (m - 64) * 64 + (q - 2) * 32 + c], v[c]);
                }
            }
        }
        // dz and loss sums of the CTA
        float l = lsum, d = dzsum;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            l += __shfl_xor_sync(0xffffffffu, l, off);
            d += __shfl_xor_sync(0xffffffffu, d, off);
        }
        if ((t & 31) == 0) {
            atomicAdd(&S.red[192], d);
            atomicAdd(&S.red[193], l);
        }
        __syncthreads();
        if (t < 64) {
            atomicAdd(&grad[kB1 + t], S.red[t]);
            atomicAdd(&grad[kB2 + t], S.red[64 + t]);
            atomicAdd(&grad[kW3 + t], S.red[128 + t]);
        }
        if (t == 0) {
            atomicAdd(&grad[kB3], S.red[192]);
            atomicAdd(loss, S.red[193] * inv_b);
        }
    }
    tc_fence_before();
    // tensor memory is freed only when no MMA of the CTA can still be in flight
    const bool can_free = __syncthreads_and(drained);
    if (warp == 0 && can_free) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(256u) : "memory");
    }
}

__global__ void adam_kernel(float* P, const float* G, float* M, float* Vv, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.0f - b1) * g;
    const float v = b2 * Vv[i] + (1.0f - b2) * g * g;
    M[i] = m;
    Vv[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// Per-node statistics of the candidate graph: mean and last candidate
// distance (each at least 1), in-degree.
__global__ void node_stats_kernel(const int32_t* xy, const int32_t* nn, int n, int cl, float* dmean,
                                  float* dlast, int* indeg)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int2* p = reinterpret_cast<const int2*>(xy);
    int d = 0;
    if (lane < cl) {
        const int j = nn[(size_t)i * 32 + lane];
        d = euc2d(p[i], p[j]);
        atomicAdd(&indeg[j], 1);
    }
    int s = d;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const int dl = __shfl_sync(0xffffffffu, d, cl - 1);
    if (lane == 0) {
        dmean[i] = fmaxf((float)s / (float)cl, 1.0f);
        dlast[i] = (float)max(dl, 1);
    }
}

__global__ void features_kernel(const int32_t* xy, const int32_t* nn, int n, int cl, const float* dmean,
                                const float* dlast, const int* indeg, uint16_t* feat)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * 32) return;
    const int i = (int)(e >> 5), k = (int)(e & 31);
    float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (k < cl) {
        const int2* p = reinterpret_cast<const int2*>(xy);
        const int j = nn[e];
        const float d = (float)euc2d(p[i], p[j]);
        const float fcl = (float)cl;
        f[0] = (float)k / fcl;
        f[1] = d / dmean[i];
        f[2] = d / dlast[i];
        f[3] = (float)(p[j].x - p[i].x) / dlast[i];
        f[4] = (float)(p[j].y - p[i].y) / dlast[i];
        float rv = 1.0f;
        for (int q = 0; q < cl; ++q)
            if (nn[(size_t)j * 32 + q] == i) { rv = (float)q / fcl; break; }
        f[5] = rv;
        f[6] = d / dlast[j];
        f[7] = (float)indeg[j] / fcl;
    }
    uint4 out;
    out.x = pack_bf16(f[0], f[1]);
    out.y = pack_bf16(f[2], f[3]);
    out.z = pack_bf16(f[4], f[5]);
    out.w = pack_bf16(f[6], f[7]);
    *reinterpret_cast<uint4*>(feat + e * 8) = out;
}

__global__ void count_best_edges_kernel(const int32_t* nn, const int32_t* best, int n, int cl, float* count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int u = best[i], v = best[i + 1 < n ? i + 1 : 0];
    for (int side = 0; side < 2; ++side) {
        const int a = side ? v : u, b = side ? u : v;
        for (int k = 0; k < cl; ++k)
            if (nn[(size_t)a * 32 + k] == b) { atomicAdd(&count[(size_t)a * 32 + k], 1.0f); break; }
    }
}

// One warp per node: keep the `keep` best scores (ties -> lower rank) in rank
// order, reweighted w' = w * p; pad the rest of the row.
__global__ void apply_prior_kernel(int32_t* nn, float* w, const float* score, int n, int cl, int keep)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const size_t e = (size_t)i * 32 + lane;
    const bool valid = lane < cl;
    const float p = valid ? score[e] : -1.0f;
    if (valid && !(p >= 0.0f && p <= 1.0f)) atomicExch(&g_bad_score, 1);
    const int j = nn[e];
    const float wv = w[e];
    int rank = 0;   // candidates that beat this one
    for (int o = 0; o < 32; ++o) {
        const float po = __shfl_sync(0xffffffffu, p, o);
        if (o < cl && valid && (po > p || (po == p && o < lane))) ++rank;
    }
    const bool kept = valid && rank < keep;
    const unsigned bal = __ballot_sync(0xffffffffu, kept);
    const int pos = __popc(bal & ((1u << lane) - 1u));
    __syncwarp();
    if (kept) {
        nn[(size_t)i * 32 + pos] = j;
        w[(size_t)i * 32 + pos] = __fmul_rn(wv, p);
    }
    __syncwarp();
    if (lane >= keep) {
        nn[e] = -1;
        w[e] = 0.0f;
    }
}

acs_status launched(cudaError_t e) { return e == cudaSuccess ? ACS_OK : ACS_ECUDA; }

// Host side of the tensor-core status: the bounds the kernels get, and
// whether a give-up has been reported (then the MLP calls refuse to launch).
TcWait g_wait = {kWaitNs, 0};
bool g_tc_failed = false;

// Reads (after synchronising `st`) the device status word; on a recorded
// give-up marks the tensor-core path failed and returns ACS_ETIMEOUT.
acs_status tc_status(cudaStream_t st)
{
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return ACS_ECUDA;
    }
    int32_t v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return ACS_ECUDA;
    }
    if (v != 0) {
        g_tc_failed = true;
        return ACS_ETIMEOUT;
    }
    return ACS_OK;
}

}  // namespace

extern "C" {

acs_status acs_prior_features(acs_ctx* ctx, int32_t instance, uint16_t* dev_feat, void* stream)
{
    CtxView v;
    if (!dev_feat) return ACS_EINVAL;
    if (acs_status s = ctx_view(ctx, instance, &v)) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // scratch of the candidate-graph statistics (stream-ordered allocation)
    void* scratch = nullptr;
    const size_t bytes = (size_t)v.n * (2 * sizeof(float) + sizeof(int));
    if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) { cudaGetLastError(); return ACS_ENOMEM; }
    float* dmean = static_cast<float*>(scratch);
    float* dlast = dmean + v.n;
    int* indeg = reinterpret_cast<int*>(dlast + v.n);
    cudaError_t e = cudaMemsetAsync(indeg, 0, sizeof(int) * v.n, st);
    if (e == cudaSuccess) {
        node_stats_kernel<<<(v.n + 7) / 8, 256, 0, st>>>(v.xy, v.nn, v.n, v.cl, dmean, dlast, indeg);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int64_t rows = (int64_t)v.n * 32;
        features_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(v.xy, v.nn, v.n, v.cl, dmean,
                                                                       dlast, indeg, dev_feat);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    return launched(e);
}

acs_status acs_prior_count_best_edges(acs_ctx* ctx, int32_t instance, float* dev_count, void* stream)
{
    CtxView v;
    if (!dev_count) return ACS_EINVAL;
    if (acs_status s = ctx_view(ctx, instance, &v)) return s;
    if (!v.has_best) return ACS_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    count_best_edges_kernel<<<(v.n + 255) / 256, 256, 0, st>>>(v.nn, v.best, v.n, v.cl, dev_count);
    return launched(cudaGetLastError());
}

acs_status acs_mlp_forward(const float* dev_params, const uint16_t* dev_feat, int64_t rows, float* dev_p,
                           void* stream)
{
    if (rows == 0) return ACS_OK;
    if (!dev_params || !dev_feat || !dev_p || rows < 0 || ((uintptr_t)dev_feat & 15)) return ACS_EINVAL;
    if (g_tc_failed) return ACS_ESTATE;
    if (cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_smem(kTcMaxGroups)) != cudaSuccess)
        return ACS_ECUDA;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) return ACS_ECUDA;
    // groups per CTA: enough to give every SM its share of the tiles, at most
    // 8; persistent with one CTA per SM beyond 8 tiles per SM
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;
    const int64_t per_sm = (tiles + sms - 1) / sms;
    const int groups = (int)(per_sm < kTcMaxGroups ? per_sm : kTcMaxGroups);
    const int64_t ctas = (tiles + groups - 1) / groups;
    const int grid = (int)(ctas < sms ? ctas : sms);
    mlp_forward_tc_kernel<<<grid, kTcRows * groups, tc_smem(groups), (cudaStream_t)stream>>>(
        dev_params, dev_feat, rows, dev_p, tc_tmem_cols(groups), g_wait);
    return launched(cudaGetLastError());
}

acs_status acs_mlp_train_batch(const float* dev_params, const uint16_t* dev_feat, const float* dev_label,
                               int64_t total, int64_t first, int64_t batch, int64_t perm_a, int64_t perm_c,
                               float* dev_grad, float* dev_loss, void* stream)
{
    if (!dev_params || !dev_feat || !dev_label || !dev_grad || !dev_loss || total < 1 || batch < 1 ||
        first < 0 || perm_a < 1 || perm_c < 0 || ((uintptr_t)dev_feat & 15))
        return ACS_EINVAL;
    if (g_tc_failed) return ACS_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(dev_grad, 0, sizeof(float) * ACS_MLP_PARAMS, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev_loss, 0, sizeof(float), st);
    const size_t smem = sizeof(TrainSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return ACS_ECUDA;
    const int64_t blocks = (batch + kTcRows - 1) / kTcRows;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)(blocks < sms ? blocks : sms);
    mlp_train_kernel<<<grid, kTcRows, smem, st>>>(dev_params, dev_feat, dev_label, total, first, batch,
                                                  perm_a, perm_c, dev_grad, dev_loss, g_wait);
    return launched(cudaGetLastError());
}

acs_status acs_mlp_adam(float* dev_params, const float* dev_grad, float* dev_m, float* dev_v, int32_t step,
                        float lr, float beta1, float beta2, float eps, void* stream)
{
    if (!dev_params || !dev_grad || !dev_m || !dev_v || step < 1) return ACS_EINVAL;
    if (g_tc_failed) return ACS_ESTATE;
    // bias corrections in double: 1 - beta2^t cancels heavily in FP32 for small t
    const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
    const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
    adam_kernel<<<(ACS_MLP_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        dev_params, dev_grad, dev_m, dev_v, ACS_MLP_PARAMS, lr, beta1, beta2, eps, c1, c2);
    return launched(cudaGetLastError());
}

acs_status acs_apply_prior(acs_ctx* ctx, int32_t instance, const float* dev_p, int32_t keep, void* stream)
{
    CtxView v;
    if (!dev_p) return ACS_EINVAL;
    if (acs_status s = ctx_view(ctx, instance, &v)) return s;
    if (keep < 1 || keep > v.cl) return ACS_EINVAL;
    if (g_tc_failed) return ACS_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    // scores from a scoring launch whose wait gave up are incomplete
    if (acs_status ts = tc_status(st)) {
        ctx_poison(ctx);
        return ts;
    }
    apply_prior_kernel<<<(v.n + 7) / 8, 256, 0, st>>>(v.nn, v.w, dev_p, v.n, v.cl, keep);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = ctx_set_cl(ctx, instance, keep);
    int32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&bad, g_bad_score, sizeof(bad));
    if (e == cudaSuccess && bad) {
        const int32_t zero = 0;
        cudaMemcpyToSymbol(g_bad_score, &zero, sizeof(zero));
        e = cudaErrorInvalidValue;   // rows rewritten from scores that are not probabilities
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx_poison(ctx);
        return ACS_ECUDA;
    }
    return ACS_OK;
}

acs_status acs_set_candidates(acs_ctx* ctx, int32_t instance, const int32_t* nn, const float* w, int32_t cl)
{
    CtxView v;
    if (!nn || !w) return ACS_EINVAL;
    if (acs_status s = ctx_view(ctx, instance, &v)) return s;
    if (cl < 1 || cl > 32 || cl > v.n - 1) return ACS_EINVAL;
    for (int i = 0; i < v.n; ++i)
        for (int k = 0; k < cl; ++k) {
            const int32_t j = nn[(size_t)i * cl + k];
            if (j < 0 || j >= v.n || j == i || !(w[(size_t)i * cl + k] >= 0.0f)) return ACS_EINVAL;
        }
    int32_t* rn = new (std::nothrow) int32_t[(size_t)v.n * 32];
    float* rw = new (std::nothrow) float[(size_t)v.n * 32];
    if (!rn || !rw) {
        delete[] rn;
        delete[] rw;
        return ACS_ENOMEM;
    }
    for (int i = 0; i < v.n; ++i)
        for (int k = 0; k < 32; ++k) {
            rn[(size_t)i * 32 + k] = k < cl ? nn[(size_t)i * cl + k] : -1;
            rw[(size_t)i * 32 + k] = k < cl ? w[(size_t)i * cl + k] : 0.0f;
        }
    cudaStream_t st = (cudaStream_t)v.stream;
    cudaError_t e = cudaMemcpyAsync(v.nn, rn, sizeof(int32_t) * v.n * 32, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.w, rw, sizeof(float) * v.n * 32, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    delete[] rn;
    delete[] rw;
    if (e == cudaSuccess) e = ctx_set_cl(ctx, instance, cl);
    if (e != cudaSuccess) {
        ctx_poison(ctx);
        return ACS_ECUDA;
    }
    return ACS_OK;
}

acs_status acs_mlp_sync(void* stream)
{
    if (g_tc_failed) return ACS_ESTATE;
    return tc_status((cudaStream_t)stream);
}

acs_status acs_mlp_test_wait_hook(int64_t wait_ns, int32_t phantom)
{
    if (wait_ns < 0 || (phantom != 0 && phantom != 1)) return ACS_EINVAL;
    g_wait.ns = wait_ns == 0 ? kWaitNs : (unsigned long long)wait_ns;
    g_wait.phantom = phantom;
    return ACS_OK;
}

}  // extern "C"
