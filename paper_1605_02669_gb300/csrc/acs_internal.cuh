// acs_internal.cuh -- types shared by the host side and the kernels of libacs.
#pragma once
#include <cstdint>

namespace acs {

constexpr int kMaxCl = 32;          // candidate rows are padded to one warp
constexpr int kMaxN = 65536;        // edge keys lo*n+hi fit in 32 bits
constexpr int kMaxM = 1024;         // one ant per thread in the update phase
constexpr int kCoordLimit = 1 << 20;
constexpr uint32_t kEmpty = 0xffffffffu;

// Per-instance descriptor (device memory, read-only during a launch).
struct InstDesc {
    int32_t n;          // nodes
    int32_t cl;         // effective candidate width (<= 32, <= n-1)
    int32_t W;          // 32-bit visited words per ant = ceil(n/32)
    int32_t instance;   // Philox counter word 3
    int64_t xy_off;     // coords: xy[2*(xy_off + i) + {0,1}]
    int64_t row_off;    // candidate rows: nn/w[32*(row_off + c) + k]
    int64_t tau_off;    // matrix: tau[tau_off + c*n + j]; SPM: slot base spm_*[tau_off + c*s + i]
    int64_t node_off;   // per-node arrays (SPM tail, best tour): [node_off + c]
    int64_t tour_off;   // tours[tour_off + a*n + step]
    int64_t ant_off;    // lens[ant_off + a]
    int64_t vis_off;    // global visited words (when not in shared memory)
    int64_t hw_off;     // heuristic matrix hw[hw_off + c*n + j] (when present)
    float tau0;
    int32_t pad;
};

// Kernel arguments of the construct kernel (one iteration of Alg. 1 on every
// instance of a context).
struct ConstructArgs {
    const InstDesc* desc;
    const int32_t* order;     // instances in longest-first order
    int32_t num_inst;
    int32_t m;                // ants
    const int32_t* xy;
    const int32_t* nn;        // [rows][32], -1 padded
    const float* w;           // [rows][32], 0 padded
    const float* hw;          // heuristic matrix (same offsets as the matrix), or null
    float* tau;               // matrix entries, or SPM trail values
    int32_t* spm_idx;         // SPM neighbour per slot
    int32_t* spm_tail;        // SPM tail per node
    int32_t* tours;
    int64_t* lens;
    int32_t* best;            // best-so-far tours [sum n]
    int64_t* best_len;        // [B], INT64_MAX before the first iteration
    int64_t* iteration;       // [B]
    unsigned long long* stats;// [B][4]
    uint32_t* vis_global;     // visited words when they do not fit in smem
    const float* P;           // decay table P[0..m]
    int32_t* status;          // nonzero = an internal check failed
    float q0, rho;
    int32_t beta, s, period;
    uint32_t key0, key1;
    int32_t vis_in_smem, xy_in_smem, max_n;
    int32_t mc;               // ants per CTA of a cluster = ceil(m / cluster size)
    int32_t nrec;             // SPM records per CTA in shared memory (0 = global)
    int32_t skip_default;     // SPM: a local update of an absent edge inserts nothing
    const int32_t* ext;       // SPM: per node the kExtList nodes with the largest full-scan
                              // keys of an absent trail, best first, -1 padded; or null
    int32_t* sched;           // next-instance counter (zeroed before each launch) when the
                              // batch has more instances than resident clusters; null =
                              // cluster k takes instances k, k + clusters, ...
};

// Length of the SPM's extended neighbour lists (rows of ConstructArgs::ext).
constexpr int kExtList = 256;
// Added to an SPM kernel mode to select the variant that uses those lists.
constexpr int kExtVariant = 3;

// Shared-memory carve of the construct kernel; the same arithmetic runs on
// the host (to size the launch) and on the device (to place the arrays).
// mc = ants owned by one CTA of the cluster, m = ants of the instance.
struct SmemLayout {
    uint32_t P, cur, start, nxt, tsel, len, pedge, qant, qc, qpart, xj, eqal, gkey, gu, gv, grep, gcnt,
        ev0, ev1, misc, ridx, rval, rtail, vis, xy, total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// mc = ants owned by one CTA of the cluster, m = ants of the instance, nrec =
// SPM records held in shared memory by one CTA (0 = records stay in global
// memory), s = SPM slots per record (0 for the matrix).
__host__ __device__ inline SmemLayout smem_layout(int m, int mc, int nrec, int s, int W, int max_n,
                                                  bool vis_in_smem, bool xy_in_smem)
{
    SmemLayout L;
    uint32_t o = 0;
    L.P = o;     o = align16(o + 4u * (m + 1));
    L.cur = o;   o = align16(o + 4u * mc);
    L.start = o; o = align16(o + 4u * mc);
    L.nxt = o;   o = align16(o + 4u * mc);
    L.tsel = o;  o = align16(o + 4u * mc);
    L.len = o;   o = align16(o + 8u * mc);
    L.pedge = o; o = align16(o + 4u * mc);
    L.qant = o;  o = align16(o + 4u * mc);
    L.qc = o;    o = align16(o + 4u * mc);
    L.qpart = o; o = align16(o + 8u * mc);
    L.xj = o;    o = align16(o + 4u * mc);
    L.eqal = o;  o = align16(o + 4u * m);
    L.gkey = o;  o = align16(o + 4u * m);
    L.gu = o;    o = align16(o + 4u * m);
    L.gv = o;    o = align16(o + 4u * m);
    L.grep = o;  o = align16(o + 4u * m);
    L.gcnt = o;  o = align16(o + 4u * m);
    L.ev0 = o;   o = align16(o + 4u * m);
    L.ev1 = o;   o = align16(o + 4u * m);
    L.misc = o;  o = align16(o + 256u);
    L.ridx = o;  o = align16(o + 4u * (uint32_t)nrec * (uint32_t)s);
    L.rval = o;  o = align16(o + 4u * (uint32_t)nrec * (uint32_t)s);
    L.rtail = o; o = align16(o + 4u * (uint32_t)nrec);
    L.vis = o;   if (vis_in_smem) o = align16(o + 4u * (uint32_t)mc * (uint32_t)W);
    L.xy = o;    if (xy_in_smem) o = align16(o + 8u * (uint32_t)max_n);
    L.total = o;
    return L;
}

// What the learned-prior entry points need from a context (acs_api.cu).
struct CtxView {
    int n, cl;
    const int32_t* xy;   // coordinates of the instance [n][2]
    int32_t* nn;         // candidate rows [n][32]
    float* w;            // candidate weights [n][32]
    const int32_t* best; // best-so-far tour [n]
    void* stream;        // cudaStream_t of the context
    bool has_best;
};

}  // namespace acs
