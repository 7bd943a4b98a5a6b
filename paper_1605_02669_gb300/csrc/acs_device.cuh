// acs_device.cuh -- device building blocks of libacs: Philox4x32-10, the
// EUC_2D distance and the heuristic weight. Arithmetic is IEEE FP32 with
// explicit round-to-nearest intrinsics (no FMA contraction; the library is
// also compiled with -fmad=false).
#pragma once
#include <cstdint>

namespace acs {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor bijection on a 4-word counter; the 2-word key advances by the
// Weyl increments (golden ratio and sqrt(3)-1 in 32-bit fixed point) between
// rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a0 = c.x, a2 = c.z;
        const uint32_t hi0 = __umulhi(0xD2511F53u, a0), lo0 = 0xD2511F53u * a0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, a2), lo1 = 0xCD9E8D57u * a2;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// 24 random bits on the 2^-24 grid of [0,1).
__device__ __forceinline__ float unit24(uint32_t x)
{
    return __fmul_rn(__uint2float_rn(x >> 8), 5.9604644775390625e-08f);
}

// EUC_2D: nint(sqrt(dx^2+dy^2)). A float square root gives an estimate within
// one unit for radicands below 2^42; integer corrections make it the exact
// floor, and sqrt(s) >= r+1/2 <=> s-r^2 > r rounds half up without ties.
__device__ __forceinline__ int32_t euc2d(int2 a, int2 b)
{
    const long long dx = (long long)a.x - b.x, dy = (long long)a.y - b.y;
    const long long s = dx * dx + dy * dy;
    long long r = (long long)sqrtf((float)s);
    while (r > 0 && r * r > s) --r;
    while ((r + 1) * (r + 1) <= s) ++r;
    return (int32_t)(r + ((s - r * r) > r ? 1 : 0));
}

// Heuristic weight eta^beta, eta = 1/max(d,1), as 1/(x^beta) with x^beta by
// repeated multiplication from the left.
__device__ __forceinline__ float heuristic(int32_t d, int beta)
{
    const float x = (float)(d > 1 ? d : 1);
    float p = 1.0f;
    for (int i = 0; i < beta; ++i) p = (i == 0) ? x : __fmul_rn(p, x);
    return __fdiv_rn(1.0f, p);
}

// Folded local update tau0 + P[k]*(tau - tau0) and global update
// tau + rho*(Delta - tau), each operation rounded on its own.
__device__ __forceinline__ float local_rule(float t, float tau0, float Pk)
{
    return __fadd_rn(tau0, __fmul_rn(Pk, __fsub_rn(t, tau0)));
}

__device__ __forceinline__ float global_rule(float t, float delta, float rho)
{
    return __fadd_rn(t, __fmul_rn(rho, __fsub_rn(delta, t)));
}

// Full-scan key of node j: (product bits, node) packed so that the larger
// product wins and, among equal products, the lower node index
// (non-negative floats order like their bit patterns). Nonzero for j >= 0.
__device__ __forceinline__ unsigned long long pack_pj(float p, int j)
{
    return ((unsigned long long)__float_as_uint(p) << 32) |
           (unsigned long long)(0xffffffffu - (uint32_t)j);
}

__device__ __forceinline__ uint32_t hash32(uint32_t k)
{
    return k * 2654435761u;
}

}  // namespace acs
