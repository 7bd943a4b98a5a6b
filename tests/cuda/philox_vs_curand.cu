// Test helper: the library's Philox4x32-10 (acs_device.cuh) beside cuRAND's
// device function of the same name, on the same counters and keys.
#include <cstdint>

#include <cuda_runtime.h>
#include <curand_kernel.h>

#include "acs_device.cuh"

__global__ void both(const uint4* ctr, const uint2* key, int count, uint4* ours, uint4* theirs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    ours[i] = acs::philox4x32_10(ctr[i], key[i].x, key[i].y);
    theirs[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int philox_pair(const uint32_t* ctr, const uint32_t* key, int count, uint32_t* ours,
                           uint32_t* theirs)
{
    uint4 *dc = nullptr, *d1 = nullptr, *d2 = nullptr;
    uint2* dk = nullptr;
    const size_t b4 = sizeof(uint4) * (size_t)count, b2 = sizeof(uint2) * (size_t)count;
    if (cudaMalloc(&dc, b4) || cudaMalloc(&d1, b4) || cudaMalloc(&d2, b4) || cudaMalloc(&dk, b2))
        return 1;
    cudaMemcpy(dc, ctr, b4, cudaMemcpyHostToDevice);
    cudaMemcpy(dk, key, b2, cudaMemcpyHostToDevice);
    both<<<(count + 255) / 256, 256>>>(dc, dk, count, d1, d2);
    int rc = cudaDeviceSynchronize() != cudaSuccess;
    cudaMemcpy(ours, d1, b4, cudaMemcpyDeviceToHost);
    cudaMemcpy(theirs, d2, b4, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(d1);
    cudaFree(d2);
    cudaFree(dk);
    return rc;
}
