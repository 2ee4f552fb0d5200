// Shared-memory atomicOr throughput: the measured ceiling of the vote kernel, whose work is one
// shared atomic per cell update (the paper's shared-memory remedy for the A[B[i]] += 1 scatter,
// Sec. 6.1 and Sec. 8).  Each warp issues back-to-back 32-lane atomicOr instructions into a
// 16 KB tile in shared memory; the result is lane-atomics per second over the whole GPU.
#include <cuda_runtime.h>

#include <vector>

#include "hough_internal.cuh"

namespace hough {

namespace {

constexpr int kWords = 4096;   // 16 KB tile
constexpr int kThreads = 512;

__global__ void __launch_bounds__(kThreads) smem_or_kernel(int pattern, int iters, unsigned *sink)
{
    __shared__ unsigned tile[kWords];
    for (int q = threadIdx.x; q < kWords; q += kThreads) tile[q] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // pattern 0: lane l of warp w hits word (w * 32 + l) mod kWords, one word per bank;
    // pattern 1: a multiplicative-hash walk, so successive instructions hit unrelated words
    unsigned addr = (unsigned)(warp * 32 + lane) % kWords;
    const unsigned bit = 1u << (lane & 15);
    for (int it = 0; it < iters; ++it) {
        atomicOr(&tile[addr], bit);
        if (pattern == 0) {
            addr = (addr + 32u * 16u) % kWords;
        } else {
            addr = (addr * 2654435761u + 40503u * (unsigned)lane + 1u) % kWords;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(sink, tile[blockIdx.x % kWords]);
}

}  // namespace

cudaError_t run_smem_or_bench(int device, int pattern, double ms, double *atomics_per_s, uint64_t *launches)
{
    cudaError_t e;
    if ((e = cudaSetDevice(device))) return e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    unsigned *sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(unsigned)))) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int grid = sms * 4;   // four 512-thread CTAs per SM: 64 warps, full occupancy
    int iters = 256;
    float t = 0.f;
    // grow the loop until one launch takes about `ms`
    for (int tries = 0; tries < 20; ++tries) {
        cudaEventRecord(a);
        smem_or_kernel<<<grid, kThreads>>>(pattern, iters, sink);
        cudaEventRecord(b);
        ++*launches;
        if ((e = cudaEventSynchronize(b))) break;
        cudaEventElapsedTime(&t, a, b);
        if (t >= ms * 0.5 || iters >= (1 << 24)) break;
        iters *= 4;
    }
    if (!e) {
        cudaEventRecord(a);
        smem_or_kernel<<<grid, kThreads>>>(pattern, iters, sink);
        cudaEventRecord(b);
        ++*launches;
        e = cudaEventSynchronize(b);
        cudaEventElapsedTime(&t, a, b);
        *atomics_per_s = (double)grid * kThreads * (double)iters / (t * 1e-3);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return e ? e : cudaGetLastError();
}

}  // namespace hough
