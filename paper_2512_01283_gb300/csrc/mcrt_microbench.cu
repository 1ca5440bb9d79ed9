// mcrt_microbench.cu -- throughput of the FP64 reductions the step-1 tallies are made of
// (the ceiling of the tally kernels besides plain copy bandwidth): scalar FP64 atomic
// adds with no return value, and 256-byte bulk reduce-adds of FP64 rows from shared
// memory (the form the tally kernels use), into a buffer that fits in L2 or one that
// does not.
#include <cuda_runtime.h>

#include "mcrt_internal.h"
#include "mcrt_packet.cuh"

namespace mcrt {

namespace {

// op i adds to the row (or word) at a multiplicative hash of i: spread over the buffer,
// no two consecutive ops on the same line
__device__ __forceinline__ unsigned long long spread(unsigned long long i, unsigned long long n) {
    return ((i * 0x9E3779B97F4A7C15ull) >> 11) % n;
}

__global__ void __launch_bounds__(256) k_red_f64(double* __restrict__ buf, unsigned long long words,
                                                 unsigned long long n_ops) {
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops;
         i += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(&buf[spread(i, words)], 1.0);
}

// one 256-byte row (32 doubles) per op, every thread issuing from the block's one source
// row (read only, so the copies in flight can share it)
__global__ void __launch_bounds__(256) k_bulk_red_f64(double* __restrict__ buf, unsigned long long rows,
                                                      unsigned long long n_ops) {
    __shared__ __align__(128) double src[32];
    if (threadIdx.x < 32) src[threadIdx.x] = 1.0;
    __syncthreads();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned s = (unsigned)__cvta_generic_to_shared(src);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        double* dst = buf + spread(i, rows) * 32;
        asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], 256;" ::"l"(dst), "r"(s)
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    bulk_wait_all();
}

}  // namespace

cudaError_t launch_microbench(int kind, double* buf, unsigned long long bytes, unsigned long long n_ops, int n_sm,
                              cudaStream_t s) {
    (void)cudaGetLastError();  // report this launch's error only
    const unsigned grid = (unsigned)n_sm * 8u;
    if (kind == 0)
        k_red_f64<<<grid, 256, 0, s>>>(buf, bytes / sizeof(double), n_ops);
    else
        k_bulk_red_f64<<<grid, 256, 0, s>>>(buf, bytes / 256, n_ops);
    return cudaGetLastError();
}

}  // namespace mcrt
