// Deterministic FP64 reductions over vector columns (fixed partition and fixed tree order, so a
// result is bitwise reproducible from run to run).
#pragma once

#include <cuda_runtime.h>

namespace iedd {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 128;  // partial sums per column

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the CTA, returned to thread 0 (fixed tree).
__device__ __forceinline__ double block_sum(double v, double *sh /* >= 32 */) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// part[k * kRedBlocks + b] = sum over chunk b of a[k*lda+i] * (b ? b[k*ldb+i] : 1)
__global__ void __launch_bounds__(kRedThreads)
dot_partial_kernel(const double *__restrict__ a, long long lda, const double *__restrict__ b,
                   long long ldb, long long N, double *__restrict__ part) {
    __shared__ double sh[32];
    const int k = blockIdx.y;
    const long long chunk = (N + kRedBlocks - 1) / kRedBlocks;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < N ? lo + chunk : N;
    const double *ak = a + (long long)k * lda;
    const double *bk = b ? b + (long long)k * ldb : nullptr;
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s += bk ? ak[i] * bk[i] : ak[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[(long long)k * kRedBlocks + blockIdx.x] = s;
}

// out[k] = sum_b part[k * kRedBlocks + b]   (one warp-tree per column)
__global__ void __launch_bounds__(kRedBlocks)
dot_final_kernel(const double *__restrict__ part, double *__restrict__ out) {
    __shared__ double sh[32];
    const int k = blockIdx.x;
    double v = part[(long long)k * kRedBlocks + threadIdx.x];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[k] = v;
}

}  // namespace iedd
