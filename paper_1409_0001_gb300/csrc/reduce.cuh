// reduce.cuh -- deterministic block and grid reductions shared by the solver kernels.
// A kernel reduces one double per thread to a block partial in a fixed order, stores
// it, and the last block to arrive (atomic ticket) adds all partials in block order,
// so every reduction gives the same bits on every run.  Works for 1-D and 2-D blocks
// of kThreads threads.
#pragma once

#include <cuda_runtime.h>

namespace cgk {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kThreads / 32];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) ws[t >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (t == 0)
        for (int w = 0; w < kThreads / 32; ++w) r += ws[w];
    __syncthreads();
    return r;
}

// The same block reduction in FP32, for the residual norms of the mixed-precision
// passes (their values are FP32 already and the convergence test needs them to far less
// than FP32 accuracy; GB300 runs FP64 arithmetic at a small fraction of its FP32 rate,
// so even a block reduction in FP64 shows in these short passes).  The result is
// promoted to FP64 for the grid-wide sum.
__device__ __forceinline__ double block_sum_f(float v) {
    __shared__ float wsf[kThreads / 32];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) wsf[t >> 5] = v;
    __syncthreads();
    float r = 0.0f;
    if (t == 0)
        for (int w = 0; w < kThreads / 32; ++w) r += wsf[w];
    __syncthreads();
    return (double)r;
}

// Stores this block's partial(s) at partials[q * nb + bid]; true in the last block.
__device__ __forceinline__ bool arrive(double *partials, int nparts, const double *vals, int bid,
                                       int nb, unsigned int *ticket) {
    __shared__ bool last;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if (t == 0) {
        for (int q = 0; q < nparts; ++q) partials[q * nb + bid] = vals[q];
        __threadfence();
        unsigned k = atomicAdd(ticket, 1u);
        last = (k == (unsigned)nb - 1);
    }
    __syncthreads();
    return last;
}

// In the last block: total of partials[q][0..nb) in a fixed order (valid on thread 0).
__device__ __forceinline__ double finish_sum(const double *partials, int q, int nb) {
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    double s = 0.0;
    const double *pq = partials + (size_t)q * nb;
    for (int i = t; i < nb; i += kThreads) s += __ldcg(pq + i);
    return block_sum(s);
}

__device__ __forceinline__ bool is_thread0() { return threadIdx.x == 0 && threadIdx.y == 0; }

// Copies a 7-entry diagonal table into shared memory (dynamic indexing of a kernel
// parameter array would go through local memory).  One thread copies it with constant
// indices: a thread-dependent index into the parameter array made every thread of the
// kernel store a local copy of it first.  Visible after the first barrier of sweep25,
// before any consume().
template <class T>
__device__ __forceinline__ void stage_table(T *dst, const T *src) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
        for (int i = 0; i < 7; ++i) dst[i] = src[i];
    }
}


}  // namespace
}  // namespace cgk
