// Arithmetic-throughput probes: the denominators of the rooflines that the benchmark reports
// for its FP64, FP32 and double-float kernels. Each thread runs kChains independent
// dependent chains x <- x a + b for `iters` iterations (2 flops a step), enough independent
// work per warp that the issue rate of the arithmetic pipe, not the latency of one chain,
// bounds the kernel. The chains' sum is stored only under a condition that never holds for
// these inputs (it keeps the compiler from removing the chains).
#pragma once
#include <cuda_runtime.h>

#include "bl_df64.cuh"

namespace bl {

constexpr int kPeakThreads = 256;

template <class T, int kChains>
__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(T* __restrict__ sink, int iters,
                                                                 T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x % 7 + c) * T(0.125);
#pragma unroll 16
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = x[0];
#pragma unroll
    for (int c = 1; c < kChains; ++c) s += x[c];
    if (s == T(-1.0e30)) sink[blockIdx.x] = s;
}

// The same chains in this library's double-float arithmetic: x <- x a + b as the compensated
// product-sum the geodesic integrator uses for its stage sums (DFDot: one product term and
// one added term, renormalised once), counted as 2 flops like a native FMA.
template <int kChains>
__global__ void __launch_bounds__(kPeakThreads) df64_chain_kernel(float* __restrict__ sink, int iters,
                                                                  float a_hi, float a_lo,
                                                                  float b_hi, float b_lo) {
    const df64 a(a_hi, a_lo), b(b_hi, b_lo);
    df64 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = df64(float(threadIdx.x % 7 + c) * 0.125f, 0.0f);
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            DFDot d;
            d.first(x[c], a);
            d.add_term(b);
            x[c] = d.get();
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].hi + x[c].lo;
    if (s == -1.0e30f) sink[blockIdx.x] = s;
}

}  // namespace bl
