// Device helpers shared by the kernel translation units. Each translation
// unit that includes this file gets its own copy of the constant tables and
// must call its init function (filled from swe::tables()) before launching.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "swe_internal.h"

namespace swe {

// Packed derivative matrices, inverse Vandermonde matrices and LGL weights of
// all degrees 1..NMAX (offsets mat_offset(N), vec_offset(N)).
static __constant__ double c_D[MAT_TOTAL];
static __constant__ double c_Vinv[MAT_TOTAL];
static __constant__ double c_w[VEC_TOTAL];

static inline void upload_tables() {
    const Tables& t = tables();
    cudaMemcpyToSymbol(c_D, t.D, sizeof(t.D));
    cudaMemcpyToSymbol(c_Vinv, t.Vinv, sizeof(t.Vinv));
    cudaMemcpyToSymbol(c_w, t.w, sizeof(t.w));
}

template <int N>
__device__ __forceinline__ double Dm(int i, int j) {
    return c_D[mat_offset(N) + i * (N + 1) + j];
}

template <int N>
__device__ __forceinline__ double wq(int i) {
    return c_w[vec_offset(N) + i];
}

__device__ __forceinline__ bool stopped(const int* stop) {
    return stop != nullptr && *(volatile const int*)stop != 0;
}

// Positive doubles order like their bit patterns as unsigned integers.
__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

inline int grid_for(long long work, int threads) {
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 2147483647LL) b = 2147483647LL;
    return (int)b;
}

}  // namespace swe
