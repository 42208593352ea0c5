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

// 1/x for normal x in [2^-1022, 2^1022): the hardware's approximate
// reciprocal (PTX rcp.approx.ftz.f64) refined by two steps of Newton's
// iteration for f(r) = 1/r - x, r <- r + r (1 - x r), each of which squares
// the relative error; the result is within one unit in the last place of 1/x
// (four FP64 fused multiply-adds instead of a correctly rounded division).
__device__ __forceinline__ double recip_normal(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// x in the range of recip_normal (an integer test of the bit pattern; false
// for zero, negative, subnormal, huge, infinite and NaN x).
__device__ __forceinline__ bool recip_range(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return b - 0x0010000000000000ULL < 0x7fd0000000000000ULL - 0x0010000000000000ULL;
}

// 1/x for x > 0 (the division outside the range of recip_normal).
__device__ __forceinline__ double recip_pos(double x) {
    return recip_range(x) ? recip_normal(x) : 1.0 / x;
}

// sqrt(x) for x >= 0: for x in the range of recip_normal, the hardware's
// approximate reciprocal square root (PTX rsqrt.approx.ftz.f64) y, then
// s = x y and two Newton (Heron) corrections s <- s + (y/2)(x - s^2) with
// the slope 1/(2 sqrt x) taken from y; the first squares the relative error
// of y, the second multiplies the remainder by it again, so the result is
// within one unit in the last place (six FP64 instructions). Zero and
// values outside that range take the library square root.
__device__ __forceinline__ double sqrt_pos(double x) {
    if (!recip_range(x)) return sqrt(x);
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double hy = 0.5 * y;
    double s = x * y;
    s = fma(hy, fma(-s, s, x), s);
    return fma(hy, fma(-s, s, x), s);
}

// x != 0 (either sign of zero counts as zero), from the bit pattern: an
// integer test, so that it costs no FP64 instruction.
__device__ __forceinline__ bool nonzero(double x) {
    return ((unsigned long long)__double_as_longlong(x) << 1) != 0ULL;
}

// max(x, 0) by the sign bit (an integer test, no FP64 instruction).
__device__ __forceinline__ double pos_part(double x) {
    return (long long)__double_as_longlong(x) > 0 ? x : 0.0;
}

// -x by the sign bit.
__device__ __forceinline__ double negated(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// Velocities u = hu/h, v = hv/h where h > 0, zero where h <= 0.
__device__ __forceinline__ void velocities(double h, double hu, double hv, double& u, double& v) {
    if (recip_range(h)) {
        const double r = recip_normal(h);
        u = hu * r;
        v = hv * r;
    } else if ((long long)__double_as_longlong(h) > 0) {
        u = hu / h;  // subnormal, huge, infinite or NaN h
        v = hv / h;
    } else {
        u = v = 0.0;
    }
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
