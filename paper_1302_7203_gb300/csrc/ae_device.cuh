// ae_device.cuh -- device arithmetic for the arrowhead eigen-solver (sm_103a).
//
// * rcp(): FP64 reciprocal by one third-order Newton-Raphson step
//   r1 = r0 (1 + e + e^2), e = 1 - x r0, seeded by the PTX instruction
//   rcp.approx.ftz.f64.  If r0 has relative error e0 then r1 has e0^3 before
//   the final rounding, so a seed good to ~2^-20 gives a faithful result.
//   Tested against IEEE division by the GPU test suite (ae_debug_rcp).
// * Double-double ("doubled working precision", Sec. 4 of the paper) from
//   error-free transformations: TwoSum (Knuth), FastTwoSum (Dekker) and
//   TwoProd by fused multiply-add.  Inputs are binary doubles padded with a
//   zero tail, which is the "binary input" reading of Sec. 4.1.
// * Deterministic warp reductions (xor butterflies: every lane ends with the
//   bit-identical value, independent of scheduling).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ae {

constexpr unsigned FULL = 0xffffffffu;
constexpr double TWO_EPS = 4.440892098500626e-16;   // 2 * 2^-52, Algorithm 3's stop

__device__ __forceinline__ double rcp_seed(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

__device__ __forceinline__ double rcp(double x) {
    double r = rcp_seed(x);
    double e = fma(-x, r, 1.0);
    e = fma(e, e, e);
    return fma(r, e, r);
}

// 1.0 held in a register: FP64 FMAs that take a constant-bank operand run at
// a lower rate than ones on registers alone
static __device__ double g_unit = 1.0;
__device__ __forceinline__ double unit_reg() { return __ldcg(&g_unit); }

__device__ __forceinline__ double rcp_o(double x, double one) {
    double r = rcp_seed(x);
    double e = fma(-x, r, one);
    e = fma(e, e, e);
    return fma(r, e, r);
}

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}

// TwoSum by magnitude order: FastTwoSum with the larger operand first yields
// the same exact error term as TwoSum, in three floating-point operations
// plus one comparison and two selects.
__device__ __forceinline__ dd two_sum_ord(double a, double b) {
    const bool o = fabs(a) >= fabs(b);
    const double x = o ? a : b, y = o ? b : a;
    const double s = x + y;
    return {s, y - (s - x)};
}

// Compensated accumulation of same-sign double-double terms (Sum2 of Ogita,
// Rump and Oishi, with the error-free TwoSum on the running sum): hi is the
// plain sum, lo collects the exact rounding errors and the terms' tails.  The
// caller renormalises every few terms, which keeps |lo| <= k eps |hi| and the
// result within O(n k eps^2) of the exact sum.
__device__ __forceinline__ void csum_add(dd &acc, dd t) {
    const dd s = two_sum_ord(acc.hi, t.hi);
    acc.hi = s.hi;
    acc.lo += s.lo + t.lo;
}

__device__ __forceinline__ dd two_prod(double a, double b) {
    double p = a * b;
    return {p, fma(a, b, -p)};
}

// accurate sum of two double-double numbers
__device__ __forceinline__ dd dd_add(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

// sum of two double-doubles of the same sign (no cancellation possible)
__device__ __forceinline__ dd dd_add_same(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dd dd_mul(dd x, dd y) {
    dd p = two_prod(x.hi, y.hi);
    p.lo = fma(x.hi, y.lo, fma(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_mul_d(dd x, double b) {
    dd p = two_prod(x.hi, b);
    p.lo = fma(x.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_sqrt(dd x) {
    if (!(x.hi > 0.0)) return {0.0, 0.0};
    const double s = sqrt(x.hi);
    const dd r = dd_add(x, dd_neg(two_prod(s, s)));
    return fast_two_sum(s, r.hi / (2.0 * s));
}

// x / y with two partial quotients; the FMA residual x.hi - q1 y.hi is
// (nearly) exact because q1 is within an ulp of the quotient
__device__ __forceinline__ dd dd_div(dd x, dd y) {
    double r = rcp(y.hi);
    double q1 = x.hi * r;
    double res = fma(-q1, y.hi, x.hi);
    res = res + x.lo - q1 * y.lo;
    double q2 = res * r;
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ dd warp_sum_dd(dd v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dd w = {__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
        v = dd_add(v, w);
    }
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// atomic max of a nonnegative double through its bit pattern
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
    if (!(v >= 0.0)) return;
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace ae
