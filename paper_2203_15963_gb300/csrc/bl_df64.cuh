// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two floats
// with |lo| <= ulp(hi)/2, giving a ~48-bit significand from FP32 instructions. On GB300 an
// SM issues 128 FP32 lane-operations per cycle against 2 FP64 ones, so df64 evaluates the
// geodesic right-hand side several times faster than native double at ~1e-14 relative
// rounding. Algorithms (error-free transformations):
//   TwoSum      Knuth, TAOCP vol. 2, 4.2.2 -- s + e = a + b exactly, no branch;
//   Fast2Sum    Dekker 1971 -- s + e = a + b exactly when |a| >= |b|;
//   TwoProd     with FMA: p = a b, e = fma(a, b, -p), p + e = a b exactly;
//   double-length addition (Dekker 1971) and the FMA product of double-words (Joldes,
//   Muller & Popescu 2017, "Tight and rigorous error bounds for basic building blocks of
//   double-word arithmetic", structure of their Alg. 12);
//   1/x and 1/sqrt(x): a Newton step to second order from the hardware float approximation,
//   with the residual formed exactly by FMAs (the refinement used for double-word
//   reciprocals, e.g. in Hida, Li & Bailey's QD library).
#pragma once
#include <cuda_runtime.h>

namespace bl {

// The df64 overloads of sqrt, rsqrt and fabs below would hide the global float/double ones
// inside this namespace; bring those into scope explicitly.
using ::fabs;
using ::rsqrt;
using ::sqrt;

struct __align__(8) df64 {
    float hi, lo;
    __host__ __device__ constexpr df64() : hi(0.0f), lo(0.0f) {}
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // exact split of a double into two floats (rounded to ~48 bits)
    __host__ __device__ constexpr explicit df64(double d)
        : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr explicit df64(int i) : hi((float)i), lo(0.0f) {}
    __host__ __device__ constexpr explicit df64(float f) : hi(f), lo(0.0f) {}
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df64(s, e);
}
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return df64(s, b - (s - a));
}
__device__ __forceinline__ df64 df_two_prod(float a, float b) {
    const float p = a * b;
    return df64(p, fmaf(a, b, -p));
}

// Addition: TwoSum of the high parts, the low parts added in float, one renormalisation
// (Dekker's double-length addition). Its relative error is ~2^-48 except where x and y
// nearly cancel; in the integrator such cancellation only occurs in the embedded error
// estimate, which steers the step size and tolerates it.
__device__ __forceinline__ df64 operator+(const df64& x, const df64& y) {
    df64 s = df_two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(const df64& x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(const df64& x, const df64& y) { return x + (-y); }
__device__ __forceinline__ df64 operator*(const df64& x, const df64& y) {
    df64 p = df_two_prod(x.hi, y.hi);
    p.lo = fmaf(x.hi, y.lo, p.lo);
    p.lo = fmaf(x.lo, y.hi, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}
// x y without the final renormalisation: (p, e) with p the rounded product and |e| about one
// ulp of p, valid as an operand of a further product or sum (used inside product chains)
__device__ __forceinline__ df64 df_mul_nn(const df64& x, const df64& y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return df64(p, e);
}
__device__ __forceinline__ df64 df_mul_f(const df64& x, float b) {
    df64 p = df_two_prod(x.hi, b);
    p.lo = fmaf(x.lo, b, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}
// 1/x: hardware FP32 seed y0 (~1 ulp), residual e = 1 - x y0 formed with FMAs (the product
// x.hi y0 is exact inside the first one), then 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + ...)
// to second order; relative error ~5e-14.
__device__ __forceinline__ df64 rcp(const df64& x) {
    const float y0 = __fdividef(1.0f, x.hi);
    float e = fmaf(-x.hi, y0, 1.0f);
    e = fmaf(-x.lo, y0, e);
    const float t = fmaf(e, e, e);
    return df_fast_two_sum(y0, __fmul_rn(y0, t));
}
__device__ __forceinline__ df64 operator/(const df64& x, const df64& y) { return x * rcp(y); }
// 1/sqrt(x): hardware FP32 seed y0 (~1 ulp), residual u = x y0^2 - 1 formed with an exact
// product (p + ep = x.hi y0) and FMAs, then 1/sqrt(x) = y0 (1 + u)^(-1/2) =
// y0 (1 - u/2 + 3 u^2 / 8 - ...) to second order; relative error ~7e-14.
__device__ __forceinline__ df64 rsqrt(const df64& x) {
    const float y0 = rsqrtf(x.hi);
    const float p = __fmul_rn(x.hi, y0);
    const float ep = fmaf(x.hi, y0, -p);
    float u = fmaf(p, y0, -1.0f);
    u = fmaf(ep, y0, u);
    u = fmaf(x.lo * y0, y0, u);
    const float t = u * fmaf(0.375f, u, -0.5f);
    return df_fast_two_sum(y0, __fmul_rn(y0, t));
}
__device__ __forceinline__ df64 sqrt(const df64& x) {
    if (x.hi <= 0.0f) return df64(0.0f, 0.0f);
    return x * rsqrt(x);
}
// Dot product sum_j a_j x_j of double-float operands without renormalising after each term:
// the high parts of the products are added with TwoSum, and every rounding error and low-order
// cross product goes into one float; one Fast2Sum at the end returns the double-float result.
// This is the compensated dot product Dot2 of Ogita, Rump & Oishi (2005, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, Algorithm 5.3) with the operands' low words folded into the
// error term; its error is of order eps^2 sum_j |a_j x_j|, as for sums of double-float
// products, in 12 FP32 instructions a term instead of 18. The rounded product and the TwoSum
// use the _rn intrinsics, which the compiler never fuses into an FMA.
struct DFDot {
    float s, c;
    __device__ __forceinline__ void first(const df64& a, const df64& x) {
        s = __fmul_rn(a.hi, x.hi);
        c = fmaf(a.hi, x.hi, -s);
        c = fmaf(a.hi, x.lo, c);
        c = fmaf(a.lo, x.hi, c);
    }
    __device__ __forceinline__ void add(const df64& a, const df64& x) {
        const float p = __fmul_rn(a.hi, x.hi);
        float q = fmaf(a.hi, x.hi, -p);
        q = fmaf(a.hi, x.lo, q);
        q = fmaf(a.lo, x.hi, q);
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
        s = t;
        c += e + q;
    }
    // adds a double-float term (not a product): its high word through TwoSum, its low word
    // to the error term
    __device__ __forceinline__ void add_term(const df64& t) {
        const float u = __fadd_rn(s, t.hi);
        const float z = __fsub_rn(u, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(u, z)), __fsub_rn(t.hi, z));
        s = u;
        c += e + t.lo;
    }
    __device__ __forceinline__ df64 get() const { return df_fast_two_sum(s, c); }
    // y + h (s + c) in one pass (no renormalisation of the sum first): the product's high part
    // enters a TwoSum with y.hi, everything else the low word, one Fast2Sum at the end
    __device__ __forceinline__ df64 axpy(const df64& h, const df64& y) const {
        const float p = __fmul_rn(h.hi, s);
        float q = fmaf(h.hi, s, -p);
        q = fmaf(h.hi, c, q);
        q = fmaf(h.lo, s, q);
        const float t = __fadd_rn(y.hi, p);
        const float z = __fsub_rn(t, y.hi);
        const float e = __fadd_rn(__fsub_rn(y.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
        return df_fast_two_sum(t, y.lo + q + e);
    }
};

// x 2^k for a double-float x: exact, both words scaled (k a small integer power of two in f)
__device__ __forceinline__ df64 df_scale(const df64& x, float f) { return df64(x.hi * f, x.lo * f); }

__device__ __forceinline__ df64& operator+=(df64& x, const df64& y) { x = x + y; return x; }
__device__ __forceinline__ df64& operator-=(df64& x, const df64& y) { x = x - y; return x; }
__device__ __forceinline__ df64& operator*=(df64& x, const df64& y) { x = x * y; return x; }
__device__ __forceinline__ bool operator<(const df64& x, const df64& y) {
    return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}
__device__ __forceinline__ bool operator>(const df64& x, const df64& y) { return y < x; }
__device__ __forceinline__ df64 fabs(const df64& x) { return x.hi < 0.0f ? -x : x; }
__device__ __forceinline__ double df_to_double(const df64& x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ df64 df_from_double(double d) { return df64(d); }

}  // namespace bl
