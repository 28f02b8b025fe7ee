// Double-single ("float-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, which carries about 48 significand bits.  The
// operations are built from error-free transformations: Knuth's TwoSum
// (a + b = s + e exactly) and the FMA-based product (a b = p + e exactly with
// e = fma(a, b, -p)); addition adds the low parts to the TwoSum error before
// renormalising, as in Dekker's 1971 construction.  Absolute rounding errors
// are about 2^-48 of the operands' magnitude, so cancellation behaves as in a
// 48-bit floating-point format.
//
// Used by the mixed-precision form for the explicit operator evaluations
// (convective operator and L u): on GB300 the FP32 pipe issues 64 times more
// operations per clock than the FP64 pipe.
#pragma once
#include <cuda_runtime.h>

namespace sisdc {

// keep the FP32/FP64 overloads visible next to the dsf ones declared below
using ::fabs;
using ::fmax;

struct dsf {
    float hi, lo;
    dsf() = default;
    __host__ __device__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
    // nearest FP32 pair of a double (FP64 subtraction, exact: hi carries the
    // leading 24 bits, the remainder fits the double's precision)
    __host__ __device__ constexpr explicit dsf(double d)
        : hi(static_cast<float>(d)), lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
    __host__ __device__ constexpr explicit dsf(int i) : hi(static_cast<float>(i)), lo(0.0f) {}
    __host__ __device__ explicit operator double() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

__device__ __forceinline__ dsf ds_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dsf(s, e);
}

// |a| >= |b| or a == 0
__device__ __forceinline__ dsf ds_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dsf(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dsf operator+(dsf a, dsf b) {
    const dsf s = ds_two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ds_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.hi, -a.lo); }
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }

__device__ __forceinline__ dsf operator*(dsf a, dsf b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);              // exact error of the leading product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ds_fast_two_sum(p, e);
}

__device__ __forceinline__ dsf& operator+=(dsf& a, dsf b) { return a = a + b; }
__device__ __forceinline__ dsf& operator-=(dsf& a, dsf b) { return a = a - b; }
__device__ __forceinline__ dsf& operator*=(dsf& a, dsf b) { return a = a * b; }
__device__ __forceinline__ bool operator==(dsf a, dsf b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator>(dsf a, dsf b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

__device__ __forceinline__ dsf fabs(dsf a) { return (a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f)) ? -a : a; }
__device__ __forceinline__ dsf fmax(dsf a, dsf b) { return b > a ? b : a; }

}  // namespace sisdc
