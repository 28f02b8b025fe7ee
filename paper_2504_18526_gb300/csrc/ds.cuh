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

#include <type_traits>

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

// ---- FP32 <-> FP64 and double-single conversions on the integer pipe -------
// On GB300 the F2F conversion instructions issue on the FP64 unit, which runs
// at 1/64 of the FP32 rate and is the limiting unit of the sweep kernels.
// These forms assemble the IEEE-754 binary32/binary64 bit patterns (sign,
// biased exponent: 127 vs 1023, fraction: 23 vs 52 bits) with integer
// instructions; values outside the fast path's exponent range (zeros,
// subnormals, infinities, NaNs, extreme magnitudes) take the hardware
// conversion.

// float -> double (exact)
__device__ __forceinline__ double f2d_int(float f) {
    const unsigned u = __float_as_uint(f), mag = u & 0x7FFFFFFFu;
    if (mag - 0x00800000u < 0x7F000000u) {                       // binary32 normal
        const unsigned hi = (u & 0x80000000u) | ((mag >> 3) + 0x38000000u);   // exponent + (1023 - 127)
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    if (mag == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
}

// double -> float, rounded to nearest (ties to even)
__device__ __forceinline__ float d2f_int(double d) {
    const unsigned H = (unsigned)__double2hiint(d), L = (unsigned)__double2loint(d);
    const unsigned E = (H >> 20) & 0x7FFu;
    if (E - 897u < 254u) {                                       // result exponent 1..254 before rounding
        const unsigned m = __funnelshift_l(L, (H & 0x7FFFFFFFu) - 0x38000000u, 3);   // exponent|fraction, truncated
        const unsigned rest = L & 0x1FFFFFFFu;                   // the 29 dropped fraction bits
        const unsigned up = (rest > 0x10000000u) | ((rest == 0x10000000u) & m);
        return __uint_as_float((H & 0x80000000u) | (m + up));   // a carry moves into the exponent
    }
    return __double2float_rn(d);
}

// double -> double-single: hi = d truncated to 24 significand bits, lo = the
// remainder d - hi (29 bits) truncated to 24; |lo| < ulp(hi), and hi + lo is
// within 2^-47 |d| of d.  Fast path for 2^-74 <= |d| < 2^128.
__device__ __forceinline__ dsf ds_from_double_int(double d) {
    const unsigned H = (unsigned)__double2hiint(d), L = (unsigned)__double2loint(d);
    const unsigned E = (H >> 20) & 0x7FFu;
    if (E - 949u < 202u) {
        const unsigned s = H & 0x80000000u;
        const float hi = __uint_as_float(s | __funnelshift_l(L, (H & 0x7FFFFFFFu) - 0x38000000u, 3));
        const unsigned r = L & 0x1FFFFFFFu;
        float lo = __uint_as_float(s);
        if (r != 0u) {
            // r * 2^(E - 1075) with its leading one at bit 31 - c of r
            const unsigned c = (unsigned)__clz((int)r);
            const unsigned n = r << c;
            lo = __uint_as_float(s | ((E - 917u - c) << 23) | ((n >> 8) & 0x7FFFFFu));
        }
        return dsf(hi, lo);
    }
    return dsf(d);
}

// double-single -> double: the two exact widenings and one FP64 add
__device__ __forceinline__ double ds_to_double_int(dsf a) { return f2d_int(a.hi) + f2d_int(a.lo); }

// conversions between FP64 and the arithmetic type V of an operator evaluation
template <class V>
__device__ __forceinline__ V to_v(double d) {
    if constexpr (std::is_same<V, float>::value) return d2f_int(d);
    else if constexpr (std::is_same<V, dsf>::value) return ds_from_double_int(d);
    else return d;
}
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f2d_int(v); }
__device__ __forceinline__ double to_f64(dsf v) { return ds_to_double_int(v); }

}  // namespace sisdc
